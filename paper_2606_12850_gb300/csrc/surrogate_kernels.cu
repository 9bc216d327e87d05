// CUDA kernels of the seismogram surrogate (sm_103a): one tiled float32 product kernel whose
// operand loaders express the dense layers, the width-3 convolutions (with nearest
// upsampling folded into the index map) and their backward products; bias, activation,
// loss and Adam kernels. Weights are read as bfloat16 and widened to float32; every sum is
// accumulated in float32 in a fixed order (split-K partial sums are added in split order).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "surrogate_internal.h"

namespace sgk {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, GT = 256;
constexpr float kGeluC = 0.7978845608028654f;  // sqrt(2 / pi)
constexpr float kGeluA = 0.044715f;

__device__ __forceinline__ float gelu(float x) {
  return 0.5f * x * (1.f + tanhf(kGeluC * (x + kGeluA * x * x * x)));
}
__device__ __forceinline__ float gelu_grad(float x) {
  const float t = tanhf(kGeluC * (x + kGeluA * x * x * x));
  return 0.5f * (1.f + t) + 0.5f * x * (1.f - t * t) * kGeluC * (1.f + 3.f * kGeluA * x * x);
}

// C[m][n] = sum_k A(m, k) B(k, n) over k in this CTA's split; A and B are loader functors
// (kAlong: which index is contiguous in memory, so that consecutive threads load
// consecutive words), EP the epilogue, or a split-K partial into ws[z][M][N].
template <class LA, class LB, class EP>
__global__ void __launch_bounds__(GT) gemm_kernel(int M, int N, int K, int kchunk, LA la, LB lb, EP ep, float* ws) {
  __shared__ float As[BK][BM + 4];
  __shared__ float Bs[BK][BN + 4];
  const int tid = threadIdx.x;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int tm = (tid >> 4) * 4, tn = (tid & 15) * 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int r = 0; r < BM * BK / GT; ++r) {
      const int idx = tid + r * GT;
      const int kk = LA::kAlongK ? idx % BK : idx / BM;
      const int mm = LA::kAlongK ? idx / BK : idx % BM;
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < kend) ? la(m, k) : 0.f;
    }
#pragma unroll
    for (int r = 0; r < BN * BK / GT; ++r) {
      const int idx = tid + r * GT;
      const int nn = LB::kAlongN ? idx % BN : idx / BK;
      const int kk = LB::kAlongN ? idx / BN : idx % BK;
      const int n = n0 + nn, k = k0 + kk;
      Bs[kk][nn] = (n < N && k < kend) ? lb(k, n) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tm + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tn + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + tm + i, n = n0 + tn + j;
      if (m < M && n < N) {
        if (ws)
          ws[(static_cast<size_t>(blockIdx.z) * M + m) * N + n] = acc[i][j];
        else
          ep(m, n, acc[i][j]);
      }
    }
}

template <class EP>
__global__ void splitk_finalize_kernel(int M, int N, int splits, const float* __restrict__ ws, EP ep) {
  const size_t total = static_cast<size_t>(M) * N;
  for (size_t idx = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<size_t>(gridDim.x) * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += ws[static_cast<size_t>(z) * total + idx];
    ep(static_cast<int>(idx / N), static_cast<int>(idx % N), s);
  }
}

int grid_for(size_t n) {
  const size_t g = (n + 255) / 256;
  return static_cast<int>(g < 1 ? 1 : (g > 65535 * 16 ? 65535 * 16 : g));
}

int splits_for(int M, int N, int K) {
  const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  int s = (608 + tiles - 1) / tiles;
  const int kmax = (K + 255) / 256;
  if (s > kmax) s = kmax;
  if (s > 64) s = 64;
  return s < 1 ? 1 : s;
}

template <class LA, class LB, class EP>
int run_gemm(int M, int N, int K, LA la, LB lb, EP ep, float* ws, bool allow_split, cudaStream_t s) {
  if (M <= 0 || N <= 0) return 0;
  const int splits = (allow_split && ws) ? splits_for(M, N, K) : 1;
  int kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + BK - 1) / BK * BK;
  const int used = K > 0 ? (K + kchunk - 1) / kchunk : 1;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, used);
  gemm_kernel<<<grid, GT, 0, s>>>(M, N, K, kchunk, la, lb, ep, used > 1 ? ws : nullptr);
  if (used > 1)
    splitk_finalize_kernel<<<grid_for(static_cast<size_t>(M) * N), 256, 0, s>>>(M, N, used, ws, ep);
  return static_cast<int>(cudaGetLastError());
}

// ---- loaders ------------------------------------------------------------------------------
struct RowMajorA {  // A(m, k) = P[m * ld + k]
  static constexpr bool kAlongK = true;
  const float* P;
  int ld;
  __device__ float operator()(int m, int k) const { return P[static_cast<size_t>(m) * ld + k]; }
};
struct ColMajorA {  // A(m, k) = P[k * ld + m]
  static constexpr bool kAlongK = false;
  const float* P;
  int ld;
  __device__ float operator()(int m, int k) const { return P[static_cast<size_t>(k) * ld + m]; }
};
struct RowMajorB {  // B(k, n) = P[k * ld + n]
  static constexpr bool kAlongN = true;
  const float* P;
  int ld;
  __device__ float operator()(int k, int n) const { return P[static_cast<size_t>(k) * ld + n]; }
};
struct WeightRowB {  // B(k, n) = W[k * ld + n], bf16
  static constexpr bool kAlongN = true;
  const bf16* W;
  int ld;
  __device__ float operator()(int k, int n) const { return __bfloat162float(W[static_cast<size_t>(k) * ld + n]); }
};
struct WeightColB {  // B(k, n) = W[n * ld + k], bf16
  static constexpr bool kAlongN = false;
  const bf16* W;
  int ld;
  __device__ float operator()(int k, int n) const { return __bfloat162float(W[static_cast<size_t>(n) * ld + k]); }
};
struct ConvWeightA {  // A(o, k) = W[o][k], k = c * 3 + d
  static constexpr bool kAlongK = true;
  const bf16* W;
  int ld;
  __device__ float operator()(int m, int k) const { return __bfloat162float(W[static_cast<size_t>(m) * ld + k]); }
};
struct ConvInputB {  // B(k = c*3+d, n = b*L+t) = X[b][c][(t + d - 1) / up], zero outside [0, L)
  static constexpr bool kAlongN = true;
  const float* X;
  int Ci, Lin, L, up;
  __device__ float operator()(int k, int n) const {
    const int c = k / 3, d = k - 3 * c;
    const int b = n / L, t = n - b * L;
    const int sidx = t + d - 1;
    if (sidx < 0 || sidx >= L) return 0.f;
    return X[(static_cast<size_t>(b) * Ci + c) * Lin + sidx / up];
  }
};
struct ConvWeightTA {  // A(c, k = (o*3+d)*up + r) = W[o][c][d]
  static constexpr bool kAlongK = false;
  const bf16* W;
  int Ci, up;
  __device__ float operator()(int m, int k) const {
    const int od = k / up;
    const int o = od / 3, d = od - 3 * o;
    return __bfloat162float(W[(static_cast<size_t>(o) * Ci + m) * 3 + d]);
  }
};
struct ConvGradB {  // B(k = (o*3+d)*up + r, n = b*Lin + t') = dZ[b][o][up t' + r - d + 1]
  static constexpr bool kAlongN = true;
  const float* dZ;
  int Co, Lin, L, up;
  __device__ float operator()(int k, int n) const {
    const int od = k / up, r = k - od * up;
    const int o = od / 3, d = od - 3 * o;
    const int b = n / Lin, tp = n - b * Lin;
    const int t = up * tp + r - d + 1;
    if (t < 0 || t >= L) return 0.f;
    return dZ[(static_cast<size_t>(b) * Co + o) * L + t];
  }
};
struct ConvGradA {  // A(o, k = b*L + t) = dZ[b][o][t]
  static constexpr bool kAlongK = true;
  const float* dZ;
  int Co, L;
  __device__ float operator()(int m, int k) const {
    const int b = k / L, t = k - b * L;
    return dZ[(static_cast<size_t>(b) * Co + m) * L + t];
  }
};
struct ConvInputWB {  // B(k = b*L + t, n = c*3 + d) = X[b][c][(t + d - 1) / up]
  static constexpr bool kAlongN = false;
  const float* X;
  int Ci, Lin, L, up;
  __device__ float operator()(int k, int n) const {
    const int b = k / L, t = k - b * L;
    const int c = n / 3, d = n - 3 * c;
    const int sidx = t + d - 1;
    if (sidx < 0 || sidx >= L) return 0.f;
    return X[(static_cast<size_t>(b) * Ci + c) * Lin + sidx / up];
  }
};

// ---- epilogues ----------------------------------------------------------------------------
struct LinearEp {  // (m = b, n = j)
  float* pre;
  float* out;
  const float* bias;
  int N;
  bool act;
  __device__ void operator()(int m, int n, float v) const {
    const float p = v + bias[n];
    const size_t i = static_cast<size_t>(m) * N + n;
    pre[i] = p;
    if (out) out[i] = act ? gelu(p) : p;
  }
};
struct StoreEp {  // C[m][n]
  float* C;
  int N;
  __device__ void operator()(int m, int n, float v) const { C[static_cast<size_t>(m) * N + n] = v; }
};
struct ConvEp {  // (m = o, n = b*L + t)
  float* pre;
  float* out;
  const float* bias;
  int Co, L;
  __device__ void operator()(int m, int n, float v) const {
    const int b = n / L, t = n - b * L;
    const float p = v + bias[m];
    const size_t i = (static_cast<size_t>(b) * Co + m) * L + t;
    pre[i] = p;
    if (out) out[i] = gelu(p);
  }
};
struct ConvDataEp {  // (m = c, n = b*Lin + t')
  float* dX;
  int Ci, Lin;
  __device__ void operator()(int m, int n, float v) const {
    const int b = n / Lin, tp = n - b * Lin;
    dX[(static_cast<size_t>(b) * Ci + m) * Lin + tp] = v;
  }
};

// ---- elementwise and reductions -------------------------------------------------------------
__global__ void column_sums_kernel(int B, int N, const float* __restrict__ dZ, float* __restrict__ db) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += dZ[static_cast<size_t>(b) * N + j];
    db[j] = s;
  }
}

__global__ void channel_sums_kernel(int B, int Co, int L, const float* __restrict__ dZ, float* __restrict__ db) {
  __shared__ float red[256];
  const int o = blockIdx.x;
  float s = 0.f;
  const size_t per = static_cast<size_t>(B) * L;
  for (size_t i = threadIdx.x; i < per; i += blockDim.x) {
    const size_t b = i / L, t = i - b * L;
    s += dZ[(b * Co + o) * L + t];
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[o] = red[0];
}

__global__ void gelu_backward_kernel(size_t n, const float* __restrict__ pre, float* __restrict__ dz) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    dz[i] *= gelu_grad(pre[i]);
}

__global__ void mse_kernel(size_t n, const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ dy,
                           double* __restrict__ partials) {
  __shared__ double red[256];
  const float scale = 2.f / static_cast<float>(n);
  double s = 0.0;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const float e = y[i] - t[i];
    dy[i] = scale * e;
    s += static_cast<double>(e) * e;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void adam_kernel(size_t n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, bf16* __restrict__ pb, float lr, float b1, float b2, float eps,
                            float inv_c1, float inv_c2) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi * inv_c1) / (sqrtf(vi * inv_c2) + eps);
    p[i] = pi;
    pb[i] = __float2bfloat16_rn(pi);
  }
}

// y[b][c][t] = sum_k x[b][k0 + k] D[b][k*C + c][t]   (the output is linear in the last K
// input features: the moment-tensor entries)
__global__ void contract_forward_kernel(int B, int K, int C, int L, int in_dim, int k0, const float* __restrict__ x,
                                        const float* __restrict__ D, float* __restrict__ y) {
  const size_t total = static_cast<size_t>(B) * C * L;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t b = i / (static_cast<size_t>(C) * L);
    const size_t ct = i - b * C * L;
    float s = 0.f;
    for (int k = 0; k < K; ++k) s = fmaf(x[b * in_dim + k0 + k], D[(b * K + k) * C * L + ct], s);
    y[i] = s;
  }
}

// dD[b][k*C + c][t] = x[b][k0 + k] dy[b][c][t]
__global__ void contract_backward_kernel(int B, int K, int C, int L, int in_dim, int k0, const float* __restrict__ x,
                                         const float* __restrict__ dy, float* __restrict__ dD) {
  const size_t total = static_cast<size_t>(B) * K * C * L;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t CL = static_cast<size_t>(C) * L;
    const size_t bk = i / CL, ct = i - bk * CL;
    const size_t b = bk / K, k = bk - b * K;
    dD[i] = x[b * in_dim + k0 + k] * dy[b * CL + ct];
  }
}

__global__ void to_bf16_kernel(size_t n, const float* __restrict__ p, bf16* __restrict__ pb) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    pb[i] = __float2bfloat16_rn(p[i]);
}

}  // namespace

size_t splitk_floats(int M, int N, int K) {
  const int s = splits_for(M, N, K);
  return s > 1 ? static_cast<size_t>(s) * M * N : 0;
}

int linear_forward(int B, int K, int N, const float* X, const bf16* W, const float* bias, float* pre, float* out,
                   bool act, cudaStream_t s) {
  return run_gemm(B, N, K, RowMajorA{X, K}, WeightColB{W, K}, LinearEp{pre, out, bias, N, act}, nullptr, false, s);
}

int linear_backward_data(int B, int K, int N, const float* dZ, const bf16* W, float* dX, cudaStream_t s) {
  return run_gemm(B, K, N, RowMajorA{dZ, N}, WeightRowB{W, K}, StoreEp{dX, K}, nullptr, false, s);
}

int linear_backward_weight(int B, int K, int N, const float* dZ, const float* X, float* dW, float* db, float* ws,
                           cudaStream_t s) {
  int r = run_gemm(N, K, B, ColMajorA{dZ, N}, RowMajorB{X, K}, StoreEp{dW, K}, ws, true, s);
  if (r) return r;
  column_sums_kernel<<<grid_for(N), 256, 0, s>>>(B, N, dZ, db);
  return static_cast<int>(cudaGetLastError());
}

int conv_forward(int B, int Ci, int Co, int Lin, int up, const float* X, const bf16* W, const float* bias,
                 float* pre, float* out, cudaStream_t s) {
  const int L = Lin * up;
  return run_gemm(Co, B * L, Ci * 3, ConvWeightA{W, Ci * 3}, ConvInputB{X, Ci, Lin, L, up},
                  ConvEp{pre, out, bias, Co, L}, nullptr, false, s);
}

int conv_backward_data(int B, int Ci, int Co, int Lin, int up, const float* dZ, const bf16* W, float* dX,
                       cudaStream_t s) {
  const int L = Lin * up;
  return run_gemm(Ci, B * Lin, Co * 3 * up, ConvWeightTA{W, Ci, up}, ConvGradB{dZ, Co, Lin, L, up},
                  ConvDataEp{dX, Ci, Lin}, nullptr, false, s);
}

int conv_backward_weight(int B, int Ci, int Co, int Lin, int up, const float* dZ, const float* X, float* dW,
                         float* db, float* ws, cudaStream_t s) {
  const int L = Lin * up;
  int r = run_gemm(Co, Ci * 3, B * L, ConvGradA{dZ, Co, L}, ConvInputWB{X, Ci, Lin, L, up}, StoreEp{dW, Ci * 3}, ws,
                   true, s);
  if (r) return r;
  channel_sums_kernel<<<Co, 256, 0, s>>>(B, Co, L, dZ, db);
  return static_cast<int>(cudaGetLastError());
}

int gelu_backward(size_t n, const float* pre, float* dz, cudaStream_t s) {
  gelu_backward_kernel<<<grid_for(n), 256, 0, s>>>(n, pre, dz);
  return static_cast<int>(cudaGetLastError());
}

int mse_grad(size_t n, const float* y, const float* t, float* dy, double* partials, cudaStream_t s) {
  mse_kernel<<<kLossBlocks, 256, 0, s>>>(n, y, t, dy, partials);
  return static_cast<int>(cudaGetLastError());
}

int adam_update(size_t n, float* p, const float* g, float* m, float* v, bf16* pb, float lr, float beta1, float beta2,
                float eps, float inv_c1, float inv_c2, cudaStream_t s) {
  adam_kernel<<<grid_for(n), 256, 0, s>>>(n, p, g, m, v, pb, lr, beta1, beta2, eps, inv_c1, inv_c2);
  return static_cast<int>(cudaGetLastError());
}

int contract_forward(int B, int K, int C, int L, int in_dim, const float* x, const float* D, float* y, cudaStream_t s) {
  contract_forward_kernel<<<grid_for(static_cast<size_t>(B) * C * L), 256, 0, s>>>(B, K, C, L, in_dim, in_dim - K, x,
                                                                                  D, y);
  return static_cast<int>(cudaGetLastError());
}

int contract_backward(int B, int K, int C, int L, int in_dim, const float* x, const float* dy, float* dD,
                      cudaStream_t s) {
  contract_backward_kernel<<<grid_for(static_cast<size_t>(B) * K * C * L), 256, 0, s>>>(B, K, C, L, in_dim, in_dim - K,
                                                                                       x, dy, dD);
  return static_cast<int>(cudaGetLastError());
}

int to_bf16(size_t n, const float* p, bf16* pb, cudaStream_t s) {
  to_bf16_kernel<<<grid_for(n), 256, 0, s>>>(n, p, pb);
  return static_cast<int>(cudaGetLastError());
}

}  // namespace sgk
