// Internal declarations of the surrogate network's CUDA kernels (surrogate_kernels.cu),
// used by the model runtime (surrogate_capi.cpp). Activations are float32 [batch][C][L]
// (or [batch][features]); weights are read as bfloat16; every reduction runs in a fixed
// order, so results are bitwise reproducible.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>

namespace sgk {

using bf16 = __nv_bfloat16;

// How the products run. kind 0: warp-level mma.sync, 128/256 x 64 tiles. kind 1: tcgen05 with
// the accumulator in tensor memory, 128 x 128 tiles. Both round the operands to bfloat16
// (nearest even) and accumulate in float32. err: a device word that a kind-1 product sets to 1
// when one of its bounded waits for the tensor cores runs out (required for kind 1).
// pack: device scratch of pack_bytes for the convolutions' packed weights (kind 1; at least
// conv_pack_bytes of every layer).
struct Products {
  int kind = 1;
  int* err = nullptr;
  int stall_test = 0;  // 1: every kind-1 product waits for a phase nothing completes (tests the limit)
  bf16* pack = nullptr;
  size_t pack_bytes = 0;
  float* red = nullptr;   // scratch of red_floats for the bias gradients' per-slice sums
  size_t red_floats = 0;
  size_t ws_floats = 0;   // capacity of the split-K workspace a call receives (splits are clamped to it)
};
// Bytes of the packed weights of a convolution with Ci input and Co output channels.
size_t conv_pack_bytes(int Ci, int Co);

// Split-K workspace need (floats) of the weight-gradient products for an M x N result.
size_t splitk_floats(int M, int N, int K);

// Y = act(X W^T + b): X [B][K], W [N][K] (bf16), pre/out [B][N]; out may alias nothing.
int linear_forward(int B, int K, int N, const float* X, const bf16* W, const float* bias, float* pre, float* out,
                   bool gelu, const Products& pr, cudaStream_t s);
// dX [B][K] = dZ [B][N] W [N][K]; split over N through ws (splitk_floats(B, K, N)) when given
int linear_backward_data(int B, int K, int N, const float* dZ, const bf16* W, float* dX, float* ws,
                         const Products& pr, cudaStream_t s);
// dW [N][K] = dZ^T X; db [N] = column sums of dZ
int linear_backward_weight(int B, int K, int N, const float* dZ, const float* X, float* dW, float* db, float* ws,
                           const Products& pr, cudaStream_t s);

// Width-3 'same' convolution of the input upsampled by `up` along time:
// pre[b][o][t] = bias[o] + sum_{c,d} W[o][c][d] X[b][c][(t + d - 1) / up] (zero outside),
// t < L = Lin * up; out = gelu(pre) when out != nullptr. Kind 1 runs its own tcgen05 kernel
// (the input window staged once for the three taps), kind 0 the generic product.
int conv_forward(int B, int Ci, int Co, int Lin, int up, const float* X, const bf16* W, const float* bias,
                 float* pre, float* out, const Products& pr, cudaStream_t s);
// dX [B][Ci][Lin] from dZ [B][Co][L] (the upsampling adjoint sums the repeated samples)
int conv_backward_data(int B, int Ci, int Co, int Lin, int up, const float* dZ, const bf16* W, float* dX,
                       const Products& pr, cudaStream_t s);
// dW [Co][Ci][3] and db [Co]
int conv_backward_weight(int B, int Ci, int Co, int Lin, int up, const float* dZ, const float* X, float* dW,
                         float* db, float* ws, const Products& pr, cudaStream_t s);

// dz[i] *= gelu'(pre[i])
int gelu_backward(size_t n, const float* pre, float* dz, cudaStream_t s);
// dy = 2 (y - t) / n; partials[kLossBlocks] = per-block sums of (y - t)^2 in float64
constexpr int kLossBlocks = 608;
int mse_grad(size_t n, const float* y, const float* t, float* dy, double* partials, cudaStream_t s);
// Adam on n master parameters, then the bf16 mirror
int adam_update(size_t n, float* p, const float* g, float* m, float* v, bf16* pb, float lr, float beta1, float beta2,
                float eps, float inv_c1, float inv_c2, cudaStream_t s);
int to_bf16(size_t n, const float* p, bf16* pb, cudaStream_t s);
// y [B][C][L] = sum_k x[b][in_dim - K + k] D[b][k*C + c][t], and its adjoint in D
int contract_forward(int B, int K, int C, int L, int in_dim, const float* x, const float* D, float* y, cudaStream_t s);
int contract_backward(int B, int K, int C, int L, int in_dim, const float* x, const float* dy, float* dD,
                      cudaStream_t s);

}  // namespace sgk
