// CUDA kernels of libsemgb (sm_103a): the matrix-free elastic force kernel with colour-by-
// colour assembly, the Newmark streaming passes, sources/receivers and energy partials.
#include <cuda_runtime.h>

#include <cmath>

#include "sem_internal.h"

namespace semgb {

// Per-NGLL slots so that contexts of different order can coexist in one process.
__constant__ float c_h[kMaxNgll + 1][kMaxNgll * kMaxNgll];   // hprime[i*n + l] = l_l'(xi_i)
__constant__ float c_hw[kMaxNgll + 1][kMaxNgll * kMaxNgll];  // [l*n + i] = w_l * hprime[l][i]
__constant__ float c_w[kMaxNgll + 1][kMaxNgll];

int upload_basis(int n, const double* w, const double* h, void* stream) {
  float hf[kMaxNgll * kMaxNgll], hwf[kMaxNgll * kMaxNgll], wf[kMaxNgll];
  for (int i = 0; i < n; ++i) {
    wf[i] = static_cast<float>(w[i]);
    for (int l = 0; l < n; ++l) {
      hf[i * n + l] = static_cast<float>(h[i * n + l]);
      hwf[l * n + i] = static_cast<float>(w[l] * h[l * n + i]);
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t mat = sizeof(float) * kMaxNgll * kMaxNgll;
  cudaError_t e = cudaMemcpyToSymbolAsync(c_h, hf, sizeof(float) * n * n, mat * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyToSymbolAsync(c_hw, hwf, sizeof(float) * n * n, mat * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyToSymbolAsync(c_w, wf, sizeof(float) * n, sizeof(float) * kMaxNgll * n,
                                cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? 0 : static_cast<int>(e);
}

// ---------------------------------------------------------------------------------------
// Force kernel (Sec. II-B matrix-free stiffness action + Sec. IV-C coloured assembly).
//
// One thread owns one xi-line (j, k) of one element: the NGLL values of u along xi sit in
// its registers, so the xi-derivative and the xi-transposed product need no shared memory;
// the eta and zeta contractions read the element cube that the element's NGLL^2 threads
// stage in shared memory. CTAs hold E = T / NGLL^2 elements. The element record (ibool,
// inverse Jacobian, J, kappa, mu) is read with coalesced loads: for a fixed i the NGLL^2
// line threads of an element read consecutive words. Assembly writes through ibool with
// plain stores or read-modify-writes: elements of one launch share no node.
// ---------------------------------------------------------------------------------------
template <int N>
struct ForceCfg {
  static constexpr int NP = N * N * N;
  static constexpr int NL = N * N;
  static constexpr int T = (N <= 5) ? 128 : 256;
  static constexpr int E = T / NL;
  static constexpr int REC = (kRecFields * NP + 3) / 4 * 4;
  static constexpr int SMEM_FLOATS = E * 9 * NP;
};

template <int N>
__global__ void __launch_bounds__(ForceCfg<N>::T)
    forces_kernel(const float* __restrict__ rec, const float* __restrict__ u, float* __restrict__ f,
                  int e0, int e1) {
  using C = ForceCfg<N>;
  constexpr int NP = C::NP, NL = C::NL, E = C::E, REC = C::REC;
  extern __shared__ float smem[];
  const float* __restrict__ H = c_h[N];
  const float* __restrict__ HW = c_hw[N];
  const float* __restrict__ W = c_w[N];

  const int t = threadIdx.x;
  const int le = t / NL;
  const int line = t - le * NL;  // = j + N k
  const int j = line % N;
  const int k = line / N;
  const int e = e0 + blockIdx.x * E + le;
  const bool in_cta = le < E;
  const bool active = in_cta && e < e1;
  float* su = smem + (in_cta ? le : 0) * 9 * NP;  // u cube [3][NP], index i + N*line
  float* st = su + 3 * NP;                         // eta and zeta fluxes [6][NP]
  const float* __restrict__ r = rec + static_cast<size_t>(active ? e : e0) * REC;

  uint32_t g[N];
  float ux[N], uy[N], uz[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    g[i] = 0u;
    ux[i] = uy[i] = uz[i] = 0.f;
  }
  if (active) {
#pragma unroll
    for (int i = 0; i < N; ++i) g[i] = __float_as_uint(__ldg(r + i * NL + line));
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const size_t gi = 3 * static_cast<size_t>(g[i] & ~kFirstTouchBit);
      ux[i] = __ldg(u + gi);
      uy[i] = __ldg(u + gi + 1);
      uz[i] = __ldg(u + gi + 2);
    }
  }
  if (in_cta) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      su[0 * NP + i + N * line] = ux[i];
      su[1 * NP + i + N * line] = uy[i];
      su[2 * NP + i + N * line] = uz[i];
    }
  }
  __syncthreads();

  float hj[N], hk[N];
#pragma unroll
  for (int l = 0; l < N; ++l) {
    hj[l] = H[j * N + l];
    hk[l] = H[k * N + l];
  }
  float fx[N], fy[N], fz[N];
#pragma unroll
  for (int i = 0; i < N; ++i) fx[i] = fy[i] = fz[i] = 0.f;

#pragma unroll
  for (int i = 0; i < N; ++i) {
    // reference derivatives (Sec. II-B): xi from registers, eta and zeta from the cube
    float dxi_x = 0.f, dxi_y = 0.f, dxi_z = 0.f;
    float det_x = 0.f, det_y = 0.f, det_z = 0.f;
    float dze_x = 0.f, dze_y = 0.f, dze_z = 0.f;
#pragma unroll
    for (int l = 0; l < N; ++l) {
      const float h = H[i * N + l];
      dxi_x += h * ux[l];
      dxi_y += h * uy[l];
      dxi_z += h * uz[l];
      const int pe = i + N * (l + N * k);
      det_x += hj[l] * su[0 * NP + pe];
      det_y += hj[l] * su[1 * NP + pe];
      det_z += hj[l] * su[2 * NP + pe];
      const int pz = i + N * (j + N * l);
      dze_x += hk[l] * su[0 * NP + pz];
      dze_y += hk[l] * su[1 * NP + pz];
      dze_z += hk[l] * su[2 * NP + pz];
    }
    // inverse Jacobian, J and moduli at this point
    const int q = i * NL + line;
    float G[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) G[a] = active ? __ldg(r + (kG + a) * NP + q) : 0.f;
    const float jac = active ? __ldg(r + kJac * NP + q) : 0.f;
    const float kappa = active ? __ldg(r + kKappa * NP + q) : 0.f;
    const float mu = active ? __ldg(r + kMu * NP + q) : 0.f;

    // physical gradient du_c/dx_d
    const float uxx = dxi_x * G[0] + det_x * G[3] + dze_x * G[6];
    const float uxy = dxi_x * G[1] + det_x * G[4] + dze_x * G[7];
    const float uxz = dxi_x * G[2] + det_x * G[5] + dze_x * G[8];
    const float uyx = dxi_y * G[0] + det_y * G[3] + dze_y * G[6];
    const float uyy = dxi_y * G[1] + det_y * G[4] + dze_y * G[7];
    const float uyz = dxi_y * G[2] + det_y * G[5] + dze_y * G[8];
    const float uzx = dxi_z * G[0] + det_z * G[3] + dze_z * G[6];
    const float uzy = dxi_z * G[1] + det_z * G[4] + dze_z * G[7];
    const float uzz = dxi_z * G[2] + det_z * G[5] + dze_z * G[8];

    // isotropic Hooke stress: sigma = lambda tr(eps) I + 2 mu eps, lambda = kappa - 2/3 mu
    const float lam = kappa - (2.f / 3.f) * mu;
    const float tr = uxx + uyy + uzz;
    const float sxx = lam * tr + 2.f * mu * uxx;
    const float syy = lam * tr + 2.f * mu * uyy;
    const float szz = lam * tr + 2.f * mu * uzz;
    const float sxy = mu * (uxy + uyx);
    const float sxz = mu * (uxz + uzx);
    const float syz = mu * (uyz + uzy);

    // fluxes t_{r,c} = J sum_d sigma_cd dxi_r/dx_d
    const float txi_x = jac * (sxx * G[0] + sxy * G[1] + sxz * G[2]);
    const float txi_y = jac * (sxy * G[0] + syy * G[1] + syz * G[2]);
    const float txi_z = jac * (sxz * G[0] + syz * G[1] + szz * G[2]);
    const float tet_x = jac * (sxx * G[3] + sxy * G[4] + sxz * G[5]);
    const float tet_y = jac * (sxy * G[3] + syy * G[4] + syz * G[5]);
    const float tet_z = jac * (sxz * G[3] + syz * G[4] + szz * G[5]);
    const float tze_x = jac * (sxx * G[6] + sxy * G[7] + sxz * G[8]);
    const float tze_y = jac * (sxy * G[6] + syy * G[7] + syz * G[8]);
    const float tze_z = jac * (sxz * G[6] + syz * G[7] + szz * G[8]);

    // xi-transposed product stays in registers: F(i') += w_i hprime[i][i'] t_xi(i)
#pragma unroll
    for (int ip = 0; ip < N; ++ip) {
      const float hw = HW[i * N + ip];
      fx[ip] += hw * txi_x;
      fy[ip] += hw * txi_y;
      fz[ip] += hw * txi_z;
    }
    if (in_cta) {
      const int p = i + N * line;
      st[0 * NP + p] = tet_x;
      st[1 * NP + p] = tet_y;
      st[2 * NP + p] = tet_z;
      st[3 * NP + p] = tze_x;
      st[4 * NP + p] = tze_y;
      st[5 * NP + p] = tze_z;
    }
  }
  __syncthreads();

  float hwj[N], hwk[N];
#pragma unroll
  for (int l = 0; l < N; ++l) {
    hwj[l] = HW[l * N + j];
    hwk[l] = HW[l * N + k];
  }
  const float wj = W[j], wk = W[k];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float ex = 0.f, ey = 0.f, ez = 0.f, zx = 0.f, zy = 0.f, zz = 0.f;
#pragma unroll
    for (int l = 0; l < N; ++l) {
      const int pe = i + N * (l + N * k);
      ex += hwj[l] * st[0 * NP + pe];
      ey += hwj[l] * st[1 * NP + pe];
      ez += hwj[l] * st[2 * NP + pe];
      const int pz = i + N * (j + N * l);
      zx += hwk[l] * st[3 * NP + pz];
      zy += hwk[l] * st[4 * NP + pz];
      zz += hwk[l] * st[5 * NP + pz];
    }
    const float wi = W[i];
    const float Fx = -(wj * wk * fx[i] + wi * wk * ex + wi * wj * zx);
    const float Fy = -(wj * wk * fy[i] + wi * wk * ey + wi * wj * zy);
    const float Fz = -(wj * wk * fz[i] + wi * wk * ez + wi * wj * zz);
    if (active) {
      const size_t gi = 3 * static_cast<size_t>(g[i] & ~kFirstTouchBit);
      if (g[i] & kFirstTouchBit) {
        f[gi] = Fx;
        f[gi + 1] = Fy;
        f[gi + 2] = Fz;
      } else {
        f[gi] += Fx;
        f[gi + 1] += Fy;
        f[gi + 2] += Fz;
      }
    }
  }
}

template <int N>
int launch_forces_n(const float* rec, const float* u, float* f, int e0, int e1, cudaStream_t s) {
  using C = ForceCfg<N>;
  if (e1 <= e0) return 0;
  static unsigned long long attr_done = 0;  // one bit per device ordinal
  const int smem = C::SMEM_FLOATS * static_cast<int>(sizeof(float));
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(attr_done & bit)) {
    cudaError_t e = cudaFuncSetAttribute(forces_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return static_cast<int>(e);
    attr_done |= bit;
  }
  const int grid = (e1 - e0 + C::E - 1) / C::E;
  forces_kernel<N><<<grid, C::T, smem, s>>>(rec, u, f, e0, e1);
  return static_cast<int>(cudaGetLastError());
}

int launch_forces(int n, const float* rec, const float* u, float* f, int e0, int e1, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (n) {
    case 2: return launch_forces_n<2>(rec, u, f, e0, e1, s);
    case 3: return launch_forces_n<3>(rec, u, f, e0, e1, s);
    case 4: return launch_forces_n<4>(rec, u, f, e0, e1, s);
    case 5: return launch_forces_n<5>(rec, u, f, e0, e1, s);
    case 6: return launch_forces_n<6>(rec, u, f, e0, e1, s);
    case 7: return launch_forces_n<7>(rec, u, f, e0, e1, s);
    case 8: return launch_forces_n<8>(rec, u, f, e0, e1, s);
    case 9: return launch_forces_n<9>(rec, u, f, e0, e1, s);
    case 10: return launch_forces_n<10>(rec, u, f, e0, e1, s);
    default: return static_cast<int>(cudaErrorInvalidValue);
  }
}

int forces_kernel_smem_bytes(int n) {
  switch (n) {
    case 2: return ForceCfg<2>::SMEM_FLOATS * 4;
    case 3: return ForceCfg<3>::SMEM_FLOATS * 4;
    case 4: return ForceCfg<4>::SMEM_FLOATS * 4;
    case 5: return ForceCfg<5>::SMEM_FLOATS * 4;
    case 6: return ForceCfg<6>::SMEM_FLOATS * 4;
    case 7: return ForceCfg<7>::SMEM_FLOATS * 4;
    case 8: return ForceCfg<8>::SMEM_FLOATS * 4;
    case 9: return ForceCfg<9>::SMEM_FLOATS * 4;
    case 10: return ForceCfg<10>::SMEM_FLOATS * 4;
    default: return 0;
  }
}

int forces_elements_per_cta(int n) { return n >= 2 && n <= 10 ? ((n <= 5 ? 128 : 256) / (n * n)) : 0; }

// ---------------------------------------------------------------------------------------
// Newmark streaming passes (Sec. I / V-C explicit second-order Newmark, diagonal mass).
// Fields are [nglob_pad][3] float32 with nglob_pad % 4 == 0: a thread owns four nodes,
// i.e. three float4 of each field and one float4 of the inverse mass.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float4 mass_lanes(const float4 m, int part) {
  // the three float4 words of 4 nodes (x0 y0 z0 x1 | y1 z1 x2 y2 | z2 x3 y3 z3)
  return part == 0 ? make_float4(m.x, m.x, m.x, m.y)
                   : (part == 1 ? make_float4(m.y, m.y, m.z, m.z) : make_float4(m.z, m.w, m.w, m.w));
}

// u <- u + dt v + dt^2/2 a ; v <- v + dt/2 a  (first step from a complete state)
__global__ void predictor_kernel(float4* __restrict__ u, float4* __restrict__ v, const float4* __restrict__ a,
                                 int n4, float dt, float hdt, float hdt2) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += gridDim.x * blockDim.x) {
#pragma unroll
    for (int part = 0; part < 3; ++part) {
      const int w = 3 * t + part;
      const float4 av = a[w];
      float4 vv = v[w];
      float4 uv = u[w];
      uv.x += dt * vv.x + hdt2 * av.x;
      uv.y += dt * vv.y + hdt2 * av.y;
      uv.z += dt * vv.z + hdt2 * av.z;
      uv.w += dt * vv.w + hdt2 * av.w;
      vv.x += hdt * av.x;
      vv.y += hdt * av.y;
      vv.z += hdt * av.z;
      vv.w += hdt * av.w;
      u[w] = uv;
      v[w] = vv;
    }
  }
}

// Corrector of step n-1 fused with the predictor of step n:
//   a = M^-1 a_raw ; v = v_half + dt/2 a ; u += dt v + dt^2/2 a ; v_half = v + dt/2 a
// a_raw is left in place (the next force pass overwrites it).
__global__ void fused_newmark_kernel(float4* __restrict__ u, float4* __restrict__ v,
                                     const float4* __restrict__ a, const float4* __restrict__ minv, int n4,
                                     float dt, float hdt, float hdt2) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += gridDim.x * blockDim.x) {
    const float4 m = minv[t];
#pragma unroll
    for (int part = 0; part < 3; ++part) {
      const int w = 3 * t + part;
      const float4 mm = mass_lanes(m, part);
      const float4 ar = a[w];
      float4 vv = v[w];
      float4 uv = u[w];
      const float ax = ar.x * mm.x, ay = ar.y * mm.y, az = ar.z * mm.z, aw = ar.w * mm.w;
      vv.x += hdt * ax;
      vv.y += hdt * ay;
      vv.z += hdt * az;
      vv.w += hdt * aw;
      uv.x += dt * vv.x + hdt2 * ax;
      uv.y += dt * vv.y + hdt2 * ay;
      uv.z += dt * vv.z + hdt2 * az;
      uv.w += dt * vv.w + hdt2 * aw;
      vv.x += hdt * ax;
      vv.y += hdt * ay;
      vv.z += hdt * az;
      vv.w += hdt * aw;
      u[w] = uv;
      v[w] = vv;
    }
  }
}

// Corrector alone (completes the state): a = M^-1 a_raw ; v = v_half + dt/2 a
__global__ void corrector_kernel(float4* __restrict__ v, float4* __restrict__ a, const float4* __restrict__ minv,
                                 int n4, float hdt) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += gridDim.x * blockDim.x) {
    const float4 m = minv[t];
#pragma unroll
    for (int part = 0; part < 3; ++part) {
      const int w = 3 * t + part;
      const float4 mm = mass_lanes(m, part);
      float4 ar = a[w];
      float4 vv = v[w];
      ar.x *= mm.x;
      ar.y *= mm.y;
      ar.z *= mm.z;
      ar.w *= mm.w;
      vv.x += hdt * ar.x;
      vv.y += hdt * ar.y;
      vv.z += hdt * ar.z;
      vv.w += hdt * ar.w;
      a[w] = ar;
      v[w] = vv;
    }
  }
}

static int stream_grid(int n4) {
  const int per = 256;
  int g = (n4 + per - 1) / per;
  return g < 1 ? 1 : g;
}

int launch_predictor(const DevProblem& p, void* stream) {
  const int n4 = p.nglob_pad / 4;
  predictor_kernel<<<stream_grid(n4), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<float4*>(p.u), reinterpret_cast<float4*>(p.v), reinterpret_cast<const float4*>(p.a), n4,
      static_cast<float>(p.dt), static_cast<float>(0.5 * p.dt), static_cast<float>(0.5 * p.dt * p.dt));
  return static_cast<int>(cudaGetLastError());
}

int launch_fused_newmark(const DevProblem& p, void* stream) {
  const int n4 = p.nglob_pad / 4;
  fused_newmark_kernel<<<stream_grid(n4), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<float4*>(p.u), reinterpret_cast<float4*>(p.v), reinterpret_cast<const float4*>(p.a),
      reinterpret_cast<const float4*>(p.minv), n4, static_cast<float>(p.dt), static_cast<float>(0.5 * p.dt),
      static_cast<float>(0.5 * p.dt * p.dt));
  return static_cast<int>(cudaGetLastError());
}

int launch_corrector(const DevProblem& p, void* stream) {
  const int n4 = p.nglob_pad / 4;
  corrector_kernel<<<stream_grid(n4), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<float4*>(p.v), reinterpret_cast<float4*>(p.a), reinterpret_cast<const float4*>(p.minv), n4,
      static_cast<float>(0.5 * p.dt));
  return static_cast<int>(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------
// Sources and receivers (Sec. V-C): Ricker point forces added to a_raw at t_{n+1}, then the
// displacement u^{n+1} sampled at the receiver nodes; advances the device step counter.
// Source nodes are distinct (the host merges duplicates), so the adds do not race.
// ---------------------------------------------------------------------------------------
__global__ void sources_record_kernel(float* __restrict__ a, const float* __restrict__ u, DevCtl* ctl,
                                      int nsrc, const int* __restrict__ src_node,
                                      const double* __restrict__ src_force, double f0, double t0, double dt,
                                      int nrec, const int* __restrict__ rec_node) {
  const long long n = ctl->step;
  const int col = ctl->col;
  const int ncols = ctl->ncols;
  float* seis = ctl->seis;
  __syncthreads();
  const double tau = static_cast<double>(n + 1) * dt - t0;
  const double x = M_PI * f0 * tau;
  const double aa = x * x;
  const double R = (1.0 - 2.0 * aa) * exp(-aa);
  for (int s = threadIdx.x; s < nsrc; s += blockDim.x) {
    const size_t g = 3 * static_cast<size_t>(src_node[s]);
    a[g] += static_cast<float>(src_force[3 * s] * R);
    a[g + 1] += static_cast<float>(src_force[3 * s + 1] * R);
    a[g + 2] += static_cast<float>(src_force[3 * s + 2] * R);
  }
  if (seis != nullptr && col < ncols) {
    for (int q = threadIdx.x; q < 3 * nrec; q += blockDim.x) {
      const int r = q / 3, c = q - 3 * r;
      seis[static_cast<size_t>(q) * ncols + col] = u[3 * static_cast<size_t>(rec_node[r]) + c];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl->step = n + 1;
    ctl->col = col + 1;
  }
}

__global__ void set_ctl_kernel(DevCtl* ctl, long long step, int ncols, float* seis) {
  ctl->step = step;
  ctl->col = 0;
  ctl->ncols = ncols;
  ctl->seis = seis;
  ctl->err = 0;
}

int launch_set_ctl(DevCtl* ctl, long long step, int ncols, float* seis, void* stream) {
  set_ctl_kernel<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(ctl, step, ncols, seis);
  return static_cast<int>(cudaGetLastError());
}

int launch_sources_record(const DevProblem& p, void* stream) {
  sources_record_kernel<<<1, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      p.a, p.u, p.ctl, p.nsrc, p.src_node, p.src_force, p.f0, p.t0, p.dt, p.nrec, p.rec_node);
  return static_cast<int>(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------
// Energy partial sums: per block, sum_I |v_I|^2 / minv_I and sum_I u_I . f_I in float64.
// ---------------------------------------------------------------------------------------
__global__ void energy_partials_kernel(const float* __restrict__ u, const float* __restrict__ v,
                                       const float* __restrict__ f, const float* __restrict__ minv, int nglob_pad,
                                       double* __restrict__ partials) {
  __shared__ double sk[256], sp[256];
  double kin = 0.0, pot = 0.0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < nglob_pad; g += gridDim.x * blockDim.x) {
    const float m = minv[g];
    if (m > 0.f) {
      const double vx = v[3 * g], vy = v[3 * g + 1], vz = v[3 * g + 2];
      kin += (vx * vx + vy * vy + vz * vz) / static_cast<double>(m);
    }
    pot += static_cast<double>(u[3 * g]) * f[3 * g] + static_cast<double>(u[3 * g + 1]) * f[3 * g + 1] +
           static_cast<double>(u[3 * g + 2]) * f[3 * g + 2];
  }
  sk[threadIdx.x] = kin;
  sp[threadIdx.x] = pot;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sk[threadIdx.x] += sk[threadIdx.x + w];
      sp[threadIdx.x] += sp[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = sk[0];
    partials[2 * blockIdx.x + 1] = sp[0];
  }
}

int launch_energy_partials(const float* u, const float* v, const float* f, const float* minv, int nglob_pad,
                           double* partials, int nblocks, void* stream) {
  energy_partials_kernel<<<nblocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(u, v, f, minv, nglob_pad,
                                                                                   partials);
  return static_cast<int>(cudaGetLastError());
}

}  // namespace semgb
