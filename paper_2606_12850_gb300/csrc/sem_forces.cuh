// Force kernel template of libsemgb, compiled once per NGLL: each sem_forces_<N>.cu
// defines SEM_NGLL and includes this file, so the orders build in parallel and every
// translation unit owns the constant-memory copy of its 1D basis.
#pragma once
#include <cuda_runtime.h>

#include "sem_internal.h"

#define SEM_CAT2(a, b) a##b
#define SEM_CAT(a, b) SEM_CAT2(a, b)

#ifndef SEM_NGLL
#error "define SEM_NGLL before including sem_forces.cuh"
#endif

namespace semgb {
namespace {

__constant__ float c_h[SEM_NGLL * SEM_NGLL];   // hprime[i*n + l] = l_l'(xi_i)
__constant__ float c_hw[SEM_NGLL * SEM_NGLL];  // [l*n + i] = w_l * hprime[l][i]
__constant__ float c_w[SEM_NGLL];

// ---------------------------------------------------------------------------------------
// Force kernel (Sec. II-B matrix-free stiffness action + Sec. IV-C coloured assembly),
// optionally fused with the Newmark node update.
//
// Threads work in teams: one warp per team for NGLL <= 5 (then a team only ever needs
// __syncwarp, so warps of a CTA drift freely and hide each other's memory latency), the
// whole CTA for NGLL >= 6. A team holds E = TEAM / NGLL^2 elements of one colour.
//  1. gather, one thread per local point: consecutive threads take consecutive points p,
//     so a warp reads whole xi-rows of the global arrays. At a node's first touch in the
//     colour order the same thread applies the Newmark update of the node (MODE 1:
//     predictor from a complete state; MODE 2: corrector of the previous step, then the
//     predictor), so the step needs no separate pass over the global arrays;
//  2. one thread per xi-line (j, k): the xi-derivative and xi-transposed product stay in
//     registers; eta and zeta derivatives accumulate whole xi-rows of the shared cube,
//     read with 128-bit loads (rows are padded to a multiple of 4 floats); Jacobian map,
//     Hooke stress and fluxes per point;
//  3. eta and zeta transposed products from the shared flux rows, element forces back
//     into the thread's own row;
//  4. scatter in the gather's order: a store at the node's first touch, a
//     read-modify-write otherwise (elements of one launch share no node: no atomics,
//     fixed summation order).
// Shared memory per element: u (then F), eta-flux and zeta-flux as [NGLL^2 rows][RS]
// (row = xi-line, [i][3] inside), ibool as [NP].
// ---------------------------------------------------------------------------------------
template <int N>
struct ForceCfg {
  static constexpr int NP = N * N * N;
  static constexpr int NL = N * N;
  static constexpr bool WARP_TEAM = NL <= 32;
  static constexpr int T = WARP_TEAM ? 128 : 256;     // threads per CTA
  static constexpr int TEAM = WARP_TEAM ? 32 : T;     // threads per team
  static constexpr int TEAMS = T / TEAM;              // teams per CTA
  static constexpr int E = TEAM / NL;                 // elements per team
  static constexpr int EPC = TEAMS * E;               // elements per CTA
  static constexpr int RS = (3 * N + 3) / 4 * 4;      // floats per padded xi-row
  static constexpr int RV = RS / 4;                   // float4 per row
  static constexpr int NPA = (NP + 3) / 4 * 4;
  static constexpr int ES = 3 * NL * RS + NPA + (E > 1 ? 4 : 0);  // floats per element
  static constexpr int TS = E * ES;                   // floats per team
  static constexpr int SMEM_FLOATS = TEAMS * TS;
  static constexpr int REC = (kRecFields * NP + 3) / 4 * 4;
  static constexpr bool LINE_VEC = N <= 7;            // whole-row register accumulation
};

template <bool WARP>
__device__ __forceinline__ void team_sync() {
  if (WARP)
    __syncwarp();
  else
    __syncthreads();
}

template <int N>
__device__ __forceinline__ void load_row(const float* rowp, float (&row)[ForceCfg<N>::RS]) {
  const float4* r4 = reinterpret_cast<const float4*>(rowp);
#pragma unroll
  for (int m = 0; m < ForceCfg<N>::RV; ++m) {
    const float4 q = r4[m];
    row[4 * m] = q.x;
    row[4 * m + 1] = q.y;
    row[4 * m + 2] = q.z;
    row[4 * m + 3] = q.w;
  }
}

#ifndef SEM_FORCES_MIN_BLOCKS
#define SEM_FORCES_MIN_BLOCKS 1
#endif

template <int N, int MODE>
__global__ void __launch_bounds__(ForceCfg<N>::T, SEM_FORCES_MIN_BLOCKS)
    forces_kernel(const float* __restrict__ rec, float* u, float* __restrict__ f, float* __restrict__ v,
                  const float* __restrict__ minv, int e0, int e1, float dt, float hdt, float hdt2) {
  using C = ForceCfg<N>;
  constexpr int NP = C::NP, NL = C::NL, E = C::E, REC = C::REC, TEAM = C::TEAM, ES = C::ES, RS = C::RS;
  constexpr bool WT = C::WARP_TEAM;
  extern __shared__ float4 smem4[];
  const float* __restrict__ H = c_h;
  const float* __restrict__ HW = c_hw;
  const float* __restrict__ W = c_w;

  const int team = threadIdx.x / TEAM;
  const int tl = threadIdx.x - team * TEAM;
  const int ebase = e0 + (blockIdx.x * C::TEAMS + team) * E;
  const int ne = min(E, e1 - ebase);
  if (WT && ne <= 0) return;  // a warp team with no element (never a CTA team)
  float* ts = reinterpret_cast<float*>(smem4) + team * C::TS;

  // 1. gather (+ Newmark at first touch), one thread per local point
  for (int idx = tl; idx < ne * NP; idx += TEAM) {
    const int le = idx / NP;
    const int p = idx - le * NP;
    const int line = p / N;
    const int i = p - line * N;
    float* eb = ts + le * ES;
    const uint32_t w = __float_as_uint(__ldg(rec + static_cast<size_t>(ebase + le) * REC + p));
    reinterpret_cast<uint32_t*>(eb + 3 * NL * RS)[p] = w;
    const size_t g = w & ~kFirstTouchBit;
    float* dst = eb + line * RS + 3 * i;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t gi = 3 * g + c;
      float uu = u[gi];
      if (MODE != 0 && (w & kFirstTouchBit)) {
        float acc = f[gi];
        if (MODE == 2) acc *= minv[g];
        float vv = v[gi];
        if (MODE == 2) vv += hdt * acc;  // corrector of the previous step
        uu += dt * vv + hdt2 * acc;      // predictor
        vv += hdt * acc;
        u[gi] = uu;
        v[gi] = vv;
      }
      dst[c] = uu;
    }
  }
  team_sync<WT>();

  // 2. per xi-line derivatives, stress and fluxes
  const int le = tl / NL;
  const int line = tl - le * NL;  // = j + N k
  const int j = line % N;
  const int k = line / N;
  const bool active = le < ne;
  float* eb = ts + (active ? le : 0) * ES;
  float* rows_u = eb;
  float* rows_te = eb + NL * RS;
  float* rows_tz = eb + 2 * NL * RS;
  const float* __restrict__ r = rec + static_cast<size_t>(ebase + (active ? le : 0)) * REC;

  float fxi[3 * N];
#pragma unroll
  for (int q = 0; q < 3 * N; ++q) fxi[q] = 0.f;
  {
    float uo[RS];
    load_row<N>(rows_u + line * RS, uo);
    float hj[N], hk[N];
#pragma unroll
    for (int l = 0; l < N; ++l) {
      hj[l] = H[j * N + l];
      hk[l] = H[k * N + l];
    }
    float deta[C::LINE_VEC ? 3 * N : 1], dzet[C::LINE_VEC ? 3 * N : 1];
    if (C::LINE_VEC) {
#pragma unroll
      for (int q = 0; q < 3 * N; ++q) deta[q] = dzet[q] = 0.f;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        float row[RS];
        load_row<N>(rows_u + (l + N * k) * RS, row);
#pragma unroll
        for (int q = 0; q < 3 * N; ++q) deta[q] += hj[l] * row[q];
        load_row<N>(rows_u + (j + N * l) * RS, row);
#pragma unroll
        for (int q = 0; q < 3 * N; ++q) dzet[q] += hk[l] * row[q];
      }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
      float dxi_x = 0.f, dxi_y = 0.f, dxi_z = 0.f;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        const float h = H[i * N + l];
        dxi_x += h * uo[3 * l];
        dxi_y += h * uo[3 * l + 1];
        dxi_z += h * uo[3 * l + 2];
      }
      float det_x, det_y, det_z, dze_x, dze_y, dze_z;
      if (C::LINE_VEC) {
        det_x = deta[3 * i];
        det_y = deta[3 * i + 1];
        det_z = deta[3 * i + 2];
        dze_x = dzet[3 * i];
        dze_y = dzet[3 * i + 1];
        dze_z = dzet[3 * i + 2];
      } else {
        det_x = det_y = det_z = dze_x = dze_y = dze_z = 0.f;
#pragma unroll
        for (int l = 0; l < N; ++l) {
          const float* pe = rows_u + (l + N * k) * RS + 3 * i;
          det_x += hj[l] * pe[0];
          det_y += hj[l] * pe[1];
          det_z += hj[l] * pe[2];
          const float* pz = rows_u + (j + N * l) * RS + 3 * i;
          dze_x += hk[l] * pz[0];
          dze_y += hk[l] * pz[1];
          dze_z += hk[l] * pz[2];
        }
      }
      const int q = i * NL + line;
      float G[9];
#pragma unroll
      for (int a = 0; a < 9; ++a) G[a] = active ? __ldg(r + (kG + a) * NP + q) : 0.f;
      const float jac = active ? __ldg(r + kJac * NP + q) : 0.f;
      const float kappa = active ? __ldg(r + kKappa * NP + q) : 0.f;
      const float mu = active ? __ldg(r + kMu * NP + q) : 0.f;

      const float uxx = dxi_x * G[0] + det_x * G[3] + dze_x * G[6];
      const float uxy = dxi_x * G[1] + det_x * G[4] + dze_x * G[7];
      const float uxz = dxi_x * G[2] + det_x * G[5] + dze_x * G[8];
      const float uyx = dxi_y * G[0] + det_y * G[3] + dze_y * G[6];
      const float uyy = dxi_y * G[1] + det_y * G[4] + dze_y * G[7];
      const float uyz = dxi_y * G[2] + det_y * G[5] + dze_y * G[8];
      const float uzx = dxi_z * G[0] + det_z * G[3] + dze_z * G[6];
      const float uzy = dxi_z * G[1] + det_z * G[4] + dze_z * G[7];
      const float uzz = dxi_z * G[2] + det_z * G[5] + dze_z * G[8];

      const float lam = kappa - (2.f / 3.f) * mu;
      const float tr = uxx + uyy + uzz;
      const float sxx = lam * tr + 2.f * mu * uxx;
      const float syy = lam * tr + 2.f * mu * uyy;
      const float szz = lam * tr + 2.f * mu * uzz;
      const float sxy = mu * (uxy + uyx);
      const float sxz = mu * (uxz + uzx);
      const float syz = mu * (uyz + uzy);

      const float txi_x = jac * (sxx * G[0] + sxy * G[1] + sxz * G[2]);
      const float txi_y = jac * (sxy * G[0] + syy * G[1] + syz * G[2]);
      const float txi_z = jac * (sxz * G[0] + syz * G[1] + szz * G[2]);
#pragma unroll
      for (int ip = 0; ip < N; ++ip) {
        const float hw = HW[i * N + ip];
        fxi[3 * ip] += hw * txi_x;
        fxi[3 * ip + 1] += hw * txi_y;
        fxi[3 * ip + 2] += hw * txi_z;
      }
      if (active) {
        float* te = rows_te + line * RS + 3 * i;
        te[0] = jac * (sxx * G[3] + sxy * G[4] + sxz * G[5]);
        te[1] = jac * (sxy * G[3] + syy * G[4] + syz * G[5]);
        te[2] = jac * (sxz * G[3] + syz * G[4] + szz * G[5]);
        float* tz = rows_tz + line * RS + 3 * i;
        tz[0] = jac * (sxx * G[6] + sxy * G[7] + sxz * G[8]);
        tz[1] = jac * (sxy * G[6] + syy * G[7] + syz * G[8]);
        tz[2] = jac * (sxz * G[6] + syz * G[7] + szz * G[8]);
      }
    }
  }
  team_sync<WT>();

  // 3. eta and zeta transposed products; forces into the thread's own u row
  {
    float hwj[N], hwk[N];
#pragma unroll
    for (int l = 0; l < N; ++l) {
      hwj[l] = HW[l * N + j];
      hwk[l] = HW[l * N + k];
    }
    float eacc[3 * N], zacc[3 * N];
#pragma unroll
    for (int q = 0; q < 3 * N; ++q) eacc[q] = zacc[q] = 0.f;
#pragma unroll
    for (int l = 0; l < N; ++l) {
      float row[RS];
      load_row<N>(rows_te + (l + N * k) * RS, row);
#pragma unroll
      for (int q = 0; q < 3 * N; ++q) eacc[q] += hwj[l] * row[q];
      load_row<N>(rows_tz + (j + N * l) * RS, row);
#pragma unroll
      for (int q = 0; q < 3 * N; ++q) zacc[q] += hwk[l] * row[q];
    }
    const float wj = W[j], wk = W[k];
    if (active) {
      float out[RS];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const float wi = W[i];
#pragma unroll
        for (int c = 0; c < 3; ++c)
          out[3 * i + c] = -(wj * wk * fxi[3 * i + c] + wi * wk * eacc[3 * i + c] + wi * wj * zacc[3 * i + c]);
      }
#pragma unroll
      for (int q = 3 * N; q < RS; ++q) out[q] = 0.f;
      float4* o4 = reinterpret_cast<float4*>(rows_u + line * RS);
#pragma unroll
      for (int m = 0; m < C::RV; ++m) o4[m] = make_float4(out[4 * m], out[4 * m + 1], out[4 * m + 2], out[4 * m + 3]);
    }
  }
  team_sync<WT>();

  // 4. scatter in the gather's coalesced order
  for (int idx = tl; idx < ne * NP; idx += TEAM) {
    const int e = idx / NP;
    const int p = idx - e * NP;
    const int ln = p / N;
    const int i = p - ln * N;
    const float* sb = ts + e * ES;
    const uint32_t w = reinterpret_cast<const uint32_t*>(sb + 3 * NL * RS)[p];
    const size_t g3 = 3 * static_cast<size_t>(w & ~kFirstTouchBit);
    const float* src = sb + ln * RS + 3 * i;
    if (w & kFirstTouchBit) {
      f[g3] = src[0];
      f[g3 + 1] = src[1];
      f[g3 + 2] = src[2];
    } else {
      f[g3] += src[0];
      f[g3 + 1] += src[1];
      f[g3 + 2] += src[2];
    }
  }
}

template <int N, int MODE>
int launch_forces_nm(const ForceLaunch& L, cudaStream_t s) {
  using C = ForceCfg<N>;
  if (L.e1 <= L.e0) return 0;
  static unsigned long long attr_done = 0;  // one bit per device ordinal
  const int smem = C::SMEM_FLOATS * static_cast<int>(sizeof(float));
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(attr_done & bit)) {
    cudaError_t e = cudaFuncSetAttribute(forces_kernel<N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return static_cast<int>(e);
    attr_done |= bit;
  }
  const int grid = (L.e1 - L.e0 + C::EPC - 1) / C::EPC;
  forces_kernel<N, MODE><<<grid, C::T, smem, s>>>(L.rec, L.u, L.f, L.v, L.minv, L.e0, L.e1, L.dt, L.hdt, L.hdt2);
  return static_cast<int>(cudaGetLastError());
}


}  // namespace

int SEM_CAT(upload_basis_, SEM_NGLL)(const double* w, const double* h, void* stream, int n) {
  constexpr int N = SEM_NGLL;
  if (n != N) return static_cast<int>(cudaErrorInvalidValue);
  float hf[N * N], hwf[N * N], wf[N];
  for (int i = 0; i < N; ++i) {
    wf[i] = static_cast<float>(w[i]);
    for (int l = 0; l < N; ++l) {
      hf[i * N + l] = static_cast<float>(h[i * N + l]);
      hwf[l * N + i] = static_cast<float>(w[l] * h[l * N + i]);
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyToSymbolAsync(c_h, hf, sizeof(hf), 0, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_hw, hwf, sizeof(hwf), 0, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_w, wf, sizeof(wf), 0, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return static_cast<int>(e);
}

int SEM_CAT(launch_forces_, SEM_NGLL)(const ForceLaunch& L, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (L.mode) {
    case 0: return launch_forces_nm<SEM_NGLL, 0>(L, s);
    case 1: return launch_forces_nm<SEM_NGLL, 1>(L, s);
    case 2: return launch_forces_nm<SEM_NGLL, 2>(L, s);
    default: return static_cast<int>(cudaErrorInvalidValue);
  }
}

int SEM_CAT(forces_smem_bytes_, SEM_NGLL)() { return ForceCfg<SEM_NGLL>::SMEM_FLOATS * 4; }

}  // namespace semgb
