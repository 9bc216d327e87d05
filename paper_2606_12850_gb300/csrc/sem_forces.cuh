// Force kernel template of libsemgb, compiled once per NGLL: each sem_forces_<N>.cu
// defines SEM_NGLL and includes this file, so the orders build in parallel and every
// translation unit owns the constant-memory copy of its 1D basis.
#pragma once
#include <cuda_runtime.h>

#include <atomic>

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
__constant__ float2 c_h2[SEM_NGLL * SEM_NGLL];   // (hprime, hprime) pairs, c_h layout
__constant__ float2 c_hw2[SEM_NGLL * SEM_NGLL];  // (w hprime, w hprime) pairs, c_hw layout

// Packed float32 pair: d = a * b + c on both halves, each rounded to nearest as a scalar
// fma would be (one instruction for the pair on sm_100 and later).
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long ra, rb, rc, rd;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rc) : "f"(c.x), "f"(c.y));
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rd) : "l"(ra), "l"(rb), "l"(rc));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
  return d;
}

// ---------------------------------------------------------------------------------------
// Force kernel (Sec. II-B matrix-free stiffness action + Sec. IV-C coloured assembly).
//
// Threads work in teams: one warp per team for NGLL <= 5 (a team then only needs
// __syncwarp, so the warps of a CTA drift freely and hide each other's memory latency), two
// warps with a named barrier of their own for NGLL 7-8 (one element per team), the whole
// CTA for NGLL 6 and 9-10. A team holds E = TEAM / NGLL^2 elements of one colour.
//  0. (programmatic dependent launch) bulk-prefetch the team's element records into L2,
//     then wait for the previous grid;
//  1. gather, one thread per local point: consecutive threads take consecutive points p,
//     so a warp reads whole xi-rows of the global arrays; each thread has the loads of
//     four points in flight before it stores any of them;
//  2. contractions, one thread per line of NGLL points. From NGLL = 4 up (line owners):
//     a thread first owns an eta-line and a zeta-line and writes all N eta and zeta
//     derivatives along them; then, owning a xi-line, it forms the xi derivatives in
//     registers, the Jacobian map, the Hooke stress and the fluxes, keeps the xi-flux
//     transposed product in registers and writes the eta/zeta fluxes; then the eta/zeta-line
//     owners apply the weighted transposed products in place; at NGLL <= 3 each xi-line
//     thread reads the eta/zeta neighbours of its own points instead;
//  3. element forces into the (free) u slots;
//  4. scatter in the gather's order: a store at the node's first touch, a
//     read-modify-write otherwise (elements of one launch share no node: no atomics,
//     fixed summation order), previous values of four points loaded before any store.
// Shared memory per element: u (then F), eta and zeta derivatives (then fluxes) as [NP][3]
// each (the odd per-line stride 3N keeps the xi-line accesses conflict-free), ibool as
// [NP]; with several elements per warp the element stride is padded so that they fall in
// disjoint banks (offsets chosen by simulating the warp's access patterns).
// ---------------------------------------------------------------------------------------
template <int N>
struct ForceCfg {
  static constexpr int NP = N * N * N;
  static constexpr int NL = N * N;
  // Team kind: 0 one warp (NGLL <= 5), 1 two warps under a named barrier of their own
  // (NGLL 7-8, one element per team), 2 the whole CTA (NGLL 6 and 9-10).
  static constexpr int KIND = NL <= 32 ? 0 : (N == 7 || N == 8) ? 1 : 2;
  static constexpr bool WARP_TEAM = KIND == 0;
  static constexpr int T = KIND == 2 ? 256 : 128;     // threads per CTA
  static constexpr int TEAM = KIND == 0 ? 32 : KIND == 1 ? 64 : T;  // threads per team
  static constexpr int TEAMS = T / TEAM;              // teams per CTA
  static constexpr int E = TEAM / NL;                 // elements per team
  static constexpr int EPC = TEAMS * E;               // elements per CTA
  static constexpr int RES = N == 2 ? 7 : N == 3 ? 3 : N == 6 ? 5 : N == 7 ? 4 : N == 9 ? 9 : N == 4 || N == 10 ? 1 : 0;
  static constexpr int ES = 10 * NP + ((RES - 10 * NP) % 32 + 32) % 32;  // floats per element
  static constexpr int TS = E * ES;                   // floats per team
  static constexpr int SMEM_FLOATS = TEAMS * TS;
  static constexpr int REC = (kRecFields * NP + 3) / 4 * 4;
  // Default contraction form: line owners for the eta and zeta contractions (each shared
  // value read a fixed number of times) from NGLL = 4 up; at NGLL = 3 the per-point form is
  // faster (GB300, 128^3 mesh: 1.18 ms against 1.33 ms per sweep), at 5/7/9 the line owners
  // (0.66/0.86/0.96 ms against 0.75/0.94/1.15 ms). sem_autotune can measure both on the
  // caller's mesh and override it.
  static constexpr bool LINE_OWNERS = N >= 4;
  // CTAs per SM the register allocation must allow, from GB300 sweeps of force-sweep time
  // against the register cap: 64 registers for NGLL <= 5, 85 for NGLL = 6-7, 128 for
  // NGLL >= 8 (with the line owners the NGLL = 9 kernel fits 128 registers without spills:
  // 0.72 ms per sweep against 0.96 ms uncapped at one CTA per SM).
#ifdef SEM_FORCES_MIN_BLOCKS
  static constexpr int MIN_BLOCKS = SEM_FORCES_MIN_BLOCKS;
#else
  static constexpr int MIN_BLOCKS = KIND == 0 ? 8 : KIND == 1 ? (N == 7 ? 6 : 4) : (N <= 7 ? 3 : 2);
#endif
};

// Programmatic dependent launch (the colour launches of one sweep overlap): a colour's
// CTAs may be scheduled while the previous launch drains, prefetch their element records
// (constant for the whole run) into L2, and wait for the previous grid to complete, with
// its memory visible, before they read any wavefield. Both instructions are no-ops for a
// kernel launched without the programmatic attribute.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
__device__ __forceinline__ void prefetch_l2_line(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
__device__ __forceinline__ void wait_prerequisite_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Iterations of a bounded spin (each with a 128 ns sleep): about half a second.
constexpr unsigned int kSweepSpinLimit = 1u << 22;
__device__ __forceinline__ void allow_dependent_grid() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Barrier of one team: the warp, a named barrier (1 + team) over the team's TEAM threads
// (several warps), or the CTA.
template <int KIND, int TEAM>
__device__ __forceinline__ void team_sync(int team) {
  if constexpr (KIND == 0) {
    __syncwarp();
  } else if constexpr (KIND == 1) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + team), "n"(TEAM) : "memory");
  } else {
    __syncthreads();
  }
}

// Phases 2-3 of one team's elements (Sec. II-B): on entry the u slots of every active
// element workspace (ES floats per element, E = TEAM / NGLL^2 elements from ts on) hold the
// element's displacement [NP][3]; on return they hold its forces F = -K_e u_e [NP][3].
// rec_of(le) gives the record of the team's element le. Shared by the element kernel and
// the patch kernel, which differ only in how they gather u and assemble F.
template <int N, int KIND, int TEAM, int ES, bool LO, class RecOf>
__device__ __forceinline__ void team_element_forces(float* ts, int tl, int ne, int team, RecOf rec_of) {
  constexpr int NP = N * N * N, NL = N * N;
  const float* __restrict__ H = c_h;
  const float* __restrict__ HW = c_hw;
  const float* __restrict__ W = c_w;
  if constexpr (LO) {
    // Thread tl of the team owns one line of NGLL points of element le = tl / NL, indexed by
    // line = a + N b: the xi-line (j, k) = (a, b) in phases 2b and 4, the eta-line
    // (i, k) = (a, b) and the zeta-line (i, j) = (a, b) in phases 2a and 3. A line owner reads
    // its line once and produces all N contractions along it, so every shared value is read
    // a fixed number of times instead of N times.
    const int le = tl / NL;
    const int line = tl - le * NL;
    const int a = line % N;
    const int b = line / N;
    const bool active = le < ne;
    float* su = ts + (active ? le : 0) * ES;  // u, then F: [NP][3]
    float* se = su + 3 * NP;                   // eta derivatives, then eta fluxes [NP][3]
    float* sz = su + 6 * NP;                   // zeta derivatives, then zeta fluxes [NP][3]
    const float* __restrict__ r = rec_of(active ? le : 0);

    // 2a. eta derivatives along the eta-line (i, k) = (a, b), zeta derivatives along the
    //     zeta-line (i, j) = (a, b)
    //     (each eta value paired with the zeta value it shares a coefficient with: one
    //     packed fma per pair)
    if (active) {
      float2 v[3][N];  // (eta-line value, zeta-line value)
#pragma unroll
      for (int l = 0; l < N; ++l)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          v[c][l] = make_float2(su[3 * (a + N * (l + N * b)) + c], su[3 * (a + N * (b + N * l)) + c]);
#pragma unroll
      for (int m = 0; m < N; ++m)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float2 d = make_float2(0.f, 0.f);
#pragma unroll
          for (int l = 0; l < N; ++l) d = ffma2(c_h2[m * N + l], v[c][l], d);
          se[3 * (a + N * (m + N * b)) + c] = d.x;
          sz[3 * (a + N * (b + N * m)) + c] = d.y;
        }
    }
    team_sync<KIND, TEAM>(team);

    // 2b. along the xi-line (j, k) = (a, b): xi derivatives in registers, Jacobian map, Hooke
    //     stress, fluxes; the xi-flux transposed product stays in registers, the eta and zeta
    //     fluxes replace the derivatives they were made from
    float2 fxy[N];  // (x, y) and z of the xi-flux transposed product
    float fz[N];
    {
      float2 uxy[N];
      float uz[N];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int p = i + N * line;
        uxy[i] = make_float2(su[3 * p], su[3 * p + 1]);
        uz[i] = su[3 * p + 2];
        fxy[i] = make_float2(0.f, 0.f);
        fz[i] = 0.f;
      }
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float2 dxy = make_float2(0.f, 0.f);
        float dxi_z = 0.f;
#pragma unroll
        for (int l = 0; l < N; ++l) {
          dxy = ffma2(c_h2[i * N + l], uxy[l], dxy);
          dxi_z += H[i * N + l] * uz[l];
        }
        const float dxi_x = dxy.x, dxi_y = dxy.y;
        const int p3 = 3 * (i + N * line);
        const float det_x = se[p3], det_y = se[p3 + 1], det_z = se[p3 + 2];
        const float dze_x = sz[p3], dze_y = sz[p3 + 1], dze_z = sz[p3 + 2];
        const int q = i * NL + line;
        float G[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) G[c] = active ? __ldg(r + (kG + c) * NP + q) : 0.f;
        const float kappa = active ? __ldg(r + kJKappa * NP + q) : 0.f;  // J kappa
        const float mu = active ? __ldg(r + kJMu * NP + q) : 0.f;        // J mu

        const float uxx = dxi_x * G[0] + det_x * G[3] + dze_x * G[6];
        const float uxy = dxi_x * G[1] + det_x * G[4] + dze_x * G[7];
        const float uxz = dxi_x * G[2] + det_x * G[5] + dze_x * G[8];
        const float uyx = dxi_y * G[0] + det_y * G[3] + dze_y * G[6];
        const float uyy = dxi_y * G[1] + det_y * G[4] + dze_y * G[7];
        const float uyz = dxi_y * G[2] + det_y * G[5] + dze_y * G[8];
        const float uzx = dxi_z * G[0] + det_z * G[3] + dze_z * G[6];
        const float uzy = dxi_z * G[1] + det_z * G[4] + dze_z * G[7];
        const float uzz = dxi_z * G[2] + det_z * G[5] + dze_z * G[8];

        // J sigma (the record holds J kappa and J mu, so the fluxes need no J multiply)
        const float lam = kappa - (2.f / 3.f) * mu;
        const float tr = uxx + uyy + uzz;
        const float sxx = lam * tr + 2.f * mu * uxx;
        const float syy = lam * tr + 2.f * mu * uyy;
        const float szz = lam * tr + 2.f * mu * uzz;
        const float sxy = mu * (uxy + uyx);
        const float sxz = mu * (uxz + uzx);
        const float syz = mu * (uyz + uzy);

        const float txi_x = (sxx * G[0] + sxy * G[1] + sxz * G[2]);
        const float txi_y = (sxy * G[0] + syy * G[1] + syz * G[2]);
        const float txi_z = (sxz * G[0] + syz * G[1] + szz * G[2]);
        const float2 txy = make_float2(txi_x, txi_y);
#pragma unroll
        for (int ip = 0; ip < N; ++ip) {
          fxy[ip] = ffma2(c_hw2[i * N + ip], txy, fxy[ip]);
          fz[ip] += HW[i * N + ip] * txi_z;
        }
        if (active) {
          se[p3] = (sxx * G[3] + sxy * G[4] + sxz * G[5]);
          se[p3 + 1] = (sxy * G[3] + syy * G[4] + syz * G[5]);
          se[p3 + 2] = (sxz * G[3] + syz * G[4] + szz * G[5]);
          sz[p3] = (sxx * G[6] + sxy * G[7] + sxz * G[8]);
          sz[p3 + 1] = (sxy * G[6] + syy * G[7] + syz * G[8]);
          sz[p3 + 2] = (sxz * G[6] + syz * G[7] + szz * G[8]);
        }
      }
    }
    team_sync<KIND, TEAM>(team);

    // 3. eta and zeta transposed products along the eta- and zeta-lines, in place
    if (active) {
      float2 v[3][N];  // (eta-line flux, zeta-line flux)
#pragma unroll
      for (int l = 0; l < N; ++l)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          v[c][l] = make_float2(se[3 * (a + N * (l + N * b)) + c], sz[3 * (a + N * (b + N * l)) + c]);
#pragma unroll
      for (int m = 0; m < N; ++m)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float2 t = make_float2(0.f, 0.f);
#pragma unroll
          for (int l = 0; l < N; ++l) t = ffma2(c_hw2[l * N + m], v[c][l], t);
          se[3 * (a + N * (m + N * b)) + c] = t.x;
          sz[3 * (a + N * (b + N * m)) + c] = t.y;
        }
    }
    team_sync<KIND, TEAM>(team);

    // 3b. element forces along the xi-line (j, k) = (a, b) into the (now free) u slots
    if (active) {
      const float wj = W[a], wk = W[b];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const float wi = W[i];
        const int p = 3 * (i + N * line);
        su[p] = -(wj * wk * fxy[i].x + wi * wk * se[p] + wi * wj * sz[p]);
        su[p + 1] = -(wj * wk * fxy[i].y + wi * wk * se[p + 1] + wi * wj * sz[p + 1]);
        su[p + 2] = -(wj * wk * fz[i] + wi * wk * se[p + 2] + wi * wj * sz[p + 2]);
      }
    }
    team_sync<KIND, TEAM>(team);

  } else {
    // 2. per xi-line derivatives, stress and fluxes
    const int le = tl / NL;
    const int line = tl - le * NL;  // = j + N k
    const int j = line % N;
    const int k = line / N;
    const bool active = le < ne;
    float* su = ts + (active ? le : 0) * ES;  // u, then F: [NP][3]
    float* se = su + 3 * NP;                   // eta fluxes [NP][3]
    float* sz = su + 6 * NP;                   // zeta fluxes [NP][3]
    const float* __restrict__ r = rec_of(active ? le : 0);

    float ux[N], uy[N], uz[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int p = i + N * line;
      ux[i] = su[3 * p];
      uy[i] = su[3 * p + 1];
      uz[i] = su[3 * p + 2];
    }
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
      float dxi_x = 0.f, dxi_y = 0.f, dxi_z = 0.f;
      float det_x = 0.f, det_y = 0.f, det_z = 0.f;
      float dze_x = 0.f, dze_y = 0.f, dze_z = 0.f;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        const float h = H[i * N + l];
        dxi_x += h * ux[l];
        dxi_y += h * uy[l];
        dxi_z += h * uz[l];
        const int pe = 3 * (i + N * (l + N * k));
        det_x += hj[l] * su[pe];
        det_y += hj[l] * su[pe + 1];
        det_z += hj[l] * su[pe + 2];
        const int pz = 3 * (i + N * (j + N * l));
        dze_x += hk[l] * su[pz];
        dze_y += hk[l] * su[pz + 1];
        dze_z += hk[l] * su[pz + 2];
      }
      const int q = i * NL + line;
      float G[9];
#pragma unroll
      for (int a = 0; a < 9; ++a) G[a] = active ? __ldg(r + (kG + a) * NP + q) : 0.f;
      const float kappa = active ? __ldg(r + kJKappa * NP + q) : 0.f;  // J kappa
      const float mu = active ? __ldg(r + kJMu * NP + q) : 0.f;        // J mu

      const float uxx = dxi_x * G[0] + det_x * G[3] + dze_x * G[6];
      const float uxy = dxi_x * G[1] + det_x * G[4] + dze_x * G[7];
      const float uxz = dxi_x * G[2] + det_x * G[5] + dze_x * G[8];
      const float uyx = dxi_y * G[0] + det_y * G[3] + dze_y * G[6];
      const float uyy = dxi_y * G[1] + det_y * G[4] + dze_y * G[7];
      const float uyz = dxi_y * G[2] + det_y * G[5] + dze_y * G[8];
      const float uzx = dxi_z * G[0] + det_z * G[3] + dze_z * G[6];
      const float uzy = dxi_z * G[1] + det_z * G[4] + dze_z * G[7];
      const float uzz = dxi_z * G[2] + det_z * G[5] + dze_z * G[8];

      // J sigma (the record holds J kappa and J mu, so the fluxes need no J multiply)
      const float lam = kappa - (2.f / 3.f) * mu;
      const float tr = uxx + uyy + uzz;
      const float sxx = lam * tr + 2.f * mu * uxx;
      const float syy = lam * tr + 2.f * mu * uyy;
      const float szz = lam * tr + 2.f * mu * uzz;
      const float sxy = mu * (uxy + uyx);
      const float sxz = mu * (uxz + uzx);
      const float syz = mu * (uyz + uzy);

      const float txi_x = (sxx * G[0] + sxy * G[1] + sxz * G[2]);
      const float txi_y = (sxy * G[0] + syy * G[1] + syz * G[2]);
      const float txi_z = (sxz * G[0] + syz * G[1] + szz * G[2]);
#pragma unroll
      for (int ip = 0; ip < N; ++ip) {
        const float hw = HW[i * N + ip];
        fx[ip] += hw * txi_x;
        fy[ip] += hw * txi_y;
        fz[ip] += hw * txi_z;
      }
      if (active) {
        const int p3 = 3 * (i + N * line);
        se[p3] = (sxx * G[3] + sxy * G[4] + sxz * G[5]);
        se[p3 + 1] = (sxy * G[3] + syy * G[4] + syz * G[5]);
        se[p3 + 2] = (sxz * G[3] + syz * G[4] + szz * G[5]);
        sz[p3] = (sxx * G[6] + sxy * G[7] + sxz * G[8]);
        sz[p3 + 1] = (sxy * G[6] + syy * G[7] + syz * G[8]);
        sz[p3 + 2] = (sxz * G[6] + syz * G[7] + szz * G[8]);
      }
    }
    team_sync<KIND, TEAM>(team);

    // 3. eta and zeta transposed products; forces into the (now free) u slots
    {
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
          const int pe = 3 * (i + N * (l + N * k));
          ex += hwj[l] * se[pe];
          ey += hwj[l] * se[pe + 1];
          ez += hwj[l] * se[pe + 2];
          const int pz = 3 * (i + N * (j + N * l));
          zx += hwk[l] * sz[pz];
          zy += hwk[l] * sz[pz + 1];
          zz += hwk[l] * sz[pz + 2];
        }
        const float wi = W[i];
        if (active) {
          const int p = 3 * (i + N * line);
          su[p] = -(wj * wk * fx[i] + wi * wk * ex + wi * wj * zx);
          su[p + 1] = -(wj * wk * fy[i] + wi * wk * ey + wi * wj * zy);
          su[p + 2] = -(wj * wk * fz[i] + wi * wk * ez + wi * wj * zz);
        }
      }
    }
    team_sync<KIND, TEAM>(team);

  }
}

// Element kernel: one colour of elements per launch, each element gathered and scattered
// on its own through the ibool words of its record.
// CALLER false: u and f are the context's own padded fields [nglob][S][4] (internal node
// order). CALLER true (one shot): caller arrays [nglob][3] in caller node order, reached
// through perm (internal -> caller node). With S shots the launch works on the items
// (element, shot) of elements e0 .. e1-1 of elist, element-major: the teams of a CTA take the
// shots of one element, so its record is read from DRAM once for all of them.
template <int N, bool MS, bool LO, bool CALLER, bool ATOMIC = false>
__global__ void __launch_bounds__(ForceCfg<N>::T, ForceCfg<N>::MIN_BLOCKS)
    forces_kernel(const float* __restrict__ rec, const int* __restrict__ elist, const int* __restrict__ perm,
                  const float* __restrict__ u, float* __restrict__ f, int e0, int e1, int S_arg) {
  const int S = MS ? S_arg : 1;  // shots (a compile-time 1 for the single-shot kernel)
  using C = ForceCfg<N>;
  constexpr int NP = C::NP, E = C::E, REC = C::REC, TEAM = C::TEAM, ES = C::ES;
  extern __shared__ float4 smem4[];

  const int team = threadIdx.x / TEAM;
  const int tl = threadIdx.x - team * TEAM;
  const int ibase = (blockIdx.x * C::TEAMS + team) * E;  // first item of the team
  const int ne = min(E, (e1 - e0) * S - ibase);
  if (C::KIND != 2 && ne <= 0) return;  // a team without items (its barrier is its own)
  float* ts = reinterpret_cast<float*>(smem4) + team * C::TS;
  // record slot and shot of the team's item le (elist: record slots in colour order)
  auto elem_of = [&](int le) { return elist[e0 + (MS ? (ibase + le) / S : ibase + le)]; };
  auto shot_of = [&](int le) { return MS ? (ibase + le) % S : 0; };

  // 0. records to L2 while the previous grid finishes, then wait for its results
  if (tl < ne) prefetch_l2(rec + static_cast<size_t>(elem_of(tl)) * REC, kForceFields * NP * sizeof(float));
  wait_prerequisite_grid();
  allow_dependent_grid();

  // 1. gather, one thread per local point; GB points per thread at a time, their ibool
  //    words first and then their nodes, so that the loads of a group are all in flight
  constexpr int GB = 4;
  for (int base = tl; base < ne * NP; base += GB * TEAM) {
    uint32_t w[GB];
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      const int idx = base + r * TEAM;
      const int le = idx / NP;
      w[r] = idx < ne * NP ? __float_as_uint(__ldg(rec + static_cast<size_t>(elem_of(le)) * REC + (idx - le * NP)))
                           : 0u;
    }
    float q[GB][3];
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      const size_t g = w[r] & kNodeMask;
      if (base + r * TEAM < ne * NP) {
        if constexpr (CALLER) {
          const size_t gc = static_cast<size_t>(__ldg(perm + g));
          q[r][0] = __ldg(u + 3 * gc);
          q[r][1] = __ldg(u + 3 * gc + 1);
          q[r][2] = __ldg(u + 3 * gc + 2);
        } else {
          const int le = (base + r * TEAM) / NP;
          const float4 v = __ldg(reinterpret_cast<const float4*>(u) + g * S + shot_of(le));
          q[r][0] = v.x;
          q[r][1] = v.y;
          q[r][2] = v.z;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      const int idx = base + r * TEAM;
      if (idx < ne * NP) {
        const int le = idx / NP;
        const int p = idx - le * NP;
        float* eb = ts + le * ES;
        reinterpret_cast<uint32_t*>(eb + 9 * NP)[p] = w[r];
        eb[3 * p] = q[r][0];
        eb[3 * p + 1] = q[r][1];
        eb[3 * p + 2] = q[r][2];
      }
    }
  }
  team_sync<C::KIND, C::TEAM>(team);

  team_element_forces<N, C::KIND, TEAM, ES, LO>(ts, tl, ne, team, [&](int le) {
    return rec + static_cast<size_t>(elem_of(le)) * REC;
  });

  // 4. scatter in the gather's coalesced order; the previous values of a group of GB nodes
  //    are loaded before any of them is written back
  if constexpr (ATOMIC) {  // the colouring ablation: every element in one launch, f zeroed first
    for (int idx = tl; idx < ne * NP; idx += TEAM) {
      const int e = idx / NP;
      const float* sb = ts + e * ES;
      const uint32_t w = reinterpret_cast<const uint32_t*>(sb + 9 * NP)[idx - e * NP];
      const float* src = sb + 3 * (idx - e * NP);
      atomicAdd(reinterpret_cast<float4*>(f) + static_cast<size_t>(w & kNodeMask),
                make_float4(src[0], src[1], src[2], 0.f));
    }
    return;
  }
  if constexpr (CALLER) {
    for (int idx = tl; idx < ne * NP; idx += TEAM) {
      const int e = idx / NP;
      const float* sb = ts + e * ES;
      const uint32_t w = reinterpret_cast<const uint32_t*>(sb + 9 * NP)[idx - e * NP];
      const size_t g = static_cast<size_t>(__ldg(perm + (w & kNodeMask)));
      const float* src = sb + 3 * (idx - e * NP);
      if (w & kFirstTouchBit) {
        f[3 * g] = src[0];
        f[3 * g + 1] = src[1];
        f[3 * g + 2] = src[2];
      } else {
        f[3 * g] += src[0];
        f[3 * g + 1] += src[1];
        f[3 * g + 2] += src[2];
      }
    }
    return;
  }
  for (int base = tl; base < ne * NP; base += GB * TEAM) {
    uint32_t w[GB];
    float4 prev[GB];
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      const int idx = base + r * TEAM;
      w[r] = kFirstTouchBit;
      prev[r] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (idx < ne * NP) {
        const int e = idx / NP;
        w[r] = reinterpret_cast<const uint32_t*>(ts + e * ES + 9 * NP)[idx - e * NP];
        if (!(w[r] & kFirstTouchBit))
          prev[r] = reinterpret_cast<const float4*>(f)[static_cast<size_t>(w[r] & kNodeMask) * S + shot_of(e)];
      }
    }
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      const int idx = base + r * TEAM;
      if (idx < ne * NP) {
        const int e = idx / NP;
        const float* src = ts + e * ES + 3 * (idx - e * NP);
        reinterpret_cast<float4*>(f)[static_cast<size_t>(w[r] & kNodeMask) * S + shot_of(e)] =
            make_float4(src[0] + prev[r].x, src[1] + prev[r].y, src[2] + prev[r].z, 0.f);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Patch kernel (Sec. II-B stiffness action with the Sec. IV-C coloured assembly applied to
// patches of elements): one CTA per patch, a brick of up to PE neighbouring elements whose
// records are consecutive; the launches of one sweep take the patch colours in order.
//  0. bulk-prefetch the patch's records into L2, then wait for the previous grid;
//  1. every team gathers its own elements' points through the records' ibool words, as the
//     element kernel does (teams run independently; the nodes the patch's elements share
//     are read once from DRAM and then from L1);
//  2-3. every element's forces (team_element_forces);
//  4a. each team adds the forces of its points that are alone at their patch node (inside
//     one element of the patch: 512 of the 729 nodes of a 2 x 2 x 2 brick at NGLL 5) to the
//     node, with no wait for the other teams;
//  4b. after one CTA barrier, per shared patch node: the forces of the local points that
//     meet there summed in the fixed order of the patch table (ascending element, then
//     point; kPatchSlots slots per node read as one 16-byte word), then added to the node.
//  A node is stored instead of added at its first touch in patch-colour order
//  (kPatchFirstBit on the ibool word of the node's first local point in the patch).
//  Patches of one colour share no node, so there are no atomics, and the order of every
//  sum is fixed (bitwise reproducible results).
// Shared memory: one ES-float workspace per element, as in the element kernel.
// ---------------------------------------------------------------------------------------
template <int N>
struct PatchCfg {
  static constexpr int NP = N * N * N;
  static constexpr int NL = N * N;
  // Teams of TEAM threads holding E = TEAM / NL elements, one thread per line: one warp up
  // to NGLL 5, two warps under a named barrier for NGLL 6-8, the CTA for NGLL 9-10. (Teams
  // of several warps with more elements fill more lanes at NGLL 5-7, but the warps then wait
  // for each other at every phase: GB300, 64^3 at NGLL 5, 0.92 ms per sweep against 0.70.)
  static constexpr int TEAM = N <= 5 ? 32 : N <= 8 ? 64 : 256;
  // 0 one warp, 1 a named barrier over the team's warps, 2 the CTA
  static constexpr int KIND = TEAM == 32 ? 0 : TEAM < 256 ? 1 : 2;
  static constexpr int E = TEAM / NL;  // elements per team
  // the default brick, in elements along the lattice x, y, z (any brick of PE elements runs
  // the same kernel; GB300, 256 GLL intervals per side, one time step's fused sweep: at NGLL
  // 5, 1x4x2 0.770 ms against 2x2x2 0.778 and 4x1x2 0.774; at NGLL 7, 1x2x2 0.805 against
  // 2x2x1 0.810 and 2x1x2 0.811; at NGLL 9, 3x1x1 0.818 against 1x3x1 0.819 and 1x1x3 0.844)
  static constexpr int BX = N == 2 ? 4 : N == 3 ? 3 : N == 4 ? 4 : N == 5 || N == 7 ? 1 : N <= 8 ? 2 : N == 9 ? 3 : 2;
  static constexpr int BY = N == 2 ? 4 : N == 3 ? 3 : N == 5 ? 4 : N <= 8 ? 2 : 1;
  static constexpr int BZ = N == 2 ? 4 : N == 3 ? 3 : N <= 5 || N == 7 ? 2 : 1;
  static constexpr int PE = BX * BY * BZ;
  static constexpr int TEAMS = (PE + E - 1) / E;
  static constexpr int T = TEAMS * TEAM;
  // floats per element workspace (at least 10 NP: u/F, eta and zeta values, ibool words)
  static constexpr int ES = KIND == ForceCfg<N>::KIND ? ForceCfg<N>::ES : 10 * NP + 1;
  static constexpr int TS = E * ES;
  static constexpr int REC = ForceCfg<N>::REC;
  static constexpr int SMEM = TEAMS * TS * 4;
  static constexpr int MIN_BLOCKS = N == 3 ? 3 : N <= 5 ? 4 : N <= 7 ? 3 : 2;
  static_assert(E >= 1 && 10 * NP <= ES, "team and workspace sizes");
};

// Index of a node's 16-byte slot in a [nglob][S][4] field (S = 1 for a single shot).
template <bool MS>
__device__ __forceinline__ size_t node_slot(uint32_t w, int S, int shot) {
  if constexpr (MS)
    return static_cast<size_t>(w & kNodeMask) * S + shot;
  else
    return static_cast<size_t>(w & kNodeMask);
}

// Phases 1-3 of one patch for the calling thread's team: gather through the records' ibool
// words (GB points per thread in flight; the shared-memory copy of each word keeps the node,
// the patch first-touch flag and kAloneBit), then the element forces.
// (NM 1: the half-step velocity and 1/M of the nodes the patch touches last are prefetched
// into L2 as their points are gathered, for the Newmark update at the end of the patch; NM 2:
// the older adjoint field and 1/M, for the adjoint leapfrog.)
template <int N, bool LO, bool MS = false, int NM = 0>
__device__ __forceinline__ void patch_gather_compute(const PatchDesc& d, const float* __restrict__ rec,
                                                     const float4* __restrict__ u, float* wsb, bool u_from_l2,
                                                     int S = 1, int shot = 0, const SweepNewmark* nm = nullptr) {
  using C = PatchCfg<N>;
  constexpr int NP = C::NP, E = C::E, TEAM = C::TEAM, ES = C::ES, REC = C::REC;
  const int team = threadIdx.x / TEAM;
  const int tl = threadIdx.x - team * TEAM;
  const int ne = min(E, d.nelem - team * E);  // this team's elements
  const float* __restrict__ trec = rec + static_cast<size_t>(d.slot0 + team * E) * REC;
  constexpr int GB = 4;
  float* ts = wsb + team * C::TS;
  for (int base = tl; base < ne * NP; base += GB * TEAM) {
    uint32_t w[GB];
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      const int idx = base + r * TEAM;
      const int le = idx / NP;
      w[r] = idx < ne * NP ? __float_as_uint(__ldg(trec + static_cast<size_t>(le) * REC + (idx - le * NP))) : 0u;
    }
    if constexpr (NM != 0) {
#pragma unroll
      for (int r = 0; r < GB; ++r)
        if (w[r] & kPatchLastBit) {
          prefetch_l2_line(reinterpret_cast<const float4*>(NM == 2 ? nm->lam_old : nm->v) +
                           node_slot<MS>(w[r], S, shot));
          prefetch_l2_line(nm->minv + (w[r] & kNodeMask));
        }
    }
    float4 q[GB];
    if (u_from_l2) {
#pragma unroll
      for (int r = 0; r < GB; ++r) q[r] = __ldcg(u + node_slot<MS>(w[r], S, shot));
    } else {
#pragma unroll
      for (int r = 0; r < GB; ++r) q[r] = __ldg(u + node_slot<MS>(w[r], S, shot));
    }
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      const int idx = base + r * TEAM;
      if (idx < ne * NP) {
        const int le = idx / NP;
        const int p = idx - le * NP;
        float* eb = ts + le * ES;
        reinterpret_cast<uint32_t*>(eb + 9 * NP)[p] = w[r];
        eb[3 * p] = q[r].x;
        eb[3 * p + 1] = q[r].y;
        eb[3 * p + 2] = q[r].z;
      }
    }
  }
  if (C::KIND == 2 || ne > 0) {
    team_sync<C::KIND, TEAM>(team);
    team_element_forces<N, C::KIND, TEAM, ES, LO>(ts, tl, ne, team,
                                                  [&](int le) { return trec + static_cast<size_t>(le) * REC; });
  }
}

// Previous value of a node of f: through L1 (COHERENT false: f was last written by an
// earlier grid) or from L2 (COHERENT true: other CTAs of this grid wrote it).
template <bool COHERENT>
__device__ __forceinline__ float4 load_f(const float4* p) {
  if constexpr (COHERENT)
    return __ldcg(p);
  else
    return *p;
}

// Point sources of the step at a node the patch touches last (Sec. V-C): the Ricker wavelet
// at t_{n+1} = step dt (the counter, advanced before the sweep, read from L2) times each
// force, added to the node's complete force in the order the entries are listed.
__device__ __forceinline__ void add_point_sources(const PatchDesc& d, const SweepNewmark& nm, uint32_t node, int shot,
                                                  float& fx, float& fy, float& fz) {
  for (int i = 0; i < d.nsrc; ++i) {
    const PatchSrc& s = nm.src[d.src_off + i];
    if (s.node != static_cast<int>(node) || s.shot != shot) continue;
    const long long n = __ldcg(nm.step);
    const double tau = static_cast<double>(n) * nm.dtd - nm.t0;
    const double x = M_PI * nm.f0 * tau;
    const double aa = x * x;
    const double R = (1.0 - 2.0 * aa) * exp(-aa);
    fx += static_cast<float>(s.f[0] * R);
    fy += static_cast<float>(s.f[1] * R);
    fz += static_cast<float>(s.f[2] * R);
  }
}

// The inputs of a node's Newmark update, loaded with the previous force values so that all
// of a thread's loads are in flight together: 1/M, the half-step velocity and (mode 1) the
// displacement.
struct NodeState {
  float m;
  float4 v, u;
};
template <bool MS, bool WITH_U = false>
__device__ __forceinline__ void load_node_state(const SweepNewmark& nm, uint32_t w, int S, int shot, NodeState& st) {
  const size_t g = node_slot<MS>(w, S, shot);
  st.m = __ldg(nm.minv + (w & kNodeMask));
  st.v = __ldcg(reinterpret_cast<const float4*>(nm.v) + g);
  if (WITH_U || nm.mode == 1) st.u = __ldcg(reinterpret_cast<const float4*>(nm.u) + g);
}

// Newmark update of a node whose complete force (fx, fy, fz) is known (mode 1 or 2):
//   a = M^-1 f ; v = v_half + dt/2 a ; mode 1: u <- u + dt v + dt^2/2 a, v_half <- v + dt/2 a ;
//   mode 2: v and a stored.
template <bool MS>
__device__ __forceinline__ void newmark_node(const SweepNewmark& nm, uint32_t w, int S, int shot, const NodeState& st,
                                             float fx, float fy, float fz) {
  const size_t g = node_slot<MS>(w, S, shot);
  const float ax = fx * st.m, ay = fy * st.m, az = fz * st.m;
  const float vx = st.v.x + nm.hdt * ax, vy = st.v.y + nm.hdt * ay, vz = st.v.z + nm.hdt * az;
  if (nm.mode == 1) {
    reinterpret_cast<float4*>(nm.u)[g] = make_float4((st.u.x + nm.dt * vx) + nm.hdt2 * ax,
                                                     (st.u.y + nm.dt * vy) + nm.hdt2 * ay,
                                                     (st.u.z + nm.dt * vz) + nm.hdt2 * az, 0.f);
    reinterpret_cast<float4*>(nm.v)[g] = make_float4(vx + nm.hdt * ax, vy + nm.hdt * ay, vz + nm.hdt * az, 0.f);
  } else {
    reinterpret_cast<float4*>(nm.v)[g] = make_float4(vx, vy, vz, 0.f);
    reinterpret_cast<float4*>(nm.a)[g] = make_float4(ax, ay, az, 0.f);
  }
}

// The snapshot of the node's displacement u^{n+1} (NM 3: a Newmark sweep of a snapshot run).
__device__ __forceinline__ void snapshot_node(const SweepNewmark& nm, uint32_t w, const NodeState& st) {
  const DevCtl* ctl = nm.snap_ctl;
  const uint32_t g = w & kNodeMask;
  float* o = ctl->snap + static_cast<long long>(ctl->col - 1) * ctl->snap_per +
             3 * static_cast<size_t>(nm.snap_perm ? __ldg(nm.snap_perm + g) : static_cast<int>(g));
  o[0] = st.u.x;
  o[1] = st.u.y;
  o[2] = st.u.z;
}

// The adjoint step at a node whose force f = -K lam is complete (NM 2): the receiver
// residuals of the step at this node added to f in ascending receiver order (G / dt^2), then
// the leapfrog lam_old <- 2 lam - lam_old + dt^2 M^-1 f (the same float operations as the
// separate injection and leapfrog passes).
__device__ __forceinline__ void adjoint_receivers(const SweepNewmark& nm, int2 rr, uint32_t node, float& fx, float& fy,
                                                  float& fz) {
  const float* G = nm.idx ? nm.idx->adj_G + static_cast<long long>(nm.idx->adj_j - 1) * nm.idx->adj_gstep : nm.G;
  if (!G) return;
  for (int i = rr.x; i < rr.x + rr.y; ++i) {
    const PatchRecv e = nm.recv[i];
    if (e.node != static_cast<int>(node)) continue;
    fx += G[3 * e.r] * nm.inv_dt2;
    fy += G[3 * e.r + 1] * nm.inv_dt2;
    fz += G[3 * e.r + 2] * nm.inv_dt2;
  }
}
__device__ __forceinline__ void load_adjoint_state(const SweepNewmark& nm, uint32_t w, NodeState& st) {
  const size_t g = w & kNodeMask;
  st.m = __ldg(nm.minv + g);
  st.u = __ldcg(reinterpret_cast<const float4*>(nm.u) + g);        // lam^m
  st.v = __ldcg(reinterpret_cast<const float4*>(nm.lam_old) + g);  // lam^{m+1}
}
__device__ __forceinline__ void adjoint_node(const SweepNewmark& nm, uint32_t w, const NodeState& st, float fx,
                                             float fy, float fz) {
  const size_t g = w & kNodeMask;
  const float s = nm.dt2 * st.m;
  const float4 l = st.u, o = st.v;
  reinterpret_cast<float4*>(nm.lam_old)[g] =
      make_float4(2.f * l.x - o.x + s * fx, 2.f * l.y - o.y + s * fy, 2.f * l.z - o.z + s * fz, 0.f);
}

// Phase 4a for the calling thread's team: the forces of its points that are alone at their
// patch node added to the node (stored at its first touch; with a Newmark mode, used for the
// node's update at its last touch and not stored).
template <int N, bool COHERENT, bool MS = false, int NM = 0>
__device__ __forceinline__ void patch_write_alone(const PatchDesc& d, float4* __restrict__ f, const float* wsb,
                                                  const SweepNewmark& nm, int S = 1, int shot = 0,
                                                  int2 rr = make_int2(0, 0)) {
  using C = PatchCfg<N>;
  constexpr int NP = C::NP, E = C::E, TEAM = C::TEAM, ES = C::ES, GB = NM ? 2 : 4;
  const int team = threadIdx.x / TEAM;
  const int tl = threadIdx.x - team * TEAM;
  const int ne = min(E, d.nelem - team * E);
  const float* ts = wsb + team * C::TS;
  constexpr uint32_t last_bit = NM ? kPatchLastBit : 0u;
  for (int base = tl; base < ne * NP; base += GB * TEAM) {
    uint32_t w[GB];
    float4 prev[GB];
    NodeState st[GB];
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      const int idx = base + r * TEAM;
      w[r] = 0u;
      prev[r] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (idx < ne * NP) {
        const int e = idx / NP;
        w[r] = reinterpret_cast<const uint32_t*>(ts + e * ES + 9 * NP)[idx - e * NP];
        if ((w[r] & kAloneBit) && !(w[r] & kPatchFirstBit)) prev[r] = load_f<COHERENT>(f + node_slot<MS>(w[r], S, shot));
        if ((w[r] & kAloneBit) && (w[r] & last_bit)) {
          if constexpr (NM == 2)
            load_adjoint_state(nm, w[r], st[r]);
          else
            load_node_state<MS, NM == 3>(nm, w[r], S, shot, st[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      const int idx = base + r * TEAM;
      if (w[r] & kAloneBit) {
        const int e = idx / NP;
        const float* src = ts + e * ES + 3 * (idx - e * NP);
        float fx = src[0] + prev[r].x, fy = src[1] + prev[r].y, fz = src[2] + prev[r].z;
        if (w[r] & last_bit) {
          if constexpr (NM == 2) {
            if (rr.y) adjoint_receivers(nm, rr, w[r] & kNodeMask, fx, fy, fz);
            adjoint_node(nm, w[r], st[r], fx, fy, fz);
          } else {
            if constexpr (NM == 3) snapshot_node(nm, w[r], st[r]);
            if (d.nsrc) add_point_sources(d, nm, w[r] & kNodeMask, shot, fx, fy, fz);
            newmark_node<MS>(nm, w[r], S, shot, st[r], fx, fy, fz);
          }
        } else {
          f[node_slot<MS>(w[r], S, shot)] = make_float4(fx, fy, fz, 0.f);
        }
      }
    }
  }
}

// Phase 4b over the CTA: per shared patch node, the sum of its local points' forces in table
// order (its slots, shared-memory offsets of those forces, read as one 16-byte word), then
// one store (first touch) or one read-modify-write, or at the node's last touch (with a
// Newmark mode) its update; the previous values of GB nodes are loaded before any is written.
template <int N, bool COHERENT, bool MS = false, int NM = 0>
__device__ __forceinline__ void patch_write_shared(const PatchDesc& d, const uint16_t* __restrict__ slot_tab,
                                                   const uint16_t* __restrict__ word_tab, float4* __restrict__ f,
                                                   const float* wsb, const SweepNewmark& nm, int S = 1,
                                                   int shot = 0, int2 rr = make_int2(0, 0)) {
  using C = PatchCfg<N>;
  constexpr int T = C::T, GB = NM ? 2 : 4;
  const uint4* __restrict__ slots = reinterpret_cast<const uint4*>(slot_tab + d.slot_off);
  const uint16_t* __restrict__ words = word_tab + d.word_off;
  constexpr uint32_t last_bit = NM ? kPatchLastBit : 0u;
  for (int base = threadIdx.x; base < d.nshared; base += GB * T) {
    uint4 sl[GB];
    uint32_t w[GB];
    float4 prev[GB];
    NodeState st[GB];
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      const int t = base + r * T;
      const int tt = t < d.nshared ? t : 0;
      sl[r] = __ldg(slots + tt);
      w[r] = t < d.nshared ? reinterpret_cast<const uint32_t*>(wsb)[__ldg(words + tt)] : kPatchFirstBit;
    }
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      prev[r] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (!(w[r] & kPatchFirstBit)) prev[r] = load_f<COHERENT>(f + node_slot<MS>(w[r], S, shot));
      if (w[r] & last_bit) {
        if constexpr (NM == 2)
          load_adjoint_state(nm, w[r], st[r]);
        else
          load_node_state<MS, NM == 3>(nm, w[r], S, shot, st[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      const int t = base + r * T;
      if (t < d.nshared) {
        float sx = 0.f, sy = 0.f, sz = 0.f;
        uint4 g4 = sl[r];
        while (true) {
          const uint32_t wd[4] = {g4.x, g4.y, g4.z, g4.w};
          uint32_t chain = 0;
#pragma unroll
          for (int k = 0; k < kPatchSlots; ++k) {
            const uint32_t q = (wd[k >> 1] >> (16 * (k & 1))) & 0xFFFFu;
            if (q == kPatchNoSlot) continue;
            if (q & kPatchChain) {
              chain = q;
              continue;
            }
            const float* F = wsb + q;
            sx += F[0];
            sy += F[1];
            sz += F[2];
          }
          if (!chain) break;
          g4 = __ldg(slots + (chain & ~static_cast<uint32_t>(kPatchChain)));
        }
        float fx = prev[r].x + sx, fy = prev[r].y + sy, fz = prev[r].z + sz;
        if (w[r] & last_bit) {
          if constexpr (NM == 2) {
            if (rr.y) adjoint_receivers(nm, rr, w[r] & kNodeMask, fx, fy, fz);
            adjoint_node(nm, w[r], st[r], fx, fy, fz);
          } else {
            if constexpr (NM == 3) snapshot_node(nm, w[r], st[r]);
            if (d.nsrc) add_point_sources(d, nm, w[r] & kNodeMask, shot, fx, fy, fz);
            newmark_node<MS>(nm, w[r], S, shot, st[r], fx, fy, fz);
          }
        } else {
          f[node_slot<MS>(w[r], S, shot)] = make_float4(fx, fy, fz, 0.f);
        }
      }
    }
  }
}

// One launch per patch colour: one CTA per patch of the colour [p0, p0 + gridDim.x).
// The launches of one sweep are programmatic dependent launches: a colour's CTAs may start
// while the previous colour drains. The first colour of a sweep (p0 == 0) waits for the
// previous grid before anything (that grid may have written u). A later colour reads only u
// (which no colour writes, and which was complete before the first colour began; read from
// L2) and the records until it writes f, so it gathers and evaluates its elements first and
// waits for the previous colour only before its writes.
// With S shots (MS true) the fields are [nglob][S][4] and CTA b takes patch p0 + b / S for
// shot b % S: consecutive CTAs take the shots of one patch, so its records come from DRAM
// once (the first shot's prefetch) and from L2 for the others.
template <int N, bool LO, bool MS, int NM>
__global__ void __launch_bounds__(PatchCfg<N>::T, PatchCfg<N>::MIN_BLOCKS)
    patch_forces_kernel(const float* __restrict__ rec, const PatchDesc* __restrict__ desc,
                        const uint16_t* __restrict__ slot_tab, const uint16_t* __restrict__ word_tab,
                        const float4* __restrict__ u, float4* __restrict__ f, int p0, int S_arg,
                        const SweepNewmark nm) {
  using C = PatchCfg<N>;
  extern __shared__ float4 smem4[];
  float* wsb = reinterpret_cast<float*>(smem4);
  const int S = MS ? S_arg : 1;
  const int P = p0 + (MS ? static_cast<int>(blockIdx.x) / S : static_cast<int>(blockIdx.x));
  const int shot = MS ? static_cast<int>(blockIdx.x) - (P - p0) * S : 0;
  const PatchDesc d = desc[P];
  // 0. records to L2 (by the patch's first shot)
  if (shot == 0 && threadIdx.x < d.nelem)
    prefetch_l2(rec + static_cast<size_t>(d.slot0 + threadIdx.x) * C::REC, kForceFields * C::NP * sizeof(float));
  if (p0 == 0) wait_prerequisite_grid();
  allow_dependent_grid();
  // before the wait, u comes from L2 (the coherence point), never from a line this SM's L1
  // may hold from before the grid that wrote u
  patch_gather_compute<N, LO, MS, NM>(d, rec, u, wsb, p0 != 0, S, shot, &nm);
  if (p0 != 0) wait_prerequisite_grid();  // the previous colour's writes to f
  const int2 rr = NM == 2 && nm.recv_range ? make_int2(nm.recv_range[2 * P], nm.recv_range[2 * P + 1]) : make_int2(0, 0);
  patch_write_alone<N, false, MS, NM>(d, f, wsb, nm, S, shot, rr);  // no wait for the other teams
  __syncthreads();
  patch_write_shared<N, false, MS, NM>(d, slot_tab, word_tab, f, wsb, nm, S, shot, rr);
}

// ---------------------------------------------------------------------------------------
// Shot pairs. With several shots of one model (fields [nglob][S][4]), a CTA takes one patch
// for two shots: every thread carries both shots' values as float32 pairs (shot 2k in .x,
// 2k + 1 in .y), so one packed fma serves both shots, and every geometry and modulus value
// read from the records serves both. The workspace is the single-shot layout with every
// float widened to a pair (an element at twice its single-shot offset; u/F, eta and zeta
// values as [NP][3] pairs, the ibool words at stride 2), so the patch tables' shared-memory
// offsets apply doubled. Line owners throughout (Sec. II-B phases as in the single-shot core).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float2 bcast2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
  unsigned long long ra, rb, rd;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
  return d;
}
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) {
  unsigned long long ra, rb, rd;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
  return d;
}

// Phases 2-3 of one team's elements for a shot pair (ES2 floats per element workspace).
template <int N, int KIND, int TEAM, int ES2, class RecOf>
__device__ __forceinline__ void team_element_forces_pair(float* ts2, int tl, int ne, int team, RecOf rec_of) {
  constexpr int NP = N * N * N, NL = N * N;
  const float* __restrict__ W = c_w;
  const int le = tl / NL;
  const int line = tl - le * NL;
  const int a = line % N;
  const int b = line / N;
  const bool active = le < ne;
  float2* su = reinterpret_cast<float2*>(ts2 + (active ? le : 0) * ES2);  // u, then F: [NP][3]
  float2* se = su + 3 * NP;                                                 // eta values [NP][3]
  float2* sz = su + 6 * NP;                                                 // zeta values [NP][3]
  const float* __restrict__ r = rec_of(active ? le : 0);

  // 2a. eta derivatives along the eta-line (i, k) = (a, b), zeta derivatives along the
  //     zeta-line (i, j) = (a, b), component by component
  if (active) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float2 ve[N], vz[N];
#pragma unroll
      for (int l = 0; l < N; ++l) {
        ve[l] = su[3 * (a + N * (l + N * b)) + c];
        vz[l] = su[3 * (a + N * (b + N * l)) + c];
      }
#pragma unroll
      for (int m = 0; m < N; ++m) {
        float2 de = make_float2(0.f, 0.f), dz = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l < N; ++l) {
          de = ffma2(c_h2[m * N + l], ve[l], de);
          dz = ffma2(c_h2[m * N + l], vz[l], dz);
        }
        se[3 * (a + N * (m + N * b)) + c] = de;
        sz[3 * (a + N * (b + N * m)) + c] = dz;
      }
    }
  }
  team_sync<KIND, TEAM>(team);

  // 2b. along the xi-line (j, k) = (a, b): xi derivatives, Jacobian map, Hooke stress,
  //     fluxes (the record values broadcast to both shots); the xi-flux transposed product in
  //     registers, the eta and zeta fluxes over the derivatives
  float2 fx[N], fy[N], fz[N];
  {
    float2 ux[N], uy[N], uz[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int p = i + N * line;
      ux[i] = su[3 * p];
      uy[i] = su[3 * p + 1];
      uz[i] = su[3 * p + 2];
      fx[i] = fy[i] = fz[i] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
      float2 dxi_x = make_float2(0.f, 0.f), dxi_y = dxi_x, dxi_z = dxi_x;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        dxi_x = ffma2(c_h2[i * N + l], ux[l], dxi_x);
        dxi_y = ffma2(c_h2[i * N + l], uy[l], dxi_y);
        dxi_z = ffma2(c_h2[i * N + l], uz[l], dxi_z);
      }
      const int p3 = 3 * (i + N * line);
      const float2 det_x = se[p3], det_y = se[p3 + 1], det_z = se[p3 + 2];
      const float2 dze_x = sz[p3], dze_y = sz[p3 + 1], dze_z = sz[p3 + 2];
      const int q = i * NL + line;
      float2 G[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) G[c] = bcast2(active ? __ldg(r + (kG + c) * NP + q) : 0.f);
      const float kappa = active ? __ldg(r + kJKappa * NP + q) : 0.f;  // J kappa
      const float mu = active ? __ldg(r + kJMu * NP + q) : 0.f;        // J mu

      const float2 uxx = ffma2(dze_x, G[6], ffma2(det_x, G[3], fmul2(dxi_x, G[0])));
      const float2 uxy = ffma2(dze_x, G[7], ffma2(det_x, G[4], fmul2(dxi_x, G[1])));
      const float2 uxz = ffma2(dze_x, G[8], ffma2(det_x, G[5], fmul2(dxi_x, G[2])));
      const float2 uyx = ffma2(dze_y, G[6], ffma2(det_y, G[3], fmul2(dxi_y, G[0])));
      const float2 uyy = ffma2(dze_y, G[7], ffma2(det_y, G[4], fmul2(dxi_y, G[1])));
      const float2 uyz = ffma2(dze_y, G[8], ffma2(det_y, G[5], fmul2(dxi_y, G[2])));
      const float2 uzx = ffma2(dze_z, G[6], ffma2(det_z, G[3], fmul2(dxi_z, G[0])));
      const float2 uzy = ffma2(dze_z, G[7], ffma2(det_z, G[4], fmul2(dxi_z, G[1])));
      const float2 uzz = ffma2(dze_z, G[8], ffma2(det_z, G[5], fmul2(dxi_z, G[2])));

      // J sigma (J kappa and J mu from the record)
      const float2 lam = bcast2(kappa - (2.f / 3.f) * mu);
      const float2 mu2 = bcast2(2.f * mu), mu1 = bcast2(mu);
      const float2 ltr = fmul2(lam, fadd2(fadd2(uxx, uyy), uzz));
      const float2 sxx = ffma2(mu2, uxx, ltr);
      const float2 syy = ffma2(mu2, uyy, ltr);
      const float2 szz = ffma2(mu2, uzz, ltr);
      const float2 sxy = fmul2(mu1, fadd2(uxy, uyx));
      const float2 sxz = fmul2(mu1, fadd2(uxz, uzx));
      const float2 syz = fmul2(mu1, fadd2(uyz, uzy));

      const float2 txi_x = ffma2(sxz, G[2], ffma2(sxy, G[1], fmul2(sxx, G[0])));
      const float2 txi_y = ffma2(syz, G[2], ffma2(syy, G[1], fmul2(sxy, G[0])));
      const float2 txi_z = ffma2(szz, G[2], ffma2(syz, G[1], fmul2(sxz, G[0])));
#pragma unroll
      for (int ip = 0; ip < N; ++ip) {
        fx[ip] = ffma2(c_hw2[i * N + ip], txi_x, fx[ip]);
        fy[ip] = ffma2(c_hw2[i * N + ip], txi_y, fy[ip]);
        fz[ip] = ffma2(c_hw2[i * N + ip], txi_z, fz[ip]);
      }
      if (active) {
        se[p3] = ffma2(sxz, G[5], ffma2(sxy, G[4], fmul2(sxx, G[3])));
        se[p3 + 1] = ffma2(syz, G[5], ffma2(syy, G[4], fmul2(sxy, G[3])));
        se[p3 + 2] = ffma2(szz, G[5], ffma2(syz, G[4], fmul2(sxz, G[3])));
        sz[p3] = ffma2(sxz, G[8], ffma2(sxy, G[7], fmul2(sxx, G[6])));
        sz[p3 + 1] = ffma2(syz, G[8], ffma2(syy, G[7], fmul2(sxy, G[6])));
        sz[p3 + 2] = ffma2(szz, G[8], ffma2(syz, G[7], fmul2(sxz, G[6])));
      }
    }
  }
  team_sync<KIND, TEAM>(team);

  // 3. eta and zeta transposed products along the eta- and zeta-lines, in place
  if (active) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float2 ve[N], vz[N];
#pragma unroll
      for (int l = 0; l < N; ++l) {
        ve[l] = se[3 * (a + N * (l + N * b)) + c];
        vz[l] = sz[3 * (a + N * (b + N * l)) + c];
      }
#pragma unroll
      for (int m = 0; m < N; ++m) {
        float2 te = make_float2(0.f, 0.f), tz = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l < N; ++l) {
          te = ffma2(c_hw2[l * N + m], ve[l], te);
          tz = ffma2(c_hw2[l * N + m], vz[l], tz);
        }
        se[3 * (a + N * (m + N * b)) + c] = te;
        sz[3 * (a + N * (b + N * m)) + c] = tz;
      }
    }
  }
  team_sync<KIND, TEAM>(team);

  // 3b. element forces along the xi-line into the (now free) u slots
  if (active) {
    const float wj = W[a], wk = W[b];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const float wi = W[i];
      const float2 cjk = bcast2(-(wj * wk)), cik = bcast2(-(wi * wk)), cij = bcast2(-(wi * wj));
      const int p = 3 * (i + N * line);
      su[p] = ffma2(cij, sz[p], ffma2(cik, se[p], fmul2(cjk, fx[i])));
      su[p + 1] = ffma2(cij, sz[p + 1], ffma2(cik, se[p + 1], fmul2(cjk, fy[i])));
      su[p + 2] = ffma2(cij, sz[p + 2], ffma2(cik, se[p + 2], fmul2(cjk, fz[i])));
    }
  }
  team_sync<KIND, TEAM>(team);
}

// Points a thread gathers per pass in the pair kernel (all their loads in flight together),
// lone points and shared nodes it writes per pass (GB300, 48^3 at NGLL 5, 32 shots: a
// gather batch of 2 beats 4; write batches of 2 beat 1 by 7 %).
constexpr int kPairGatherBatch = 2;
constexpr int kPairWriteBatch = 4;
constexpr int kPairSharedBatch = 2;

// Phases 1-3 of one patch for a shot pair (s0, s0 + 1; the second absent when has1 is false:
// its lanes then carry a copy of the first, never written back).
template <int N, bool NM>
__device__ __forceinline__ void patch_gather_compute_pair(const PatchDesc& d, const float* __restrict__ rec,
                                                          const float4* __restrict__ u, float* wsb2, bool u_from_l2,
                                                          int S, int s0, bool has1, const SweepNewmark& nm) {
  using C = PatchCfg<N>;
  constexpr int NP = C::NP, E = C::E, TEAM = C::TEAM, ES2 = 2 * C::ES, REC = C::REC, GB = kPairGatherBatch;
  const int team = threadIdx.x / TEAM;
  const int tl = threadIdx.x - team * TEAM;
  const int ne = min(E, d.nelem - team * E);
  const float* __restrict__ trec = rec + static_cast<size_t>(d.slot0 + team * E) * REC;
  const int s1 = has1 ? s0 + 1 : s0;
  float* ts2 = wsb2 + team * 2 * C::TS;
  for (int base = tl; base < ne * NP; base += GB * TEAM) {
    uint32_t w[GB];
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      const int idx = base + r * TEAM;
      const int le = idx / NP;
      w[r] = idx < ne * NP ? __float_as_uint(__ldg(trec + static_cast<size_t>(le) * REC + (idx - le * NP))) : 0u;
    }
    if constexpr (NM) {
#pragma unroll
      for (int r = 0; r < GB; ++r)
        if (w[r] & kPatchLastBit) {
          prefetch_l2_line(reinterpret_cast<const float4*>(nm.v) + node_slot<true>(w[r], S, s0));
          prefetch_l2_line(nm.minv + (w[r] & kNodeMask));
        }
    }
    float4 q0[GB], q1[GB];
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      const float4* pu = u + node_slot<true>(w[r], S, s0);
      q0[r] = u_from_l2 ? __ldcg(pu) : __ldg(pu);
      q1[r] = u_from_l2 ? __ldcg(pu + (s1 - s0)) : __ldg(pu + (s1 - s0));
    }
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      const int idx = base + r * TEAM;
      if (idx < ne * NP) {
        const int le = idx / NP;
        const int p = idx - le * NP;
        float* eb2 = ts2 + le * ES2;
        reinterpret_cast<uint32_t*>(eb2 + 18 * NP)[2 * p] = w[r];
        float2* pu2 = reinterpret_cast<float2*>(eb2) + 3 * p;
        pu2[0] = make_float2(q0[r].x, q1[r].x);
        pu2[1] = make_float2(q0[r].y, q1[r].y);
        pu2[2] = make_float2(q0[r].z, q1[r].z);
      }
    }
  }
  if (C::KIND == 2 || ne > 0) {
    team_sync<C::KIND, TEAM>(team);
    team_element_forces_pair<N, C::KIND, TEAM, ES2>(ts2, tl, ne, team,
                                                    [&](int le) { return trec + static_cast<size_t>(le) * REC; });
  }
}

// The write of one node for one shot of the pair: stored (first touch), added (later
// touches), or (NM, last touch) the sources and the Newmark update.
template <bool NM>
__device__ __forceinline__ void write_node_shot(const PatchDesc& d, const SweepNewmark& nm, float4* __restrict__ f,
                                                uint32_t w, int S, int shot, float4 prev, const NodeState& st,
                                                float fx, float fy, float fz) {
  fx += prev.x;
  fy += prev.y;
  fz += prev.z;
  if (NM && (w & kPatchLastBit)) {
    if (d.nsrc) add_point_sources(d, nm, w & kNodeMask, shot, fx, fy, fz);
    newmark_node<true>(nm, w, S, shot, st, fx, fy, fz);
  } else {
    f[node_slot<true>(w, S, shot)] = make_float4(fx, fy, fz, 0.f);
  }
}

// Phase 4a for a shot pair (the points alone at their patch node, team by team; the loads
// of GB points in flight before any is written).
template <int N, bool NM>
__device__ __forceinline__ void patch_write_alone_pair(const PatchDesc& d, float4* __restrict__ f, const float* wsb2,
                                                       const SweepNewmark& nm, int S, int s0, bool has1) {
  using C = PatchCfg<N>;
  constexpr int NP = C::NP, E = C::E, TEAM = C::TEAM, ES2 = 2 * C::ES, GB = kPairWriteBatch;
  const int team = threadIdx.x / TEAM;
  const int tl = threadIdx.x - team * TEAM;
  const int ne = min(E, d.nelem - team * E);
  const float* ts2 = wsb2 + team * 2 * C::TS;
  const int s1 = has1 ? s0 + 1 : s0;
  for (int base = tl; base < ne * NP; base += GB * TEAM) {
    uint32_t w[GB];
    float4 prev0[GB], prev1[GB];
    NodeState st0[GB], st1[GB];
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      const int idx = base + r * TEAM;
      w[r] = 0u;
      prev0[r] = prev1[r] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (idx < ne * NP) {
        const int e = idx / NP;
        w[r] = reinterpret_cast<const uint32_t*>(ts2 + e * ES2 + 18 * NP)[2 * (idx - e * NP)];
        if ((w[r] & kAloneBit) && !(w[r] & kPatchFirstBit)) {
          prev0[r] = load_f<false>(f + node_slot<true>(w[r], S, s0));
          prev1[r] = load_f<false>(f + node_slot<true>(w[r], S, s1));
        }
        if (NM && (w[r] & kAloneBit) && (w[r] & kPatchLastBit)) {
          load_node_state<true>(nm, w[r], S, s0, st0[r]);
          load_node_state<true>(nm, w[r], S, s1, st1[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      const int idx = base + r * TEAM;
      if (w[r] & kAloneBit) {
        const int e = idx / NP;
        const float2* F = reinterpret_cast<const float2*>(ts2 + e * ES2) + 3 * (idx - e * NP);
        const float2 Fx = F[0], Fy = F[1], Fz = F[2];
        write_node_shot<NM>(d, nm, f, w[r], S, s0, prev0[r], st0[r], Fx.x, Fy.x, Fz.x);
        if (has1) write_node_shot<NM>(d, nm, f, w[r], S, s1, prev1[r], st1[r], Fx.y, Fy.y, Fz.y);
      }
    }
  }
}

// Phase 4b for a shot pair over the CTA (the shared patch nodes, their slots summed as pairs;
// the loads of GB nodes in flight before any is written).
template <int N, bool NM>
__device__ __forceinline__ void patch_write_shared_pair(const PatchDesc& d, const uint16_t* __restrict__ slot_tab,
                                                        const uint16_t* __restrict__ word_tab, float4* __restrict__ f,
                                                        const float* wsb2, const SweepNewmark& nm, int S, int s0,
                                                        bool has1) {
  using C = PatchCfg<N>;
  constexpr int T = C::T, GB = kPairSharedBatch;
  const uint4* __restrict__ slots = reinterpret_cast<const uint4*>(slot_tab + d.slot_off);
  const uint16_t* __restrict__ words = word_tab + d.word_off;
  const int s1 = has1 ? s0 + 1 : s0;
  for (int base = threadIdx.x; base < d.nshared; base += GB * T) {
    uint4 sl[GB];
    uint32_t w[GB];
    float4 prev0[GB], prev1[GB];
    NodeState st0[GB], st1[GB];
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      const int t = base + r * T;
      const int tt = t < d.nshared ? t : 0;
      sl[r] = __ldg(slots + tt);
      w[r] = t < d.nshared ? reinterpret_cast<const uint32_t*>(wsb2)[2 * static_cast<uint32_t>(__ldg(words + tt))]
                           : kPatchFirstBit;
    }
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      prev0[r] = prev1[r] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (!(w[r] & kPatchFirstBit)) {
        prev0[r] = load_f<false>(f + node_slot<true>(w[r], S, s0));
        prev1[r] = load_f<false>(f + node_slot<true>(w[r], S, s1));
      }
      if (NM && (w[r] & kPatchLastBit)) {
        load_node_state<true>(nm, w[r], S, s0, st0[r]);
        load_node_state<true>(nm, w[r], S, s1, st1[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      if (base + r * T >= d.nshared) continue;
      float2 sx = make_float2(0.f, 0.f), sy = sx, sz = sx;
      uint4 g4 = sl[r];
      while (true) {
        const uint32_t wd[4] = {g4.x, g4.y, g4.z, g4.w};
        uint32_t chain = 0;
#pragma unroll
        for (int k = 0; k < kPatchSlots; ++k) {
          const uint32_t q = (wd[k >> 1] >> (16 * (k & 1))) & 0xFFFFu;
          if (q == kPatchNoSlot) continue;
          if (q & kPatchChain) {
            chain = q;
            continue;
          }
          const float2* F = reinterpret_cast<const float2*>(wsb2 + 2 * q);
          sx = fadd2(sx, F[0]);
          sy = fadd2(sy, F[1]);
          sz = fadd2(sz, F[2]);
        }
        if (!chain) break;
        g4 = __ldg(slots + (chain & ~static_cast<uint32_t>(kPatchChain)));
      }
      write_node_shot<NM>(d, nm, f, w[r], S, s0, prev0[r], st0[r], sx.x, sy.x, sz.x);
      if (has1) write_node_shot<NM>(d, nm, f, w[r], S, s1, prev1[r], st1[r], sx.y, sy.y, sz.y);
    }
  }
}

// Shared memory of the pair kernel and the CTAs per SM it is compiled for.
template <int N>
struct PairCfg {
  static constexpr int SMEM = 2 * PatchCfg<N>::SMEM;
  static constexpr int FIT = (227 * 1024) / (SMEM + 1024);
  // at most the CTAs whose register share holds the pair core without large spills (about
  // 128 registers a thread from NGLL 5 up)
  static constexpr int CAP = N >= 5 ? 2 : 3;
  static constexpr int MIN_BLOCKS = FIT < 1 ? 1 : FIT > CAP ? CAP : FIT;
  static_assert(SMEM <= 227 * 1024, "pair workspace exceeds shared memory");
};

// One launch per patch colour for S shots: CTA b takes patch p0 + b / ceil(S/2) for the shot
// pair (2k, 2k + 1), k = b % ceil(S/2) (with odd S the last pair has one shot). The pairs of
// one patch are consecutive CTAs, so its records come from DRAM once (the first pair's
// prefetch) and from L2 for the others. Launch order and waits as in patch_forces_kernel.
template <int N, bool NM>
__global__ void __launch_bounds__(PatchCfg<N>::T, PairCfg<N>::MIN_BLOCKS)
    patch_forces_pair_kernel(const float* __restrict__ rec, const PatchDesc* __restrict__ desc,
                             const uint16_t* __restrict__ slot_tab, const uint16_t* __restrict__ word_tab,
                             const float4* __restrict__ u, float4* __restrict__ f, int p0, int S,
                             const SweepNewmark nm) {
  using C = PatchCfg<N>;
  extern __shared__ float4 smem4[];
  float* wsb2 = reinterpret_cast<float*>(smem4);
  const int SP = (S + 1) / 2;
  const int P = p0 + static_cast<int>(blockIdx.x) / SP;
  const int k = static_cast<int>(blockIdx.x) - (P - p0) * SP;
  const int s0 = 2 * k;
  const bool has1 = s0 + 1 < S;
  const PatchDesc d = desc[P];
  if (k == 0 && threadIdx.x < d.nelem)
    prefetch_l2(rec + static_cast<size_t>(d.slot0 + threadIdx.x) * C::REC, kForceFields * C::NP * sizeof(float));
  if (p0 == 0) wait_prerequisite_grid();
  allow_dependent_grid();
  patch_gather_compute_pair<N, NM>(d, rec, u, wsb2, p0 != 0, S, s0, has1, nm);
  if (p0 != 0) wait_prerequisite_grid();
  patch_write_alone_pair<N, NM>(d, f, wsb2, nm, S, s0, has1);
  __syncthreads();
  patch_write_shared_pair<N, NM>(d, slot_tab, word_tab, f, wsb2, nm, S, s0, has1);
}

// Persistent form: one sweep (all patch colours) in one launch. CTAs take patches in sweep
// order from sync->next, the next one as soon as they start on the current one (whose
// records are then bulk-prefetched into L2 while the current one is processed). A patch of
// colour c > 0 writes f only once every patch of colour c - 1 has finished
// (sync->done[c - 1] == the colour's patch count; one thread waits with a bounded spin,
// then the CTA reads f from L2), then counts itself into sync->done[c]. Every patch waits
// only on patches taken before it, so the sweep completes however many CTAs are resident.
// The last CTA to leave resets the counters for the next sweep. A wait that gives up sets
// sync->err and ends its CTA early (the host reports SEM_ETIMEOUT).
struct SweepShared {
  PatchDesc d;  // the current patch
  int next;     // the patch taken next
  int color;    // colour of the current patch
  int ready;    // every patch of the previous colour had finished when the patch began
  int abort;
};

template <int N>
__device__ __forceinline__ void prefetch_patch_records(const float* __restrict__ rec,
                                                       const PatchDesc* __restrict__ desc, int P, int npatch) {
  using C = PatchCfg<N>;
  if (P < npatch && threadIdx.x < 32) {
    const PatchDesc dn = desc[P];
    if (static_cast<int>(threadIdx.x) < dn.nelem)
      prefetch_l2(rec + static_cast<size_t>(dn.slot0 + threadIdx.x) * C::REC, kForceFields * C::NP * sizeof(float));
  }
}

// Patches of the previous colour (c - 1) needed before a patch of colour c may write.
__device__ __forceinline__ unsigned int prior_colour_count(const int* __restrict__ color_end, int c,
                                                           unsigned int stall) {
  // (stall != 0: a count that never arrives, so that a test can make the wait give up)
  return stall ? 0xFFFFFFFFu : static_cast<unsigned int>(color_end[c - 1] - (c > 1 ? color_end[c - 2] : 0));
}

// One patch of the persistent sweep (kept out of line so that nothing of its body is held
// in registers across patches). Returns the patch taken next, or -1 after a wait gave up.
// When the previous colour had already finished as the patch began (the common case once a
// colour is under way), the teams write their lone points as soon as their elements are
// done, as in the per-colour kernel; otherwise one thread waits (bounded) first.
template <int N, bool LO>
__device__ __noinline__ int sweep_one_patch(int P, const float* __restrict__ rec, const PatchDesc* __restrict__ desc,
                                            const uint16_t* __restrict__ slot_tab,
                                            const uint16_t* __restrict__ word_tab, const float4* __restrict__ u,
                                            float4* __restrict__ f, int npatch, const int* __restrict__ color_end,
                                            unsigned int stall, SweepSync* sync, SweepShared* sh, float* wsb) {
  __syncthreads();  // every thread is done with sh before it is replaced
  if (threadIdx.x == 0) {
    sh->d = desc[P];
    sh->next = static_cast<int>(atomicAdd(&sync->next, 1u));
    int c = 0;  // the first colour whose range ends beyond P
    while (color_end[c] <= P) ++c;
    sh->color = c;
    sh->ready = c == 0 || ld_acquire_gpu(&sync->done[c - 1]) >= prior_colour_count(color_end, c, stall);
  }
  __syncthreads();
  const PatchDesc& d = sh->d;
  const SweepNewmark none{};  // the persistent sweep assembles forces only
  prefetch_patch_records<N>(rec, desc, sh->next, npatch);
  patch_gather_compute<N, LO>(d, rec, u, wsb, false);
  const int c = sh->color;
  if (sh->ready) {
    patch_write_alone<N, true>(d, f, wsb, none);
    __syncthreads();
  } else {
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned int need = prior_colour_count(color_end, c, stall);
      unsigned int spins = 0;
      while (ld_acquire_gpu(&sync->done[c - 1]) < need) {
        if (++spins > kSweepSpinLimit) {
          atomicExch(&sync->err, 1);
          sh->abort = 1;
          break;
        }
        __nanosleep(128);
      }
    }
    __syncthreads();  // the wait is over for the CTA
    if (sh->abort) return -1;
    patch_write_alone<N, true>(d, f, wsb, none);
  }
  patch_write_shared<N, true>(d, slot_tab, word_tab, f, wsb, none);
  __syncthreads();  // all of the patch's writes issued before it counts as done
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&sync->done[c], 1u);
  }
  return sh->next;
}

template <int N, bool LO>
__global__ void __launch_bounds__(PatchCfg<N>::T, PatchCfg<N>::MIN_BLOCKS)
    patch_sweep_kernel(const float* __restrict__ rec, const PatchDesc* __restrict__ desc,
                       const uint16_t* __restrict__ slot_tab, const uint16_t* __restrict__ word_tab,
                       const float4* __restrict__ u, float4* __restrict__ f, int npatch,
                       const int* __restrict__ color_end, int ncolors, unsigned int stall, SweepSync* sync) {
  extern __shared__ float4 smem4[];
  float* wsb = reinterpret_cast<float*>(smem4);
  __shared__ SweepShared sh;
  wait_prerequisite_grid();  // the previous sweep's counter reset and the previous grid's u, f
  if (threadIdx.x == 0) {
    sh.next = static_cast<int>(atomicAdd(&sync->next, 1u));
    sh.abort = 0;
    sh.ready = 0;
  }
  __syncthreads();
  int P = sh.next;
  prefetch_patch_records<N>(rec, desc, P, npatch);
  while (P >= 0 && P < npatch)
    P = sweep_one_patch<N, LO>(P, rec, desc, slot_tab, word_tab, u, f, npatch, color_end, stall, sync, &sh, wsb);
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&sync->exited, 1u) == gridDim.x - 1) {  // every CTA has left: reset
      sync->next = 0u;
      for (int c = 0; c < ncolors; ++c) sync->done[c] = 0u;
      sync->exited = 0u;
      __threadfence();
    }
  }
}

// ---------------------------------------------------------------------------------------
// Group sweep: the persistent form over several models of one order (see GroupLaunch). CTAs
// take items in order from sync->next; an item is located by a binary search over the runs
// of items (GroupSeg), the patch of its model evaluated as in sweep_one_patch, and counted
// into sync->done[model][colour]. Every item waits only on items of its own model taken
// before it, so the sweep completes however many CTAs are resident; a bounded wait that
// gives up sets sync->err and ends its CTA (the host reports SEM_ETIMEOUT).
// ---------------------------------------------------------------------------------------
struct GroupShared {
  PatchDesc d;
  GroupModel m;
  int model;
  int color;
  int next;   // the item taken next
  int ready;
  int abort;
};

__device__ __forceinline__ int group_seg_of(const GroupSeg* __restrict__ segs, int nseg, int item) {
  int lo = 0, hi = nseg - 1;  // the last run whose first item is <= item
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (segs[mid].item0 <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Patches of colour c - 1 of a model needed before its patch of colour c may write.
__device__ __forceinline__ unsigned int group_prior_count(const GroupModel& m, int c, unsigned int stall) {
  return stall ? 0xFFFFFFFFu
               : static_cast<unsigned int>(__ldg(m.color_end + c - 1) - (c > 1 ? __ldg(m.color_end + c - 2) : 0));
}

template <int N>
__device__ __forceinline__ void group_prefetch_item(const GroupLaunch& L, int item) {
  using C = PatchCfg<N>;
  if (item < 0 || item >= L.nitems || threadIdx.x >= 32) return;
  const GroupSeg sg = L.segs[group_seg_of(L.segs, L.nseg, item)];
  const GroupModel& m = L.models[sg.model];
  const PatchDesc dn = m.desc[sg.p0 + item - sg.item0];
  if (static_cast<int>(threadIdx.x) < dn.nelem)
    prefetch_l2(m.rec + static_cast<size_t>(dn.slot0 + threadIdx.x) * C::REC, kForceFields * C::NP * sizeof(float));
}

template <int N, bool LO>
__device__ __noinline__ int group_one_item(int item, const GroupLaunch L, GroupShared* sh, float* wsb) {
  __syncthreads();  // every thread is done with sh before it is replaced
  if (threadIdx.x == 0) {
    const GroupSeg sg = L.segs[group_seg_of(L.segs, L.nseg, item)];
    sh->m = L.models[sg.model];
    sh->d = sh->m.desc[sg.p0 + item - sg.item0];
    sh->model = sg.model;
    sh->color = sg.color;
    sh->next = static_cast<int>(atomicAdd(&L.sync->next, 1u));
    const int c = sg.color;
    sh->ready = c == 0 || ld_acquire_gpu(&L.sync->done[sg.model * kMaxSweepColors + c - 1]) >=
                              group_prior_count(sh->m, c, L.stall);
  }
  __syncthreads();
  const PatchDesc& d = sh->d;
  const GroupModel& m = sh->m;
  const SweepNewmark none{};
  group_prefetch_item<N>(L, sh->next);
  float4* f = reinterpret_cast<float4*>(m.f);
  patch_gather_compute<N, LO>(d, m.rec, reinterpret_cast<const float4*>(m.u), wsb, false);
  const int c = sh->color;
  unsigned int* done = &L.sync->done[sh->model * kMaxSweepColors];
  if (sh->ready) {
    patch_write_alone<N, true>(d, f, wsb, none);
    __syncthreads();
  } else {
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned int need = group_prior_count(m, c, L.stall);
      unsigned int spins = 0;
      while (ld_acquire_gpu(&done[c - 1]) < need) {
        if (++spins > kSweepSpinLimit) {
          atomicExch(&L.sync->err, 1);
          sh->abort = 1;
          break;
        }
        __nanosleep(128);
      }
    }
    __syncthreads();  // the wait is over for the CTA
    if (sh->abort) return -1;
    patch_write_alone<N, true>(d, f, wsb, none);
  }
  patch_write_shared<N, true>(d, m.slots, m.words, f, wsb, none);
  __syncthreads();  // all of the patch's writes issued before it counts as done
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&done[c], 1u);
  }
  return sh->next;
}

template <int N, bool LO>
__global__ void __launch_bounds__(PatchCfg<N>::T, PatchCfg<N>::MIN_BLOCKS) group_sweep_kernel(const GroupLaunch L) {
  extern __shared__ float4 smem4[];
  float* wsb = reinterpret_cast<float*>(smem4);
  __shared__ GroupShared sh;
  wait_prerequisite_grid();  // the previous sweep's counter reset and the previous grids' u, f
  if (threadIdx.x == 0) {
    sh.next = static_cast<int>(atomicAdd(&L.sync->next, 1u));
    sh.abort = 0;
    sh.ready = 0;
  }
  __syncthreads();
  int item = sh.next;
  group_prefetch_item<N>(L, item);
  while (item >= 0 && item < L.nitems) item = group_one_item<N, LO>(item, L, &sh, wsb);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    sh.ready = atomicAdd(&L.sync->exited, 1u) == gridDim.x - 1;  // every CTA has left: reset
  }
  __syncthreads();
  if (sh.ready) {
    for (int t = threadIdx.x; t < L.nmodels * kMaxSweepColors; t += blockDim.x) L.sync->done[t] = 0u;
    __syncthreads();
    if (threadIdx.x == 0) {
      L.sync->next = 0u;
      L.sync->exited = 0u;
      __threadfence();
    }
  }
}

// ---------------------------------------------------------------------------------------
// Material sensitivities (the discrete adjoint of the explicit scheme): at one adjoint step,
// for every local point q of every element
//   g_rho[q]   += c_m * w_q J_q lam_I . (u_hi - 2 u_mid + u_lo)_I          (I = ibool(q))
//   g_kappa[q] += c_k * w_q J_q tr e(lam) tr e(u_mid)
//   g_mu[q]    += c_k * w_q J_q 2 (e(lam) : e(u_mid) - tr e(lam) tr e(u_mid) / 3)
// with e the discrete strain (the same derivatives and chain rule as the force kernel),
// c_m = -1 and c_k = -dt^2. lam is the adjoint field in the solver layout [nglob][4] (internal
// node order), the u_* displacement snapshots [nglob][3] in caller node order (perm maps) or,
// with perm null, in internal order. The terms are formed in float32 (the second difference
// as (u_hi - u_mid) - (u_mid - u_lo), which keeps the digits the plain form cancels) and
// added to float32 partial sums per local point in record order (element, q = i N^2 +
// line), which the host flushes into float64 accumulators every few dozen steps. No two
// threads write the same point, so there are no colours here.
// ---------------------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(ForceCfg<N>::T)
    sensitivity_kernel(const float* __restrict__ rec, const int* __restrict__ perm, const float* __restrict__ lam,
                       const float* __restrict__ u_lo,
                       const float* __restrict__ u_mid, const float* __restrict__ u_hi, float* __restrict__ g_rho,
                       float* __restrict__ g_kappa, float* __restrict__ g_mu, int nspec, double c_m, double c_k,
                       const DevCtl* __restrict__ idx) {
  using C = ForceCfg<N>;
  if (idx) {  // the snapshots of the step the device's adjoint counter names
    const float* base = idx->adj_u + static_cast<long long>(idx->adj_js - 1) * idx->adj_n3;
    u_lo = base;
    u_mid = base + idx->adj_n3;
    u_hi = base + 2 * idx->adj_n3;
  }
  constexpr int NP = C::NP, NL = C::NL, E = C::E, REC = C::REC, TEAM = C::TEAM, ES = C::ES;
  static_assert(7 * NP <= ES, "element tile holds lam, u and the mass term");
  extern __shared__ float4 smem4[];
  const float* __restrict__ H = c_h;
  const float* __restrict__ W = c_w;
  const float cm = static_cast<float>(c_m), ck = static_cast<float>(c_k);
  const int team = threadIdx.x / TEAM;
  const int tl = threadIdx.x - team * TEAM;
  const int ebase = (blockIdx.x * C::TEAMS + team) * E;
  const int ne = min(E, nspec - ebase);
  if (C::KIND != 2 && ne <= 0) return;
  float* ts = reinterpret_cast<float*>(smem4) + team * C::TS;
  constexpr int GB = 4;  // points per thread whose loads are in flight together
  for (int base = tl; base < ne * NP; base += GB * TEAM) {
    size_t g[GB];
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      const int idx = base + r * TEAM;
      const int le = idx / NP;
      g[r] = idx < ne * NP
                 ? __float_as_uint(__ldg(rec + static_cast<size_t>(ebase + le) * REC + (idx - le * NP))) & kNodeMask
                 : 0;
    }
    float4 l4[GB];
    float um[GB][3], uh[GB][3], ul[GB][3];
    size_t gc[GB];  // caller node of each point (the snapshots are in caller order)
#pragma unroll
    for (int r = 0; r < GB; ++r) gc[r] = perm ? static_cast<size_t>(__ldg(perm + g[r])) : g[r];
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      l4[r] = __ldg(reinterpret_cast<const float4*>(lam) + g[r]);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        um[r][a] = __ldg(u_mid + 3 * gc[r] + a);
        uh[r][a] = __ldg(u_hi + 3 * gc[r] + a);
        ul[r][a] = __ldg(u_lo + 3 * gc[r] + a);
      }
    }
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      const int idx = base + r * TEAM;
      if (idx >= ne * NP) continue;
      const int le = idx / NP;
      const int p = idx - le * NP;
      float* eb = ts + le * ES;
      const float lv[3] = {l4[r].x, l4[r].y, l4[r].z};
      float dot = 0.f;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        eb[3 * p + a] = lv[a];
        eb[3 * NP + 3 * p + a] = um[r][a];
        dot += lv[a] * ((uh[r][a] - um[r][a]) - (um[r][a] - ul[r][a]));
      }
      eb[6 * NP + p] = dot;
    }
  }
  team_sync<C::KIND, C::TEAM>(team);
  const int le = tl / NL;
  const int line = tl - le * NL;
  const int j = line % N;
  const int k = line / N;
  if (le >= ne) return;  // no barrier follows
  const float* fl = ts + le * ES;
  const float* fu = fl + 3 * NP;
  const float* fm = fl + 6 * NP;
  const float* __restrict__ r = rec + static_cast<size_t>(ebase + le) * REC;
  const size_t out = static_cast<size_t>(ebase + le) * NP;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float dl[3][3], du[3][3];  // [component][reference direction]
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) dl[a][b] = du[a][b] = 0.f;
#pragma unroll
    for (int l = 0; l < N; ++l) {
      const float hi = H[i * N + l], hj = H[j * N + l], hk = H[k * N + l];
      const int px = 3 * (l + N * line), pe = 3 * (i + N * (l + N * k)), pz = 3 * (i + N * (j + N * l));
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        dl[a][0] += hi * fl[px + a];
        dl[a][1] += hj * fl[pe + a];
        dl[a][2] += hk * fl[pz + a];
        du[a][0] += hi * fu[px + a];
        du[a][1] += hj * fu[pe + a];
        du[a][2] += hk * fu[pz + a];
      }
    }
    const int q = i * NL + line;
    float G[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) G[a] = __ldg(r + (kG + a) * NP + q);
    const float jac = __ldg(r + kJac * NP + q);
    float gl[3][3], gu[3][3];  // physical gradients [component][x_d]
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        gl[a][d] = dl[a][0] * G[d] + dl[a][1] * G[3 + d] + dl[a][2] * G[6 + d];
        gu[a][d] = du[a][0] * G[d] + du[a][1] * G[3 + d] + du[a][2] * G[6 + d];
      }
    float ee = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int d = 0; d < 3; ++d) ee += 0.25f * (gl[a][d] + gl[d][a]) * (gu[a][d] + gu[d][a]);
    const float trl = gl[0][0] + gl[1][1] + gl[2][2];
    const float tru = gu[0][0] + gu[1][1] + gu[2][2];
    const float wJ = W[i] * W[j] * W[k] * jac;
    g_rho[out + q] += cm * (wJ * fm[i + N * line]);
    g_kappa[out + q] += ck * (wJ * trl * tru);
    g_mu[out + q] += ck * (2.f * wJ * (ee - trl * tru * (1.f / 3.f)));
  }
}

// Raises a kernel's dynamic shared-memory limit once per device (bit per ordinal).
template <class K>
int raise_smem_limit(std::atomic<unsigned long long>& done, K kernel, int bytes) {
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return 0;
  const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return static_cast<int>(e);
  done.fetch_or(bit, std::memory_order_acq_rel);
  return 0;
}

template <bool MS, bool LO, bool CALLER, bool ATOMIC = false>
int launch_forces_ms(const ForceLaunch& L, cudaStream_t s) {
  using C = ForceCfg<SEM_NGLL>;
  static std::atomic<unsigned long long> attr_done{0};
  const int smem = C::SMEM_FLOATS * static_cast<int>(sizeof(float));
  if (int r = raise_smem_limit(attr_done, forces_kernel<SEM_NGLL, MS, LO, CALLER, ATOMIC>, smem)) return r;
  const int S = MS ? L.shots : 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(((L.e1 - L.e0) * S + C::EPC - 1) / C::EPC);
  cfg.blockDim = dim3(C::T);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return static_cast<int>(cudaLaunchKernelEx(&cfg, forces_kernel<SEM_NGLL, MS, LO, CALLER, ATOMIC>, L.rec, L.elist, L.perm, L.u, L.f, L.e0, L.e1, S));
}

int launch_forces_n(const ForceLaunch& L, cudaStream_t s) {
  if (L.e1 <= L.e0) return 0;
  using C = ForceCfg<SEM_NGLL>;
  const bool lo = L.variant == 0 ? C::LINE_OWNERS : L.variant == 1;  // 0 default, 1 line owners, 2 per point
  if (L.node_stride == 3) {
    if (L.shots != 1 || !L.perm) return static_cast<int>(cudaErrorInvalidValue);
    return launch_forces_ms<false, C::LINE_OWNERS, true>(L, s);
  }
  if (L.node_stride != kNodeStride) return static_cast<int>(cudaErrorInvalidValue);
  if (L.atomic) {
    if (L.shots != 1) return static_cast<int>(cudaErrorInvalidValue);
    return launch_forces_ms<false, C::LINE_OWNERS, false, true>(L, s);
  }
  if (L.shots > 1) return lo ? launch_forces_ms<true, true, false>(L, s) : launch_forces_ms<true, false, false>(L, s);
  return lo ? launch_forces_ms<false, true, false>(L, s) : launch_forces_ms<false, false, false>(L, s);
}

template <bool LO, bool PAIRS>
int launch_patch_lo(const PatchLaunch& L, cudaStream_t s) {
  using C = PatchCfg<SEM_NGLL>;
  static std::atomic<unsigned long long> attr_done{0}, attr_done_n{0}, attr_done_s{0}, attr_done_sn{0}, attr_done_a{0}, attr_done_ns{0}, attr_done_p{0};
  static std::atomic<int> resident[64];  // CTAs of the persistent kernel per SM, per device
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(C::T);
  cfg.dynamicSmemBytes = C::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (L.sync && !PAIRS) {  // one persistent launch for the whole sweep
    if (int r = raise_smem_limit(attr_done_p, patch_sweep_kernel<SEM_NGLL, LO>, C::SMEM)) return r;
    int dev = 0;
    cudaGetDevice(&dev);
    int per_sm = resident[dev & 63].load();
    if (per_sm <= 0) {
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, patch_sweep_kernel<SEM_NGLL, LO>, C::T,
                                                                    C::SMEM);
      if (e != cudaSuccess) return static_cast<int>(e);
      per_sm = per_sm < 1 ? 1 : per_sm;
      resident[dev & 63].store(per_sm);
    }
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return static_cast<int>(e);
    cfg.gridDim = dim3(static_cast<unsigned>(sms * per_sm));
    return static_cast<int>(cudaLaunchKernelEx(&cfg, patch_sweep_kernel<SEM_NGLL, LO>, L.rec, L.desc, L.slots, L.words,
                                               reinterpret_cast<const float4*>(L.u), reinterpret_cast<float4*>(L.f),
                                               L.npatch, L.color_end, L.ncolors, L.stall ? 1u : 0u, L.sync));
  }
  if constexpr (PAIRS) {
    using PC = PairCfg<SEM_NGLL>;
    cfg.dynamicSmemBytes = PC::SMEM;
    cfg.gridDim = dim3(static_cast<unsigned>((L.p1 - L.p0) * ((L.shots + 1) / 2)));
    if (L.nm.mode) {
      if (int r = raise_smem_limit(attr_done_n, patch_forces_pair_kernel<SEM_NGLL, true>, PC::SMEM)) return r;
      return static_cast<int>(cudaLaunchKernelEx(&cfg, patch_forces_pair_kernel<SEM_NGLL, true>, L.rec, L.desc,
                                                 L.slots, L.words, reinterpret_cast<const float4*>(L.u),
                                                 reinterpret_cast<float4*>(L.f), L.p0, L.shots, L.nm));
    }
    if (int r = raise_smem_limit(attr_done, patch_forces_pair_kernel<SEM_NGLL, false>, PC::SMEM)) return r;
    return static_cast<int>(cudaLaunchKernelEx(&cfg, patch_forces_pair_kernel<SEM_NGLL, false>, L.rec, L.desc,
                                               L.slots, L.words, reinterpret_cast<const float4*>(L.u),
                                               reinterpret_cast<float4*>(L.f), L.p0, L.shots, L.nm));
  } else if (L.shots > 1) {  // one CTA per (patch, shot)
    const int S = L.shots;
    cfg.gridDim = dim3(static_cast<unsigned>((L.p1 - L.p0) * S));
    if (L.nm.mode) {
      if (int r = raise_smem_limit(attr_done_sn, patch_forces_kernel<SEM_NGLL, LO, true, 1>, C::SMEM)) return r;
      return static_cast<int>(cudaLaunchKernelEx(&cfg, patch_forces_kernel<SEM_NGLL, LO, true, 1>, L.rec, L.desc,
                                                 L.slots, L.words, reinterpret_cast<const float4*>(L.u),
                                                 reinterpret_cast<float4*>(L.f), L.p0, S, L.nm));
    }
    if (int r = raise_smem_limit(attr_done_s, patch_forces_kernel<SEM_NGLL, LO, true, 0>, C::SMEM)) return r;
    return static_cast<int>(cudaLaunchKernelEx(&cfg, patch_forces_kernel<SEM_NGLL, LO, true, 0>, L.rec, L.desc,
                                               L.slots, L.words, reinterpret_cast<const float4*>(L.u),
                                               reinterpret_cast<float4*>(L.f), L.p0, S, L.nm));
  } else {
    const int S = 1;
    cfg.gridDim = dim3(static_cast<unsigned>(L.p1 - L.p0));
    if (L.nm.mode && L.nm.mode != 3 && L.nm.snap_ctl) {  // a snapshot run's Newmark sweep
      if (int r = raise_smem_limit(attr_done_ns, patch_forces_kernel<SEM_NGLL, LO, false, 3>, C::SMEM)) return r;
      return static_cast<int>(cudaLaunchKernelEx(&cfg, patch_forces_kernel<SEM_NGLL, LO, false, 3>, L.rec, L.desc,
                                                 L.slots, L.words, reinterpret_cast<const float4*>(L.u),
                                                 reinterpret_cast<float4*>(L.f), L.p0, S, L.nm));
    }
    if (L.nm.mode == 3) {  // the adjoint leapfrog at each node's last touch
      if (int r = raise_smem_limit(attr_done_a, patch_forces_kernel<SEM_NGLL, LO, false, 2>, C::SMEM)) return r;
      return static_cast<int>(cudaLaunchKernelEx(&cfg, patch_forces_kernel<SEM_NGLL, LO, false, 2>, L.rec, L.desc,
                                                 L.slots, L.words, reinterpret_cast<const float4*>(L.u),
                                                 reinterpret_cast<float4*>(L.f), L.p0, S, L.nm));
    }
    if (L.nm.mode) {
      if (int r = raise_smem_limit(attr_done_n, patch_forces_kernel<SEM_NGLL, LO, false, 1>, C::SMEM)) return r;
      return static_cast<int>(cudaLaunchKernelEx(&cfg, patch_forces_kernel<SEM_NGLL, LO, false, 1>, L.rec, L.desc,
                                                 L.slots, L.words, reinterpret_cast<const float4*>(L.u),
                                                 reinterpret_cast<float4*>(L.f), L.p0, S, L.nm));
    }
    if (int r = raise_smem_limit(attr_done, patch_forces_kernel<SEM_NGLL, LO, false, 0>, C::SMEM)) return r;
    return static_cast<int>(cudaLaunchKernelEx(&cfg, patch_forces_kernel<SEM_NGLL, LO, false, 0>, L.rec, L.desc,
                                               L.slots, L.words, reinterpret_cast<const float4*>(L.u),
                                               reinterpret_cast<float4*>(L.f), L.p0, S, L.nm));
  }
}

template <bool LO>
int launch_group_lo(const GroupLaunch& L, cudaStream_t s) {
  using C = PatchCfg<SEM_NGLL>;
  static std::atomic<unsigned long long> attr_done{0};
  static std::atomic<int> resident[64];  // CTAs per SM, per device
  if (int r = raise_smem_limit(attr_done, group_sweep_kernel<SEM_NGLL, LO>, C::SMEM)) return r;
  int dev = 0;
  cudaGetDevice(&dev);
  int per_sm = resident[dev & 63].load();
  if (per_sm <= 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, group_sweep_kernel<SEM_NGLL, LO>, C::T,
                                                                  C::SMEM);
    if (e != cudaSuccess) return static_cast<int>(e);
    per_sm = per_sm < 1 ? 1 : per_sm;
    resident[dev & 63].store(per_sm);
  }
  int sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return static_cast<int>(e);
  cudaLaunchConfig_t cfg = {};
  // all CTAs resident at once (a CTA may wait for items other CTAs hold), and no more than
  // there are items
  const int grid = std::min(sms * per_sm, std::max(1, L.nitems));
  cfg.gridDim = dim3(static_cast<unsigned>(grid));
  cfg.blockDim = dim3(C::T);
  cfg.dynamicSmemBytes = C::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return static_cast<int>(cudaLaunchKernelEx(&cfg, group_sweep_kernel<SEM_NGLL, LO>, L));
}

int launch_patch_n(const PatchLaunch& L, cudaStream_t s) {
  if (L.sync ? L.npatch <= 0 : L.p1 <= L.p0) return 0;
  using C = ForceCfg<SEM_NGLL>;
  const bool lo = L.variant == 0 ? C::LINE_OWNERS : L.variant == 1;
  if (L.shots > 1 && L.pairs) return launch_patch_lo<true, true>(L, s);  // shot pairs: line owners
  return lo ? launch_patch_lo<true, false>(L, s) : launch_patch_lo<false, false>(L, s);
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
  float2 h2[N * N], hw2[N * N];
  for (int q = 0; q < N * N; ++q) {
    h2[q] = make_float2(hf[q], hf[q]);
    hw2[q] = make_float2(hwf[q], hwf[q]);
  }
  if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_h2, h2, sizeof(h2), 0, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_hw2, hw2, sizeof(hw2), 0, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return static_cast<int>(e);
}

int SEM_CAT(launch_forces_, SEM_NGLL)(const ForceLaunch& L, void* stream) {
  return launch_forces_n(L, static_cast<cudaStream_t>(stream));
}

int SEM_CAT(launch_sensitivity_, SEM_NGLL)(const float* rec, const int* perm, const float* lam, const float* u_lo,
                                          const float* u_mid, const float* u_hi, float* g_rho, float* g_kappa,
                                          float* g_mu, int nspec, double c_m, double c_k, void* stream,
                                          const DevCtl* idx) {
  using C = ForceCfg<SEM_NGLL>;
  static std::atomic<unsigned long long> attr_done{0};
  const int smem = C::SMEM_FLOATS * static_cast<int>(sizeof(float));
  if (int r = raise_smem_limit(attr_done, sensitivity_kernel<SEM_NGLL>, smem)) return r;
  const int grid = (nspec + C::EPC - 1) / C::EPC;
  sensitivity_kernel<SEM_NGLL><<<grid, C::T, smem, static_cast<cudaStream_t>(stream)>>>(
      rec, perm, lam, u_lo, u_mid, u_hi, g_rho, g_kappa, g_mu, nspec, c_m, c_k, idx);
  return static_cast<int>(cudaGetLastError());
}

int SEM_CAT(forces_smem_bytes_, SEM_NGLL)() { return ForceCfg<SEM_NGLL>::SMEM_FLOATS * 4; }

int SEM_CAT(launch_patch_forces_, SEM_NGLL)(const PatchLaunch& L, void* stream) {
  return launch_patch_n(L, static_cast<cudaStream_t>(stream));
}

int SEM_CAT(launch_group_sweep_, SEM_NGLL)(const GroupLaunch& L, void* stream) {
  if (L.nitems <= 0) return 0;
  using C = ForceCfg<SEM_NGLL>;
  const bool lo = L.variant == 0 ? C::LINE_OWNERS : L.variant == 1;
  return lo ? launch_group_lo<true>(L, static_cast<cudaStream_t>(stream))
            : launch_group_lo<false>(L, static_cast<cudaStream_t>(stream));
}

void SEM_CAT(patch_layout_, SEM_NGLL)(int* es, int* ts, int* e) {
  using C = PatchCfg<SEM_NGLL>;
  *es = C::ES;
  *ts = C::TS;
  *e = C::E;
}

void SEM_CAT(patch_shape_, SEM_NGLL)(PatchShape* out) {
  using C = PatchCfg<SEM_NGLL>;
  out->bx = C::BX;
  out->by = C::BY;
  out->bz = C::BZ;
}

}  // namespace semgb
