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
__device__ __forceinline__ void wait_prerequisite_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_dependent_grid() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Barrier of one team: the warp, a named barrier (1 + team) over the team's two warps, or
// the CTA.
template <int KIND>
__device__ __forceinline__ void team_sync(int team) {
  if constexpr (KIND == 0) {
    __syncwarp();
  } else if constexpr (KIND == 1) {
    asm volatile("bar.sync %0, 64;" ::"r"(1 + team) : "memory");
  } else {
    __syncthreads();
  }
}

// VS: floats per node in u and f (4 for the context's own padded fields, 3 for caller arrays).
// With S shots (VS = 4 only) the fields are [nglob][S][4] and the launch works on the items
// (element, shot) of elements e0 .. e1-1, element-major: the teams of a CTA take the shots
// of one element, so its record is read from DRAM once for all of them.
template <int N, int VS, bool MS, bool LO>
__global__ void __launch_bounds__(ForceCfg<N>::T, ForceCfg<N>::MIN_BLOCKS)
    forces_kernel(const float* __restrict__ rec, const float* __restrict__ u, float* __restrict__ f, int e0,
                  int e1, int S_arg) {
  const int S = MS ? S_arg : 1;  // shots (a compile-time 1 for the single-shot kernel)
  using C = ForceCfg<N>;
  constexpr int NP = C::NP, NL = C::NL, E = C::E, REC = C::REC, TEAM = C::TEAM, ES = C::ES;
  extern __shared__ float4 smem4[];
  const float* __restrict__ H = c_h;
  const float* __restrict__ HW = c_hw;
  const float* __restrict__ W = c_w;

  const int team = threadIdx.x / TEAM;
  const int tl = threadIdx.x - team * TEAM;
  const int ibase = (blockIdx.x * C::TEAMS + team) * E;  // first item of the team
  const int ne = min(E, (e1 - e0) * S - ibase);
  if (C::KIND != 2 && ne <= 0) return;  // a team without items (its barrier is its own)
  float* ts = reinterpret_cast<float*>(smem4) + team * C::TS;
  // element and shot of the team's slot le
  auto elem_of = [&](int le) { return e0 + (MS ? (ibase + le) / S : ibase + le); };
  auto shot_of = [&](int le) { return MS ? (ibase + le) % S : 0; };

  // 0. records to L2 while the previous grid finishes, then wait for its results
  if (tl < ne) prefetch_l2(rec + static_cast<size_t>(elem_of(tl)) * REC, REC * sizeof(float));
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
      const size_t g = w[r] & ~kFirstTouchBit;
      if (base + r * TEAM < ne * NP) {
        if (VS == 4) {
          const int le = (base + r * TEAM) / NP;
          const float4 v = __ldg(reinterpret_cast<const float4*>(u) + g * S + shot_of(le));
          q[r][0] = v.x;
          q[r][1] = v.y;
          q[r][2] = v.z;
        } else {
          q[r][0] = __ldg(u + 3 * g);
          q[r][1] = __ldg(u + 3 * g + 1);
          q[r][2] = __ldg(u + 3 * g + 2);
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
  team_sync<C::KIND>(team);

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
    const float* __restrict__ r = rec + static_cast<size_t>(elem_of(active ? le : 0)) * REC;

    // 2a. eta derivatives along the eta-line (i, k) = (a, b), zeta derivatives along the
    //     zeta-line (i, j) = (a, b)
    if (active) {
      float ve[3][N], vz[3][N];
#pragma unroll
      for (int l = 0; l < N; ++l)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          ve[c][l] = su[3 * (a + N * (l + N * b)) + c];
          vz[c][l] = su[3 * (a + N * (b + N * l)) + c];
        }
#pragma unroll
      for (int m = 0; m < N; ++m)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float de = 0.f, dz = 0.f;
#pragma unroll
          for (int l = 0; l < N; ++l) {
            de += H[m * N + l] * ve[c][l];
            dz += H[m * N + l] * vz[c][l];
          }
          se[3 * (a + N * (m + N * b)) + c] = de;
          sz[3 * (a + N * (b + N * m)) + c] = dz;
        }
    }
    team_sync<C::KIND>(team);

    // 2b. along the xi-line (j, k) = (a, b): xi derivatives in registers, Jacobian map, Hooke
    //     stress, fluxes; the xi-flux transposed product stays in registers, the eta and zeta
    //     fluxes replace the derivatives they were made from
    float fx[N], fy[N], fz[N];
    {
      float ux[N], uy[N], uz[N];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int p = i + N * line;
        ux[i] = su[3 * p];
        uy[i] = su[3 * p + 1];
        uz[i] = su[3 * p + 2];
        fx[i] = fy[i] = fz[i] = 0.f;
      }
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float dxi_x = 0.f, dxi_y = 0.f, dxi_z = 0.f;
#pragma unroll
        for (int l = 0; l < N; ++l) {
          const float h = H[i * N + l];
          dxi_x += h * ux[l];
          dxi_y += h * uy[l];
          dxi_z += h * uz[l];
        }
        const int p3 = 3 * (i + N * line);
        const float det_x = se[p3], det_y = se[p3 + 1], det_z = se[p3 + 2];
        const float dze_x = sz[p3], dze_y = sz[p3 + 1], dze_z = sz[p3 + 2];
        const int q = i * NL + line;
        float G[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) G[c] = active ? __ldg(r + (kG + c) * NP + q) : 0.f;
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
          fx[ip] += hw * txi_x;
          fy[ip] += hw * txi_y;
          fz[ip] += hw * txi_z;
        }
        if (active) {
          se[p3] = jac * (sxx * G[3] + sxy * G[4] + sxz * G[5]);
          se[p3 + 1] = jac * (sxy * G[3] + syy * G[4] + syz * G[5]);
          se[p3 + 2] = jac * (sxz * G[3] + syz * G[4] + szz * G[5]);
          sz[p3] = jac * (sxx * G[6] + sxy * G[7] + sxz * G[8]);
          sz[p3 + 1] = jac * (sxy * G[6] + syy * G[7] + syz * G[8]);
          sz[p3 + 2] = jac * (sxz * G[6] + syz * G[7] + szz * G[8]);
        }
      }
    }
    team_sync<C::KIND>(team);

    // 3. eta and zeta transposed products along the eta- and zeta-lines, in place
    if (active) {
      float ve[3][N], vz[3][N];
#pragma unroll
      for (int l = 0; l < N; ++l)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          ve[c][l] = se[3 * (a + N * (l + N * b)) + c];
          vz[c][l] = sz[3 * (a + N * (b + N * l)) + c];
        }
#pragma unroll
      for (int m = 0; m < N; ++m)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float te = 0.f, tz = 0.f;
#pragma unroll
          for (int l = 0; l < N; ++l) {
            te += HW[l * N + m] * ve[c][l];
            tz += HW[l * N + m] * vz[c][l];
          }
          se[3 * (a + N * (m + N * b)) + c] = te;
          sz[3 * (a + N * (b + N * m)) + c] = tz;
        }
    }
    team_sync<C::KIND>(team);

    // 3b. element forces along the xi-line (j, k) = (a, b) into the (now free) u slots
    if (active) {
      const float wj = W[a], wk = W[b];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const float wi = W[i];
        const int p = 3 * (i + N * line);
        su[p] = -(wj * wk * fx[i] + wi * wk * se[p] + wi * wj * sz[p]);
        su[p + 1] = -(wj * wk * fy[i] + wi * wk * se[p + 1] + wi * wj * sz[p + 1]);
        su[p + 2] = -(wj * wk * fz[i] + wi * wk * se[p + 2] + wi * wj * sz[p + 2]);
      }
    }
    team_sync<C::KIND>(team);

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
    const float* __restrict__ r = rec + static_cast<size_t>(elem_of(active ? le : 0)) * REC;

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
        fx[ip] += hw * txi_x;
        fy[ip] += hw * txi_y;
        fz[ip] += hw * txi_z;
      }
      if (active) {
        const int p3 = 3 * (i + N * line);
        se[p3] = jac * (sxx * G[3] + sxy * G[4] + sxz * G[5]);
        se[p3 + 1] = jac * (sxy * G[3] + syy * G[4] + syz * G[5]);
        se[p3 + 2] = jac * (sxz * G[3] + syz * G[4] + szz * G[5]);
        sz[p3] = jac * (sxx * G[6] + sxy * G[7] + sxz * G[8]);
        sz[p3 + 1] = jac * (sxy * G[6] + syy * G[7] + syz * G[8]);
        sz[p3 + 2] = jac * (sxz * G[6] + syz * G[7] + szz * G[8]);
      }
    }
    team_sync<C::KIND>(team);

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
    team_sync<C::KIND>(team);

  }

  // 4. scatter in the gather's coalesced order; for the padded layout the previous values
  //    of a group of GB nodes are loaded before any of them is written back
  if constexpr (VS == 4) {
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
            prev[r] = reinterpret_cast<const float4*>(f)[static_cast<size_t>(w[r] & ~kFirstTouchBit) * S + shot_of(e)];
        }
      }
#pragma unroll
      for (int r = 0; r < GB; ++r) {
        const int idx = base + r * TEAM;
        if (idx < ne * NP) {
          const int e = idx / NP;
          const float* src = ts + e * ES + 3 * (idx - e * NP);
          reinterpret_cast<float4*>(f)[static_cast<size_t>(w[r] & ~kFirstTouchBit) * S + shot_of(e)] =
              make_float4(src[0] + prev[r].x, src[1] + prev[r].y, src[2] + prev[r].z, 0.f);
        }
      }
    }
  } else {
    for (int idx = tl; idx < ne * NP; idx += TEAM) {
      const int e = idx / NP;
      const int p = idx - e * NP;
      const float* sb = ts + e * ES;
      const uint32_t w = reinterpret_cast<const uint32_t*>(sb + 9 * NP)[p];
      const size_t g = w & ~kFirstTouchBit;
      const float* src = sb + 3 * p;
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
  }
}

// ---------------------------------------------------------------------------------------
// Material sensitivities (the discrete adjoint of the explicit scheme): at one adjoint step,
// for every local point q of every element
//   g_rho[q]   += c_m * w_q J_q lam_I . (u_hi - 2 u_mid + u_lo)_I          (I = ibool(q))
//   g_kappa[q] += c_k * w_q J_q tr e(lam) tr e(u_mid)
//   g_mu[q]    += c_k * w_q J_q 2 (e(lam) : e(u_mid) - tr e(lam) tr e(u_mid) / 3)
// with e the discrete strain (the same derivatives and chain rule as the force kernel),
// c_m = -1 and c_k = -dt^2. lam is the adjoint field in the solver layout [nglob][4], the
// u_* displacement snapshots [nglob][3]. The terms are formed in float32 (the second
// difference as (u_hi - u_mid) - (u_mid - u_lo), which keeps the digits the plain form
// cancels) and added to float64 accumulators per local point in record order (element,
// q = i N^2 + line). No two threads write the same point, so there are no colours here.
// ---------------------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(ForceCfg<N>::T)
    sensitivity_kernel(const float* __restrict__ rec, const float* __restrict__ lam, const float* __restrict__ u_lo,
                       const float* __restrict__ u_mid, const float* __restrict__ u_hi, double* __restrict__ g_rho,
                       double* __restrict__ g_kappa, double* __restrict__ g_mu, int nspec, double c_m, double c_k) {
  using C = ForceCfg<N>;
  constexpr int NP = C::NP, NL = C::NL, E = C::E, REC = C::REC, TEAM = C::TEAM, ES = C::ES;
  static_assert(7 * NP <= ES, "element tile holds lam, u and the mass term");
  extern __shared__ float4 smem4[];
  const float* __restrict__ H = c_h;
  const float* __restrict__ W = c_w;
  const int team = threadIdx.x / TEAM;
  const int tl = threadIdx.x - team * TEAM;
  const int ebase = (blockIdx.x * C::TEAMS + team) * E;
  const int ne = min(E, nspec - ebase);
  if (C::KIND != 2 && ne <= 0) return;
  float* ts = reinterpret_cast<float*>(smem4) + team * C::TS;
  constexpr int GB = 2;  // points per thread whose loads are in flight together
  for (int base = tl; base < ne * NP; base += GB * TEAM) {
    size_t g[GB];
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      const int idx = base + r * TEAM;
      const int le = idx / NP;
      g[r] = idx < ne * NP
                 ? __float_as_uint(__ldg(rec + static_cast<size_t>(ebase + le) * REC + (idx - le * NP))) & ~kFirstTouchBit
                 : 0;
    }
    float4 l4[GB];
    float um[GB][3], uh[GB][3], ul[GB][3];
#pragma unroll
    for (int r = 0; r < GB; ++r) {
      l4[r] = __ldg(reinterpret_cast<const float4*>(lam) + g[r]);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        um[r][a] = __ldg(u_mid + 3 * g[r] + a);
        uh[r][a] = __ldg(u_hi + 3 * g[r] + a);
        ul[r][a] = __ldg(u_lo + 3 * g[r] + a);
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
  team_sync<C::KIND>(team);
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
    g_rho[out + q] += c_m * static_cast<double>(wJ * fm[i + N * line]);
    g_kappa[out + q] += c_k * static_cast<double>(wJ * trl * tru);
    g_mu[out + q] += c_k * static_cast<double>(2.f * wJ * (ee - trl * tru * (1.f / 3.f)));
  }
}

template <int VS, bool MS, bool LO>
int launch_forces_vs(const ForceLaunch& L, cudaStream_t s) {
  using C = ForceCfg<SEM_NGLL>;
  static unsigned long long attr_done = 0;  // one bit per device ordinal
  const int smem = C::SMEM_FLOATS * static_cast<int>(sizeof(float));
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(attr_done & bit)) {
    cudaError_t e =
        cudaFuncSetAttribute(forces_kernel<SEM_NGLL, VS, MS, LO>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return static_cast<int>(e);
    attr_done |= bit;
  }
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
  return static_cast<int>(cudaLaunchKernelEx(&cfg, forces_kernel<SEM_NGLL, VS, MS, LO>, L.rec, L.u, L.f, L.e0, L.e1, S));
}

int launch_forces_n(const ForceLaunch& L, cudaStream_t s) {
  if (L.e1 <= L.e0) return 0;
  using C = ForceCfg<SEM_NGLL>;
  const bool lo = L.variant == 0 ? C::LINE_OWNERS : L.variant == 1;  // 0 default, 1 line owners, 2 per point
  if (L.shots > 1) {
    if (L.node_stride != 4) return static_cast<int>(cudaErrorInvalidValue);
    return lo ? launch_forces_vs<4, true, true>(L, s) : launch_forces_vs<4, true, false>(L, s);
  }
  if (L.node_stride == 4) return lo ? launch_forces_vs<4, false, true>(L, s) : launch_forces_vs<4, false, false>(L, s);
  if (L.node_stride == 3) return launch_forces_vs<3, false, C::LINE_OWNERS>(L, s);
  return static_cast<int>(cudaErrorInvalidValue);
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
  return launch_forces_n(L, static_cast<cudaStream_t>(stream));
}

int SEM_CAT(launch_sensitivity_, SEM_NGLL)(const float* rec, const float* lam, const float* u_lo, const float* u_mid,
                                          const float* u_hi, double* g_rho, double* g_kappa, double* g_mu, int nspec,
                                          double c_m, double c_k, void* stream) {
  using C = ForceCfg<SEM_NGLL>;
  static unsigned long long attr_done = 0;
  const int smem = C::SMEM_FLOATS * static_cast<int>(sizeof(float));
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(attr_done & bit)) {
    cudaError_t e =
        cudaFuncSetAttribute(sensitivity_kernel<SEM_NGLL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return static_cast<int>(e);
    attr_done |= bit;
  }
  const int grid = (nspec + C::EPC - 1) / C::EPC;
  sensitivity_kernel<SEM_NGLL><<<grid, C::T, smem, static_cast<cudaStream_t>(stream)>>>(
      rec, lam, u_lo, u_mid, u_hi, g_rho, g_kappa, g_mu, nspec, c_m, c_k);
  return static_cast<int>(cudaGetLastError());
}

int SEM_CAT(forces_smem_bytes_, SEM_NGLL)() { return ForceCfg<SEM_NGLL>::SMEM_FLOATS * 4; }

}  // namespace semgb
