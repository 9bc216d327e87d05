// CUDA kernels of libsemgb (sm_103a) other than the force kernel (sem_forces.cuh): order
// dispatch, the Newmark corrector pass, sources/receivers, energy partials.
#include <cuda_runtime.h>

#include <cmath>

#include "sem_internal.h"

namespace semgb {

// ---------------------------------------------------------------------------------------
// Dispatch to the per-order translation units (sem_forces_<N>.cu).
// ---------------------------------------------------------------------------------------
#define SEM_DECLARE_ORDER(n)                                                                                \
  int upload_basis_##n(const double* w, const double* h, void* stream, int ngll);                         \
  int launch_forces_##n(const ForceLaunch& L, void* stream);                                              \
  int forces_smem_bytes_##n();                                                                            \
  int launch_patch_forces_##n(const PatchLaunch& L, void* stream);                                        \
  int launch_group_sweep_##n(const GroupLaunch& L, void* stream);                                         \
  void patch_shape_##n(PatchShape* out);                                                                  \
  void patch_layout_##n(int* es, int* ts, int* e);                                                        \
  int launch_sensitivity_##n(const float* rec, const int* perm, const float* lam, const float* u_lo,       \
                             const float* u_mid, const float* u_hi, float* g_rho, float* g_kappa,       \
                             float* g_mu, int nspec, double c_m, double c_k, void* stream,              \
                             const DevCtl* idx);
SEM_DECLARE_ORDER(2)
SEM_DECLARE_ORDER(3)
SEM_DECLARE_ORDER(4)
SEM_DECLARE_ORDER(5)
SEM_DECLARE_ORDER(6)
SEM_DECLARE_ORDER(7)
SEM_DECLARE_ORDER(8)
SEM_DECLARE_ORDER(9)
SEM_DECLARE_ORDER(10)

#define SEM_ORDER_SWITCH(n, call) \
  switch (n) {                    \
    case 2: return call(2);       \
    case 3: return call(3);       \
    case 4: return call(4);       \
    case 5: return call(5);       \
    case 6: return call(6);       \
    case 7: return call(7);       \
    case 8: return call(8);       \
    case 9: return call(9);       \
    case 10: return call(10);     \
    default: break;               \
  }

int upload_basis(int n, const double* w, const double* h, void* stream) {
#define SEM_CALL(k) upload_basis_##k(w, h, stream, n)
  SEM_ORDER_SWITCH(n, SEM_CALL)
#undef SEM_CALL
  return static_cast<int>(cudaErrorInvalidValue);
}

int launch_group_sweep(int n, const GroupLaunch& L, void* stream) {
#define SEM_CALL(k) launch_group_sweep_##k(L, stream)
  SEM_ORDER_SWITCH(n, SEM_CALL)
#undef SEM_CALL
  return static_cast<int>(cudaErrorInvalidValue);
}

int launch_forces(int n, const ForceLaunch& L, void* stream) {
#define SEM_CALL(k) launch_forces_##k(L, stream)
  SEM_ORDER_SWITCH(n, SEM_CALL)
#undef SEM_CALL
  return static_cast<int>(cudaErrorInvalidValue);
}

int launch_sensitivity(int n, const float* rec, const int* perm, const float* lam, const float* u_lo,
                       const float* u_mid, const float* u_hi, float* g_rho, float* g_kappa, float* g_mu, int nspec,
                       double c_m, double c_k, void* stream, const DevCtl* idx) {
#define SEM_CALL(k) \
  launch_sensitivity_##k(rec, perm, lam, u_lo, u_mid, u_hi, g_rho, g_kappa, g_mu, nspec, c_m, c_k, stream, idx)
  SEM_ORDER_SWITCH(n, SEM_CALL)
#undef SEM_CALL
  return static_cast<int>(cudaErrorInvalidValue);
}

int launch_patch_forces(int n, const PatchLaunch& L, void* stream) {
#define SEM_CALL(k) launch_patch_forces_##k(L, stream)
  SEM_ORDER_SWITCH(n, SEM_CALL)
#undef SEM_CALL
  return static_cast<int>(cudaErrorInvalidValue);
}

int patch_shape(int n, PatchShape* out) {
#define SEM_CALL(k) (patch_shape_##k(out), 0)
  SEM_ORDER_SWITCH(n, SEM_CALL)
#undef SEM_CALL
  return -1;
}

int patch_layout(int n, int* es, int* ts, int* e) {
#define SEM_CALL(k) (patch_layout_##k(es, ts, e), 0)
  SEM_ORDER_SWITCH(n, SEM_CALL)
#undef SEM_CALL
  return -1;
}

int forces_kernel_smem_bytes(int n) {
#define SEM_CALL(k) forces_smem_bytes_##k()
  SEM_ORDER_SWITCH(n, SEM_CALL)
#undef SEM_CALL
  return 0;
}

int forces_elements_per_cta(int n) {
  if (n < 2 || n > 10) return 0;
  return n * n <= 32 ? 4 * (32 / (n * n)) : 256 / (n * n);
}

// ---------------------------------------------------------------------------------------
// Newmark streaming passes (Sec. I / V-C explicit second-order Newmark, diagonal mass).
// Fields are [nglob][shots][kNodeStride] float32: one thread per (node, shot) reads one
// float4 of each field (the 4th lane stays zero) and the node's inverse mass.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float4 axpy3(float4 y, float s, float4 x) {
  return make_float4(y.x + s * x.x, y.y + s * x.y, y.z + s * x.z, 0.f);
}

// Predictor from a complete state (first step): u += dt v + dt^2/2 a ; v += dt/2 a.
__global__ void predictor_kernel(float4* __restrict__ u, float4* __restrict__ v, const float4* __restrict__ a,
                                 long long n, float dt, float hdt, float hdt2) {
  for (long long g = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; g < n;
       g += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float4 ag = a[g], vg = v[g], ug = u[g];
    u[g] = axpy3(axpy3(ug, dt, vg), hdt2, ag);
    v[g] = axpy3(vg, hdt, ag);
  }
}

// Corrector of step n-1 fused with the predictor of step n:
//   a = M^-1 a_raw ; v = v_half + dt/2 a ; u += dt v + dt^2/2 a ; v_half = v + dt/2 a
// a_raw stays in place: the next force sweep overwrites it at each node's first touch.
__global__ void fused_newmark_kernel(float4* __restrict__ u, float4* __restrict__ v,
                                     const float4* __restrict__ a, const float* __restrict__ minv, long long n,
                                     int shots, float dt, float hdt, float hdt2) {
  for (long long g = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; g < n;
       g += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float m = minv[g / shots];
    const float4 ar = a[g], vh = v[g], ug = u[g];
    const float4 acc = make_float4(ar.x * m, ar.y * m, ar.z * m, 0.f);
    const float4 vf = axpy3(vh, hdt, acc);
    u[g] = axpy3(axpy3(ug, dt, vf), hdt2, acc);
    v[g] = axpy3(vf, hdt, acc);
  }
}

// Corrector alone (completes the state): a = M^-1 a_raw ; v = v_half + dt/2 a
__global__ void corrector_kernel(float4* __restrict__ v, float4* __restrict__ a, const float* __restrict__ minv,
                                 long long n, int shots, float hdt) {
  for (long long g = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; g < n;
       g += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float m = minv[g / shots];
    const float4 ar = a[g];
    const float4 acc = make_float4(ar.x * m, ar.y * m, ar.z * m, 0.f);
    a[g] = acc;
    v[g] = axpy3(v[g], hdt, acc);
  }
}

static int stream_grid(long long n) {
  const long long g = (n + 255) / 256;
  return g < 1 ? 1 : static_cast<int>(g < (1ll << 30) ? g : (1ll << 30));
}

int launch_predictor(const DevProblem& p, void* stream) {
  const long long n = static_cast<long long>(p.nglob) * p.shots;
  predictor_kernel<<<stream_grid(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<float4*>(p.u), reinterpret_cast<float4*>(p.v), reinterpret_cast<const float4*>(p.a), n,
      static_cast<float>(p.dt), static_cast<float>(0.5 * p.dt), static_cast<float>(0.5 * p.dt * p.dt));
  return static_cast<int>(cudaGetLastError());
}

int launch_fused_newmark(const DevProblem& p, void* stream) {
  const long long n = static_cast<long long>(p.nglob) * p.shots;
  fused_newmark_kernel<<<stream_grid(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<float4*>(p.u), reinterpret_cast<float4*>(p.v), reinterpret_cast<const float4*>(p.a), p.minv,
      n, p.shots, static_cast<float>(p.dt), static_cast<float>(0.5 * p.dt), static_cast<float>(0.5 * p.dt * p.dt));
  return static_cast<int>(cudaGetLastError());
}

int launch_corrector(const DevProblem& p, void* stream) {
  const long long n = static_cast<long long>(p.nglob) * p.shots;
  corrector_kernel<<<stream_grid(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<float4*>(p.v), reinterpret_cast<float4*>(p.a), p.minv, n, p.shots,
      static_cast<float>(0.5 * p.dt));
  return static_cast<int>(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------
// Adjoint leapfrog (the discrete adjoint of the scheme above, run backward in time):
//   lam_new = 2 lam - lam_old + dt^2 M^-1 F,  F = -K lam + R^T G / dt^2
// written over lam_old. Receiver residuals are added to F by one thread per receiver node,
// its receivers in ascending order (receivers may share a node).
// ---------------------------------------------------------------------------------------
__global__ void adjoint_inject_kernel(float* __restrict__ F, const float* __restrict__ G,
                                      const int* __restrict__ rnode, const int* __restrict__ roff,
                                      const int* __restrict__ rlist, int nnodes, float inv_dt2,
                                      const DevCtl* __restrict__ idx) {
  if (idx) G = idx->adj_G + static_cast<long long>(idx->adj_j - 1) * idx->adj_gstep;
  // one thread per distinct receiver node; its receivers in ascending order (the order a
  // single thread walking the receivers would add them in)
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nnodes; t += gridDim.x * blockDim.x) {
    float* Fn = F + kNodeStride * static_cast<size_t>(rnode[t]);
    for (int q = roff[t]; q < roff[t + 1]; ++q) {
      const int r = rlist[q];
      for (int c = 0; c < 3; ++c) Fn[c] += G[3 * r + c] * inv_dt2;
    }
  }
}

__global__ void adjoint_leapfrog_kernel(const float4* __restrict__ lam, float4* __restrict__ lam_old,
                                        const float4* __restrict__ F, const float* __restrict__ minv, int nglob,
                                        float dt2) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < nglob; g += gridDim.x * blockDim.x) {
    const float s = dt2 * minv[g];
    const float4 l = lam[g], o = lam_old[g], f = F[g];
    lam_old[g] = make_float4(2.f * l.x - o.x + s * f.x, 2.f * l.y - o.y + s * f.y, 2.f * l.z - o.z + s * f.z, 0.f);
  }
}

__global__ void adjoint_index_kernel(DevCtl* ctl, const float* G, const float* u, long long n3, int gstep, int j) {
  ctl->adj_G = G;
  ctl->adj_u = u;
  ctl->adj_n3 = n3;
  ctl->adj_gstep = gstep;
  ctl->adj_j = j;
  ctl->adj_js = j;
}

__global__ void adjoint_next_kernel(DevCtl* ctl, int sensitivity) {
  if (sensitivity)
    ctl->adj_js -= 1;
  else
    ctl->adj_j -= 1;
}

int launch_adjoint_index(DevCtl* ctl, const float* G, const float* u, long long n3, int gstep, int j, void* stream) {
  adjoint_index_kernel<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(ctl, G, u, n3, gstep, j);
  return static_cast<int>(cudaGetLastError());
}

int launch_adjoint_next(DevCtl* ctl, void* stream, bool sensitivity) {
  adjoint_next_kernel<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(ctl, sensitivity ? 1 : 0);
  return static_cast<int>(cudaGetLastError());
}

__global__ void flush_partials_kernel(float* __restrict__ part, double* __restrict__ acc, long long n) {
  for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < n;
       t += static_cast<long long>(gridDim.x) * blockDim.x) {
    acc[t] += static_cast<double>(part[t]);
    part[t] = 0.f;
  }
}

int launch_flush_partials(float* part, double* acc, long long n, void* stream) {
  if (n <= 0) return 0;
  flush_partials_kernel<<<stream_grid(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(part, acc, n);
  return static_cast<int>(cudaGetLastError());
}

int launch_adjoint_update(float* F, const float* G_dev, const int* rnode, const int* roff, const int* rlist,
                          int nnodes, const float* lam, float* lam_old, const float* minv, int nglob, double dt,
                          void* stream, const DevCtl* idx) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (G_dev && nnodes > 0) {
    adjoint_inject_kernel<<<(nnodes + 127) / 128, 128, 0, s>>>(F, G_dev, rnode, roff, rlist, nnodes,
                                                             static_cast<float>(1.0 / (dt * dt)), idx);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return static_cast<int>(e);
  }
  adjoint_leapfrog_kernel<<<stream_grid(nglob), 256, 0, s>>>(
      reinterpret_cast<const float4*>(lam), reinterpret_cast<float4*>(lam_old), reinterpret_cast<const float4*>(F),
      minv, nglob, static_cast<float>(dt * dt));
  return static_cast<int>(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------
// Material (Sec. II-B: isotropic moduli; Sec. I: the diagonal mass M_I = sum rho J w w w
// over the local points that share node I). One thread per local point of a record slot.
// ---------------------------------------------------------------------------------------
__device__ inline void point_moduli(const MaterialLaunch& m, size_t q, double* rho, double* kappa, double* mu,
                                    double* vp) {
  const double rh = m.rho[q], a = m.p1[q], b = m.p2[q];
  *rho = rh;
  if (m.moduli) {
    *kappa = a;
    *mu = b;
    *vp = sqrt((a + 4.0 * b / 3.0) / rh);
  } else {
    *mu = rh * b * b;
    *kappa = rh * (a * a - 2.0 * b * b) + 2.0 * *mu / 3.0;
    *vp = a;
  }
}

__global__ void material_check_kernel(MaterialLaunch m, unsigned long long* first_bad) {
  const long long n = static_cast<long long>(m.nspec) * m.ngll * m.ngll * m.ngll;
  for (long long q = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; q < n;
       q += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float rh = m.rho[q], a = m.p1[q], b = m.p2[q];
    const bool finite = isfinite(rh) && isfinite(a) && isfinite(b);
    const bool ok = finite && (m.moduli ? (rh > 0.f && b >= 0.f && a > 0.f) : (rh > 0.f && b >= 0.f && a > b));
    if (!ok) atomicMin(first_bad, static_cast<unsigned long long>(q));
  }
}

__global__ void material_records_kernel(MaterialLaunch m) {
  const int n = m.ngll, np = n * n * n;
  const long long total = static_cast<long long>(m.nspec) * np;
  const size_t RW = (static_cast<size_t>(kRecFields) * np + 3) / 4 * 4;
  for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long s = t / np;
    const int p = static_cast<int>(t - s * np);
    const int i = p % n, j = (p / n) % n, k = p / (n * n);
    const size_t q = static_cast<size_t>(m.order[s]) * np + p;
    double rh, kappa, mu, vp;
    point_moduli(m, q, &rh, &kappa, &mu, &vp);
    float* r = m.rec + s * RW;
    const int qq = i * n * n + j + n * k;
    const double J = r[kJac * np + qq];
    r[kJKappa * np + qq] = static_cast<float>(J * kappa);
    r[kJMu * np + qq] = static_cast<float>(J * mu);
  }
}

__global__ void mass_color_kernel(MaterialLaunch m, int e0, int e1, double* mass) {
  const int n = m.ngll, np = n * n * n;
  const long long total = static_cast<long long>(e1 - e0) * np;
  const size_t RW = (static_cast<size_t>(kRecFields) * np + 3) / 4 * 4;
  for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long it = t / np;
    const long long s = m.elist[e0 + it];  // record slot
    const int p = static_cast<int>(t - it * np);
    const int i = p % n, j = (p / n) % n, k = p / (n * n);
    const float* r = m.rec + s * RW;
    const uint32_t g = __float_as_uint(r[kIbool * np + p]) & kNodeMask;
    const double J = r[kJac * np + i * n * n + j + n * k];
    const double rh = m.rho[static_cast<size_t>(m.order[s]) * np + p];
    mass[g] += rh * J * m.w[i] * m.w[j] * m.w[k];  // elements of one colour share no node
  }
}

__global__ void inverse_mass_kernel(const double* __restrict__ mass, float* __restrict__ minv, int nglob) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < nglob; g += gridDim.x * blockDim.x)
    minv[g] = static_cast<float>(1.0 / mass[g]);
}

__global__ void vpmax_kernel(MaterialLaunch m, double* vpmax) {
  const int np = m.ngll * m.ngll * m.ngll;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m.nspec; e += gridDim.x * blockDim.x) {
    double best = 0.0;
    for (int p = 0; p < np; ++p) {
      double rh, kappa, mu, vp;
      point_moduli(m, static_cast<size_t>(e) * np + p, &rh, &kappa, &mu, &vp);
      best = fmax(best, vp);
    }
    vpmax[e] = best;
  }
}

int launch_material_check(const MaterialLaunch& m, unsigned long long* first_bad, void* stream) {
  const long long n = static_cast<long long>(m.nspec) * m.ngll * m.ngll * m.ngll;
  material_check_kernel<<<stream_grid(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(m, first_bad);
  return static_cast<int>(cudaGetLastError());
}

int launch_material_apply(const MaterialLaunch& m, const int* sweep_off, int nranges, double* mass, float* minv,
                          double* vpmax, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int np = m.ngll * m.ngll * m.ngll;
  material_records_kernel<<<stream_grid(static_cast<long long>(m.nspec) * np), 256, 0, s>>>(m);
  cudaError_t e = cudaMemsetAsync(mass, 0, static_cast<size_t>(m.nglob) * sizeof(double), s);
  if (e != cudaSuccess) return static_cast<int>(e);
  for (int c = 0; c < nranges; ++c) {  // each range holds elements of one colour
    const int e0 = sweep_off[c], e1 = sweep_off[c + 1];
    if (e1 > e0) mass_color_kernel<<<stream_grid(static_cast<long long>(e1 - e0) * np), 256, 0, s>>>(m, e0, e1, mass);
  }
  inverse_mass_kernel<<<stream_grid(m.nglob), 256, 0, s>>>(mass, minv, m.nglob);
  vpmax_kernel<<<stream_grid(m.nspec), 256, 0, s>>>(m, vpmax);
  return static_cast<int>(cudaGetLastError());
}

// Layout changes between the solver's fields [nglob][shots][4] (internal node order) and the
// caller's arrays [shots][nglob][3] (caller node order through perm, or internal order when
// perm is null): state copies, displacement snapshots. One thread per (node, shot).
__global__ void pack_kernel(const float4* __restrict__ u, float* __restrict__ out, const int* __restrict__ perm,
                            long long nglob, int shots) {
  const long long n = nglob * shots;
  for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < n;
       t += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long g = shots == 1 ? t : t / shots;
    const long long sh = t - g * shots;
    const float4 v = u[t];
    float* o = out + 3 * (sh * nglob + (perm ? perm[g] : g));
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
  }
}

__global__ void unpack_kernel(const float* __restrict__ in, float4* __restrict__ u, const int* __restrict__ perm,
                              long long nglob, int shots) {
  const long long n = nglob * shots;
  for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < n;
       t += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long g = shots == 1 ? t : t / shots;
    const long long sh = t - g * shots;
    const float* i = in + 3 * (sh * nglob + (perm ? perm[g] : g));
    u[t] = make_float4(i[0], i[1], i[2], 0.f);
  }
}

int launch_pack(const float* u, float* out, const int* perm, int nglob, int shots, void* stream) {
  const long long n = static_cast<long long>(nglob) * shots;
  if (n == 0) return 0;
  pack_kernel<<<stream_grid(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(reinterpret_cast<const float4*>(u), out,
                                                                             perm, nglob, shots);
  return static_cast<int>(cudaGetLastError());
}

int launch_unpack(const float* in, float* u, const int* perm, int nglob, int shots, void* stream) {
  const long long n = static_cast<long long>(nglob) * shots;
  if (n == 0) return 0;
  unpack_kernel<<<stream_grid(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(in, reinterpret_cast<float4*>(u),
                                                                               perm, nglob, shots);
  return static_cast<int>(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------
// Sources and receivers (Sec. V-C): Ricker point forces added to a_raw at t_{n+1}, then the
// displacement u^{n+1} sampled at the receiver nodes; advances the device step counter.
// Source nodes are distinct (the host merges duplicates), so the adds do not race.
// ---------------------------------------------------------------------------------------
__global__ void sources_record_kernel(float* __restrict__ a, const float* __restrict__ u, DevCtl* ctl, int shots,
                                      int nsrc, const int* __restrict__ src_node, const int* __restrict__ src_shot,
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
    const size_t g = kNodeStride * (static_cast<size_t>(src_node[s]) * shots + src_shot[s]);
    a[g] += static_cast<float>(src_force[3 * s] * R);
    a[g + 1] += static_cast<float>(src_force[3 * s + 1] * R);
    a[g + 2] += static_cast<float>(src_force[3 * s + 2] * R);
  }
  if (seis != nullptr && col < ncols) {  // seis [shots][nrec][3][ncols]
    for (int q = threadIdx.x; q < 3 * nrec * shots; q += blockDim.x) {
      const int sh = q / (3 * nrec);
      const int rq = q - sh * 3 * nrec;
      const int r = rq / 3, c = rq - 3 * r;
      seis[static_cast<size_t>(q) * ncols + col] =
          u[kNodeStride * (static_cast<size_t>(rec_node[r]) * shots + sh) + c];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl->step = n + 1;
    ctl->col = col + 1;
  }
}

// pack_kernel into the snapshot slot the step counter names (graph-replayable)
__global__ void snapshot_kernel(const float4* __restrict__ u, const DevCtl* __restrict__ ctl,
                                const int* __restrict__ perm, long long nglob, int shots) {
  float* base = ctl->snap;
  if (!base) return;
  float* out = base + static_cast<long long>(ctl->col - 1) * ctl->snap_per;
  const long long n = nglob * shots;
  for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < n;
       t += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long g = shots == 1 ? t : t / shots;
    const long long sh = t - g * shots;
    const float4 v = u[t];
    float* o = out + 3 * (sh * nglob + (perm ? perm[g] : g));
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
  }
}

int launch_snapshot(const float* u, DevCtl* ctl, const int* perm, int nglob, int shots, void* stream) {
  const long long n = static_cast<long long>(nglob) * shots;
  if (n == 0) return 0;
  snapshot_kernel<<<stream_grid(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(reinterpret_cast<const float4*>(u),
                                                                                 ctl, perm, nglob, shots);
  return static_cast<int>(cudaGetLastError());
}

__global__ void set_ctl_kernel(DevCtl* ctl, long long step, int ncols, float* seis, float* snap, long long snap_per) {
  ctl->step = step;
  ctl->col = 0;
  ctl->ncols = ncols;
  ctl->seis = seis;
  ctl->err = 0;
  ctl->snap = snap;
  ctl->snap_per = snap_per;
}

int launch_set_ctl(DevCtl* ctl, long long step, int ncols, float* seis, void* stream, float* snap,
                   long long snap_per) {
  set_ctl_kernel<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(ctl, step, ncols, seis, snap, snap_per);
  return static_cast<int>(cudaGetLastError());
}

int launch_sources_record(const DevProblem& p, void* stream) {
  sources_record_kernel<<<1, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      p.a, p.u, p.ctl, p.shots, p.nsrc, p.src_node, p.src_shot, p.src_force, p.f0, p.t0, p.dt, p.nrec, p.rec_node);
  return static_cast<int>(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------
// Divergence watchdog: flags any non-finite value of u, v or a ([nglob][kNodeStride]).
// Threads that find one write 1 into the flag word; the host clears it first.
// ---------------------------------------------------------------------------------------
__global__ void nonfinite_kernel(const float4* __restrict__ u, const float4* __restrict__ v,
                                 const float4* __restrict__ a, int nglob, int* flag) {
  bool bad = false;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nglob; t += gridDim.x * blockDim.x) {
    const float4 x = u[t], y = v[t], z = a[t];
    bad |= !(isfinite(x.x) && isfinite(x.y) && isfinite(x.z) && isfinite(x.w));
    bad |= !(isfinite(y.x) && isfinite(y.y) && isfinite(y.z) && isfinite(y.w));
    bad |= !(isfinite(z.x) && isfinite(z.y) && isfinite(z.z) && isfinite(z.w));
  }
  if (bad) *flag = 1;
}

int launch_nonfinite_check(const DevProblem& p, int* flag, void* stream) {
  const int n = p.nglob * p.shots;
  nonfinite_kernel<<<kEnergyBlocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<const float4*>(p.u), reinterpret_cast<const float4*>(p.v),
      reinterpret_cast<const float4*>(p.a), n, flag);
  return static_cast<int>(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------
// Energy partial sums: per block, sum_I |v_I|^2 / minv_I and sum_I u_I . f_I in float64.
// ---------------------------------------------------------------------------------------
__global__ void energy_partials_kernel(const float4* __restrict__ u, const float4* __restrict__ v,
                                       const float4* __restrict__ f, const float* __restrict__ minv, int nglob,
                                       int shots, double* __restrict__ partials) {
  __shared__ double sk[256], sp[256];
  double kin = 0.0, pot = 0.0;
  const long long n = static_cast<long long>(nglob) * shots;
  for (long long g = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; g < n;
       g += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float m = minv[g / shots];
    const float4 vg = v[g], ug = u[g], fg = f[g];
    const double vx = vg.x, vy = vg.y, vz = vg.z;
    kin += (vx * vx + vy * vy + vz * vz) / static_cast<double>(m);
    pot += static_cast<double>(ug.x) * fg.x + static_cast<double>(ug.y) * fg.y + static_cast<double>(ug.z) * fg.z;
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

int launch_energy_partials(const float* u, const float* v, const float* f, const float* minv, int nglob,
                           int shots, double* partials, int nblocks, void* stream) {
  energy_partials_kernel<<<nblocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<const float4*>(u), reinterpret_cast<const float4*>(v), reinterpret_cast<const float4*>(f),
      minv, nglob, shots, partials);
  return static_cast<int>(cudaGetLastError());
}

}  // namespace semgb
