// CUDA kernels of libsemgb (sm_103a) other than the force kernel (sem_forces.cuh): order
// dispatch, the Newmark corrector pass, sources/receivers, energy partials.
#include <cuda_runtime.h>

#include <cmath>

#include "sem_internal.h"

namespace semgb {

// ---------------------------------------------------------------------------------------
// Dispatch to the per-order translation units (sem_forces_<N>.cu).
// ---------------------------------------------------------------------------------------
#define SEM_DECLARE_ORDER(n)                                                        \
  int upload_basis_##n(const double* w, const double* h, void* stream, int ngll); \
  int launch_forces_##n(const ForceLaunch& L, void* stream);                      \
  int forces_smem_bytes_##n();
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

int launch_forces(int n, const ForceLaunch& L, void* stream) {
#define SEM_CALL(k) launch_forces_##k(L, stream)
  SEM_ORDER_SWITCH(n, SEM_CALL)
#undef SEM_CALL
  return static_cast<int>(cudaErrorInvalidValue);
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
// Fields are [nglob_pad][3] float32 with nglob_pad % 4 == 0: a thread owns four nodes,
// i.e. three float4 of each field and one float4 of the inverse mass.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float4 mass_lanes(const float4 m, int part) {
  // the three float4 words of 4 nodes (x0 y0 z0 x1 | y1 z1 x2 y2 | z2 x3 y3 z3)
  return part == 0 ? make_float4(m.x, m.x, m.x, m.y)
                   : (part == 1 ? make_float4(m.y, m.y, m.z, m.z) : make_float4(m.z, m.w, m.w, m.w));
}

// Predictor from a complete state (first step): u += dt v + dt^2/2 a ; v += dt/2 a.
// All loads of a thread are issued before its arithmetic so that each thread keeps nine
// 16-byte requests in flight.
__global__ void predictor_kernel(float4* __restrict__ u, float4* __restrict__ v, const float4* __restrict__ a,
                                 int n4, float dt, float hdt, float hdt2) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += gridDim.x * blockDim.x) {
    float4 av[3], vv[3], uv[3];
#pragma unroll
    for (int part = 0; part < 3; ++part) {
      av[part] = a[3 * t + part];
      vv[part] = v[3 * t + part];
      uv[part] = u[3 * t + part];
    }
#pragma unroll
    for (int part = 0; part < 3; ++part) {
      uv[part].x += dt * vv[part].x + hdt2 * av[part].x;
      uv[part].y += dt * vv[part].y + hdt2 * av[part].y;
      uv[part].z += dt * vv[part].z + hdt2 * av[part].z;
      uv[part].w += dt * vv[part].w + hdt2 * av[part].w;
      vv[part].x += hdt * av[part].x;
      vv[part].y += hdt * av[part].y;
      vv[part].z += hdt * av[part].z;
      vv[part].w += hdt * av[part].w;
      u[3 * t + part] = uv[part];
      v[3 * t + part] = vv[part];
    }
  }
}

// Corrector of step n-1 fused with the predictor of step n:
//   a = M^-1 a_raw ; v = v_half + dt/2 a ; u += dt v + dt^2/2 a ; v_half = v + dt/2 a
// a_raw stays in place: the next force sweep overwrites it at each node's first touch.
__global__ void fused_newmark_kernel(float4* __restrict__ u, float4* __restrict__ v,
                                     const float4* __restrict__ a, const float4* __restrict__ minv, int n4,
                                     float dt, float hdt, float hdt2) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += gridDim.x * blockDim.x) {
    const float4 m = minv[t];
    float4 ar[3], vv[3], uv[3];
#pragma unroll
    for (int part = 0; part < 3; ++part) {
      ar[part] = a[3 * t + part];
      vv[part] = v[3 * t + part];
      uv[part] = u[3 * t + part];
    }
#pragma unroll
    for (int part = 0; part < 3; ++part) {
      const float4 mm = mass_lanes(m, part);
      const float ax = ar[part].x * mm.x, ay = ar[part].y * mm.y, az = ar[part].z * mm.z, aw = ar[part].w * mm.w;
      float4 w = vv[part];
      w.x += hdt * ax;
      w.y += hdt * ay;
      w.z += hdt * az;
      w.w += hdt * aw;
      float4 x = uv[part];
      x.x += dt * w.x + hdt2 * ax;
      x.y += dt * w.y + hdt2 * ay;
      x.z += dt * w.z + hdt2 * az;
      x.w += dt * w.w + hdt2 * aw;
      w.x += hdt * ax;
      w.y += hdt * ay;
      w.z += hdt * az;
      w.w += hdt * aw;
      u[3 * t + part] = x;
      v[3 * t + part] = w;
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
// Divergence watchdog: flags any non-finite value of u, v or a (the fields hold 3*nglob_pad
// floats). Threads that find one write 1 into the flag word; the host clears it first.
// ---------------------------------------------------------------------------------------
__global__ void nonfinite_kernel(const float4* __restrict__ u, const float4* __restrict__ v,
                                 const float4* __restrict__ a, int n4x3, int* flag) {
  bool bad = false;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n4x3; t += gridDim.x * blockDim.x) {
    const float4 x = u[t], y = v[t], z = a[t];
    bad |= !(isfinite(x.x) && isfinite(x.y) && isfinite(x.z) && isfinite(x.w));
    bad |= !(isfinite(y.x) && isfinite(y.y) && isfinite(y.z) && isfinite(y.w));
    bad |= !(isfinite(z.x) && isfinite(z.y) && isfinite(z.z) && isfinite(z.w));
  }
  if (bad) *flag = 1;
}

int launch_nonfinite_check(const DevProblem& p, int* flag, void* stream) {
  const int n = 3 * (p.nglob_pad / 4);
  nonfinite_kernel<<<kEnergyBlocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<const float4*>(p.u), reinterpret_cast<const float4*>(p.v),
      reinterpret_cast<const float4*>(p.a), n, flag);
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
