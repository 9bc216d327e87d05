// sem_energy_noalloc: the energy sums of sem_energy for callers that cannot allocate
// device memory. The per-block partial sums live in a fixed file-scope device array
// instead of memory from cudaMalloc; the caller passes u, v and f = -K u.
#include <cuda_runtime.h>

#include <string>

#include "sem.h"
#include "sem_internal.h"

namespace semgb {
namespace {

constexpr int kNoAllocSlots = 4096;                 // partial-sum pairs in the scratch array
constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocNodesPerThread = 64;
constexpr int kNoAllocNodesPerBlock = kNoAllocThreads * kNoAllocNodesPerThread;
constexpr long long kNoAllocMaxNodes = static_cast<long long>(kNoAllocSlots) * kNoAllocNodesPerBlock;

// [kNoAllocSlots][2] doubles = 64 KiB. Every GPU that loads the library holds it until the
// process exits. All calls share it; a call overwrites the slots it uses before reading them.
static __device__ __align__(256) double g_energy_scratch[2 * kNoAllocSlots];

__global__ void __launch_bounds__(kNoAllocThreads)
    block_sums_kernel(const float* __restrict__ u, const float* __restrict__ v, const float* __restrict__ f,
                      const float* __restrict__ minv, const int* __restrict__ node_new, int nglob,
                      double* __restrict__ scratch) {
  __shared__ double sk[kNoAllocThreads], sp[kNoAllocThreads];
  const long long first = static_cast<long long>(blockIdx.x) * kNoAllocNodesPerBlock;
  const long long last = min(first + kNoAllocNodesPerBlock, static_cast<long long>(nglob));
  double kin = 0.0, pot = 0.0;
  for (long long g = first + threadIdx.x; g < last; g += kNoAllocThreads) {
    const float m = minv[node_new[g]];  // u, v, f are in caller node order, minv internal
    const double vx = v[3 * g], vy = v[3 * g + 1], vz = v[3 * g + 2];
    if (m > 0.f) kin += (vx * vx + vy * vy + vz * vz) / static_cast<double>(m);
    pot += static_cast<double>(u[3 * g]) * f[3 * g] + static_cast<double>(u[3 * g + 1]) * f[3 * g + 1] +
           static_cast<double>(u[3 * g + 2]) * f[3 * g + 2];
  }
  sk[threadIdx.x] = kin;
  sp[threadIdx.x] = pot;
  __syncthreads();
  for (int w = kNoAllocThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sk[threadIdx.x] += sk[threadIdx.x + w];
      sp[threadIdx.x] += sp[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    scratch[2 * blockIdx.x] = sk[0];
    scratch[2 * blockIdx.x + 1] = sp[0];
  }
}

// One block: sums the nblocks pairs in a fixed order and leaves
// (1/2 sum |v|^2 M, -1/2 sum u.f) in slots 0 and 1.
__global__ void __launch_bounds__(kNoAllocThreads) final_sum_kernel(double* scratch, int nblocks) {
  __shared__ double sk[kNoAllocThreads], sp[kNoAllocThreads];
  double kin = 0.0, pot = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += kNoAllocThreads) {
    kin += scratch[2 * b];
    pot += scratch[2 * b + 1];
  }
  sk[threadIdx.x] = kin;
  sp[threadIdx.x] = pot;
  __syncthreads();
  for (int w = kNoAllocThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sk[threadIdx.x] += sk[threadIdx.x + w];
      sp[threadIdx.x] += sp[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    scratch[0] = 0.5 * sk[0];
    scratch[1] = -0.5 * sp[0];  // f = -K u
  }
}

}  // namespace
}  // namespace semgb

using namespace semgb;

extern "C" int sem_energy_noalloc(sem_ctx* ctx, int nglob, const float* u_dev, const float* v_dev,
                                  const float* f_dev, double* out) {
  if (nglob < 0) return ctx_fail(ctx, SEM_EINVAL, "sem_energy_noalloc: nglob must be >= 0");
  if (nglob > kNoAllocMaxNodes)
    return ctx_fail(ctx, SEM_EINVAL,
                    ("sem_energy_noalloc: nglob = " + std::to_string(nglob) + " exceeds the maximum of " +
                     std::to_string(kNoAllocMaxNodes) + " nodes that its fixed scratch array supports")
                        .c_str());
  CtxView cv{};
  int r = ctx_view(ctx, &cv);
  if (r) return r;
  if (nglob != cv.nglob) return ctx_fail(ctx, SEM_EINVAL, "sem_energy_noalloc: nglob differs from the mesh");
  if (!u_dev || !v_dev || !f_dev || !out) return ctx_fail(ctx, SEM_EINVAL, "sem_energy_noalloc: NULL pointer");
  cudaError_t e = cudaSetDevice(cv.device);
  if (e != cudaSuccess) return ctx_fail(ctx, SEM_ECUDA, cudaGetErrorString(e));
  cudaStream_t s = static_cast<cudaStream_t>(cv.stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return ctx_fail(ctx, SEM_ECUDA, cudaGetErrorString(e));
  if (cap != cudaStreamCaptureStatusNone)
    return ctx_fail(ctx, SEM_ESTATE, "sem_energy_noalloc: the context's stream is capturing (the call synchronizes)");
  // the array's device address on the current device, looked up on every call (cheap, no
  // allocation, and never stale)
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_energy_scratch);
  if (e != cudaSuccess)
    return ctx_fail(ctx, SEM_ECUDA, (std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
  double* scratch = static_cast<double*>(p);
  const int nblocks = nglob > 0 ? (nglob + kNoAllocNodesPerBlock - 1) / kNoAllocNodesPerBlock : 1;
  block_sums_kernel<<<nblocks, kNoAllocThreads, 0, s>>>(u_dev, v_dev, f_dev, cv.minv, cv.node_new, nglob, scratch);
  final_sum_kernel<<<1, kNoAllocThreads, 0, s>>>(scratch, nblocks);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, scratch, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess)
    return ctx_fail(ctx, SEM_ECUDA, (std::string("sem_energy_noalloc: ") + cudaGetErrorString(e)).c_str());
  return SEM_OK;
}
