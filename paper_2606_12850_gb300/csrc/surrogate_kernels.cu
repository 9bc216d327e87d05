// CUDA kernels of the seismogram surrogate (sm_103a). Products (bfloat16 operands, float32
// accumulation) on the fifth-generation tensor cores: tcgen05.mma with the accumulator in
// tensor memory, for the width-3 convolutions (tc_conv_kernel), their data and weight
// gradients (tc_conv_dgrad_kernel, tc_conv_wgrad_kernel) and, through operand loaders that
// express each layer, the dense layers and their backward products (tc_gemm_kernel); the
// same products on the warp-level mma.sync kernel (gemm_kernel) as the alternative. Bias,
// activation, loss and Adam kernels. Every sum is accumulated in float32 in a fixed order
// (split-K partial sums are added in split order).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "surrogate_internal.h"

namespace sgk {
namespace {

constexpr int BN = 64;
constexpr float kGeluC = 0.7978845608028654f;  // sqrt(2 / pi)
constexpr float kGeluA = 0.044715f;

__device__ __forceinline__ float gelu(float x) {
  return 0.5f * x * (1.f + tanhf(kGeluC * (x + kGeluA * x * x * x)));
}
__device__ __forceinline__ float gelu_grad(float x) {
  const float t = tanhf(kGeluC * (x + kGeluA * x * x * x));
  return 0.5f * (1.f + t) + 0.5f * x * (1.f - t * t) * kGeluC * (1.f + 3.f * kGeluA * x * x);
}

// C[m][n] = sum_k A(m, k) B(k, n) over k in this CTA's split, on the tensor cores: the
// loader functors (kAlong: which index is contiguous in memory, so that consecutive threads
// load consecutive words) read float32 operands, which are rounded to bfloat16 (nearest
// even) into shared memory; warp-level mma.sync m16n8k16 (bf16 x bf16, float32
// accumulators). 2 BM threads, a BM x 64 tile (BM = 128 or 256), each warp a 32 x 32 part
// as 2 x 4 mma tiles, K in steps of 32. Tall tiles cut how often the activation operand of
// the wide layers is read again (once per BM rows of the result). The result goes to the
// epilogue EP, or as a split-K partial to ws[z][M][N].
constexpr int BKM = 32;          // K step of the product kernel
constexpr int SROW = BKM + 8;    // bf16 per shared row: 20 words, so 8 rows x 4 words hit 32 banks

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int BM, class LA, class LB, class EP>
__global__ void __launch_bounds__(2 * BM) gemm_kernel(int M, int N, int K, int kchunk, LA la, LB lb, EP ep, float* ws) {
  constexpr int MT = 2 * BM;  // BM / 32 warps along M, 2 along N
  __shared__ __align__(16) bf16 As[BM][SROW];  // [m][k]
  __shared__ __align__(16) bf16 Bs[BN][SROW];  // [n][k]
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 1, wn = warp & 1;
  const int g = lane >> 2, t = lane & 3;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
  for (int k0 = kbeg; k0 < kend; k0 += BKM) {
#pragma unroll
    for (int r = 0; r < BM * BKM / MT; ++r) {
      const int idx = tid + r * MT;
      const int kk = LA::kAlongK ? idx % BKM : idx / BM;
      const int mm = LA::kAlongK ? idx / BKM : idx % BM;
      const int m = m0 + mm, k = k0 + kk;
      As[mm][kk] = __float2bfloat16_rn((m < M && k < kend) ? la(m, k) : 0.f);
    }
#pragma unroll
    for (int r = 0; r < BN * BKM / MT; ++r) {
      const int idx = tid + r * MT;
      const int nn = LB::kAlongN ? idx % BN : idx / BKM;
      const int kk = LB::kAlongN ? idx / BN : idx % BKM;
      const int n = n0 + nn, k = k0 + kk;
      Bs[nn][kk] = __float2bfloat16_rn((n < N && k < kend) ? lb(k, n) : 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BKM; kk += 16) {
      uint32_t a[2][4], b[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r0 = wm * 32 + i * 16 + g;
        a[i][0] = *reinterpret_cast<const uint32_t*>(&As[r0][kk + 2 * t]);
        a[i][1] = *reinterpret_cast<const uint32_t*>(&As[r0 + 8][kk + 2 * t]);
        a[i][2] = *reinterpret_cast<const uint32_t*>(&As[r0][kk + 2 * t + 8]);
        a[i][3] = *reinterpret_cast<const uint32_t*>(&As[r0 + 8][kk + 2 * t + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c0 = wn * 32 + j * 8 + g;
        b[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[c0][kk + 2 * t]);
        b[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[c0][kk + 2 * t + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int m = m0 + wm * 32 + i * 16 + g + (r >= 2 ? 8 : 0);
        const int n = n0 + wn * 32 + j * 8 + 2 * t + (r & 1);
        if (m < M && n < N) {
          if (ws)
            ws[(static_cast<size_t>(blockIdx.z) * M + m) * N + n] = acc[i][j][r];
          else
            ep(m, n, acc[i][j][r]);
        }
      }
}

// ---- the same product on the fifth-generation tensor cores ------------------------------------
// C[m][n] = sum_k A(m, k) B(k, n) with tcgen05: a 128 x 128 tile per CTA, the float32
// accumulator in tensor memory (TMEM lanes = the 128 rows, 128 columns). Eight warps stage the
// operands: the same loader functors read float32 values, which are rounded to bfloat16
// (nearest even) and stored in shared memory in the canonical K-major layout of 8-row x
// 16-byte core matrices without swizzle (core (g, j) of an operand, rows 8g..8g+7 and K
// elements 8j..8j+7 of the stage, at byte (j * 16 + g) * 128). Each warp writes one whole core
// matrix per store instruction (8 rows x 4 words: no bank conflict), and lanes follow the
// operand's contiguous index so the global reads are sector-dense. One thread issues the
// MMAs (M = 128, N = 128, K = 16 each) and commits them to the stage's mbarrier, which tells
// the loaders when the stage may be overwritten: four stages of K = 32, so the loads of later
// stages overlap the MMAs of earlier ones. The epilogue reads TMEM (tcgen05.ld, 32 lanes x 32
// columns per warp and load), stages the tile in shared memory and calls EP (or stores a
// split-K partial) with consecutive threads on consecutive n. Every wait is bounded: a stage
// whose MMAs do not complete within kTcWaitNs sets *err, and the CTA frees its TMEM and
// returns.
constexpr int TC_BM = 128;                     // tile rows = MMA M = TMEM lanes
constexpr int TC_BN = 128;                     // tile columns = MMA N = TMEM columns
constexpr int TC_BK = 32;                      // K of a stage
constexpr int TC_STAGES = 4;
constexpr int TC_THREADS = 256;
constexpr int TC_CORE = 128;                   // bytes of a core matrix
constexpr int TC_GROUPS = TC_BM / 8;           // 8-row groups of an operand tile (BM == BN)
constexpr int TC_KCORES = TC_BK / 8;           // core matrices along K in a stage
constexpr int TC_OPERAND = TC_GROUPS * TC_KCORES * TC_CORE;  // 8 KB
constexpr int TC_STAGE = 2 * TC_OPERAND;                     // A then B
constexpr uint32_t TC_LBO = TC_GROUPS * TC_CORE;             // next core along K
constexpr uint32_t TC_SBO = TC_CORE;                         // next 8-row group
constexpr int TC_EPI_LD = TC_BN + 1;                         // floats per staged output row
// operand stages, then (reused) the epilogue's output tile; 3 CTAs a SM (3 x 128 TMEM columns)
constexpr int TC_DATA = (TC_STAGES * TC_STAGE > TC_BM * TC_EPI_LD * 4 ? TC_STAGES * TC_STAGE : TC_BM * TC_EPI_LD * 4);
constexpr int TC_SMEM = TC_DATA + 64;                        // + mbarriers and the TMEM address
constexpr unsigned long long kTcWaitNs = 2000000000ull;      // 2 s
static_assert(TC_STAGES * TC_STAGE <= TC_DATA && TC_BM * TC_EPI_LD * 4 <= TC_DATA, "shared memory plan");
static_assert(TC_GROUPS == 2 * (TC_THREADS / 32) && TC_BN / 2 % 32 == 0, "tile plan: two row groups a warp");

// Instruction descriptor of tcgen05.mma kind::f16: float32 D (bits 4-5 = 1), bfloat16 A and B
// (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at
// bits 24-28.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(TC_BN >> 3) << 17) |
                              (static_cast<uint32_t>(TC_BM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase of the given parity to complete; false after limit_ns.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns = kTcWaitNs) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_test(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: start, leading (K) and stride (8-row) byte offsets, all
// >> 4; bit 46 = descriptor version 1; no swizzle, base offset 0.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo = TC_LBO) {
  return static_cast<uint64_t>((addr >> 4) & 0x3FFFu) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
         (static_cast<uint64_t>((TC_SBO >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(da), "l"(db), "r"(kTcIdesc), "r"(accumulate)
      : "memory");
}
// The stage's mbarrier completes its phase when every MMA this thread issued so far is done.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}
// Initialises the stages' mbarriers and allocates the CTA's 128 TMEM columns; returns their
// address. All threads.
__device__ uint32_t tc_begin(uint64_t* bars, int nbars, uint32_t* slot, int tid, int warp) {
  if (tid == 0) {
    for (int s = 0; s < nbars; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(TC_BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return *slot;
}
// Waits for the MMAs of the last issued stage (the stages complete in order); true, for every
// thread, when some wait of the CTA gave up.
__device__ bool tc_finish(uint64_t* bars, int nstages, int issued, bool late) {
  if (issued > 0) {
    const int ls = issued - 1;
    if (!mbar_wait(smem_addr(&bars[ls % nstages]), (ls / nstages) & 1)) late = true;
  }
  const bool failed = __syncthreads_or(late) != 0;
  tc_fence_after();
  return failed;
}
// The accumulator (TMEM lanes = rows, 128 float32 columns) to tile[128][TC_EPI_LD] in shared
// memory (zeros when no MMA was issued; untouched when the CTA failed), then frees the TMEM.
// Warp w reads lanes 32 (w % 4) .. + 31, columns 64 (w / 4) .. + 63. All threads.
__device__ void tc_drain_tile(uint32_t tmem, float* tile, bool issued, bool failed, int warp, int lane) {
  if (!failed) {
    const int q = warp & 3, h = warp >> 2;
    float* row = tile + (q * 32 + lane) * TC_EPI_LD + h * (TC_BN / 2);
#pragma unroll
    for (int c = 0; c < TC_BN / 2; c += 32) {
      uint32_t v[32];
      if (issued) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
              "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
              "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
              "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(tmem + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(h * (TC_BN / 2) + c)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0u;
      }
#pragma unroll
      for (int i = 0; i < 32; ++i) row[c + i] = __uint_as_float(v[i]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_BN) : "memory");
}

// The part of one operand stage that a lane writes: one word (two consecutive K elements of
// one row, packed bfloat16) in each core matrix (g, j) with g in {warp, warp + 8} and j < 4.
// The lane's two rows and their loader state stay fixed for the whole K loop.
template <bool ALONG_ROWS, class F>
struct CoreFiller {
  typename F::Row rs[2];
  bool in[2];
  int r, w;
  __device__ void init(const F& f, int row0, int rows, int warp, int lane) {
    r = ALONG_ROWS ? (lane & 7) : (lane >> 2);
    w = ALONG_ROWS ? (lane >> 3) : (lane & 3);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = row0 + (warp + 8 * h) * 8 + r;
      in[h] = i < rows;
      rs[h] = f.row(in[h] ? i : row0);
    }
  }
  __device__ void fill(const F& f, uint8_t* op, int k0, int kend, int warp) const {
#pragma unroll
    for (int i = 0; i < 2 * TC_KCORES; ++i) {
      const int h = i & 1, j = i >> 1;
      const int k = k0 + j * 8 + 2 * w;
      const float v0 = (in[h] && k < kend) ? f.at(rs[h], k) : 0.f;
      const float v1 = (in[h] && k + 1 < kend) ? f.at(rs[h], k + 1) : 0.f;
      const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(v0));
      const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(v1));
      *reinterpret_cast<uint32_t*>(op + (j * TC_GROUPS + warp + 8 * h) * TC_CORE + r * 16 + w * 4) = lo | (hi << 16);
    }
  }
};

template <class LA, class LB, class EP>
__global__ void __launch_bounds__(TC_THREADS) tc_gemm_kernel(int M, int N, int K, int kchunk, LA la, LB lb, EP ep,
                                                              float* ws, int* err, int stall_test) {
  extern __shared__ __align__(128) uint8_t tc_smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(tc_smem + TC_DATA);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + TC_STAGES);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // tiles numbered m-fastest, so the row tiles that share a column block run side by side
  const int mt = (M + TC_BM - 1) / TC_BM;
  const int m0 = (blockIdx.x % mt) * TC_BM, n0 = (blockIdx.x / mt) * TC_BN;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int nst = kend > kbeg ? (kend - kbeg + TC_BK - 1) / TC_BK : 0;
  CoreFiller<!LA::kAlongK, LA> fa;
  CoreFiller<LB::kAlongN, LB> fb;
  fa.init(la, m0, M, warp, lane);
  fb.init(lb, n0, N, warp, lane);
  const uint32_t tmem = tc_begin(bars, TC_STAGES, tmem_slot, tid, warp);
  int issued = 0;
  bool late = false;
  // stall test: wait (20 ms limit) for a phase that no commit completes
  if (stall_test && !mbar_wait(smem_addr(&bars[0]), 0, 20000000ull)) late = true;
  if (__syncthreads_or(late)) issued = -1;
  for (int s = 0; s < nst && issued >= 0; ++s) {
    const int buf = s % TC_STAGES;
    if (s >= TC_STAGES && !mbar_wait(smem_addr(&bars[buf]), ((s / TC_STAGES) - 1) & 1)) late = true;
    uint8_t* a_op = tc_smem + buf * TC_STAGE;
    uint8_t* b_op = a_op + TC_OPERAND;
    const int k0 = kbeg + s * TC_BK;
    if (!late) {
      fa.fill(la, a_op, k0, kend, warp);
      fb.fill(lb, b_op, k0, kend, warp);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (__syncthreads_or(late)) break;
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a_addr = smem_addr(a_op), b_addr = smem_addr(b_op);
#pragma unroll
      for (int j = 0; j < TC_KCORES / 2; ++j)
        tc_mma(tmem, tc_desc(a_addr + 2 * j * TC_LBO), tc_desc(b_addr + 2 * j * TC_LBO), (s | j) != 0);
      tc_commit(&bars[buf]);
    }
    ++issued;
  }
  if (issued < 0) issued = 0;
  const bool failed = tc_finish(bars, TC_STAGES, issued, late);
  float* tile = reinterpret_cast<float*>(tc_smem);
  tc_drain_tile(tmem, tile, issued > 0, failed, warp, lane);
  if (failed) {
    if (tid == 0) atomicExch(err, 1);
    return;
  }
  for (int idx = tid; idx < TC_BM * TC_BN; idx += TC_THREADS) {
    const int mm = idx / TC_BN, nn = idx - mm * TC_BN;
    const int m = m0 + mm, n = n0 + nn;
    if (m < M && n < N) {
      const float v = tile[mm * TC_EPI_LD + nn];
      if (ws)
        ws[(static_cast<size_t>(blockIdx.z) * M + m) * N + n] = v;
      else
        ep(m, n, v);
    }
  }
}

// ---- the width-3 convolution forward on tcgen05, its input window staged once ---------------
// pre[b][o][t] = bias[o] + sum_{c,d} W[o][c][d] X[b][c][(t + d - 1) >> ush] (zero outside
// [0, L)), out = gelu(pre) when out != nullptr. A CTA owns 128 output channels x 128 times
// t0 .. t0 + 127 of one sample b (tiles numbered channel tile fastest). Per chunk of 32 input
// channels it stages the upsampled input window s = t0 - 1 .. t0 + 134 as K-major rows (row R
// holds time t0 - 1 + R, K = channel) and the three taps' 128 x 32 weights, packed beforehand
// into the core-matrix layout (pack_conv_weights_kernel) so that staging them is 16-byte
// copies. Tap d multiplies output time t0 + n with window row n + d: the same staged rows
// through a descriptor that starts d rows (16 bytes) later, so the window serves all three
// taps. Six MMAs (three taps x two K = 16 halves) a chunk, two chunk stages in flight; the
// epilogue adds the bias and the activation with consecutive threads on consecutive times.
constexpr int CV_CK = 32;                               // input channels a chunk
constexpr int CV_ROWS = 136;                            // window rows: >= 128 + 2, whole groups
constexpr int CV_WGROUPS = CV_ROWS / 8;
constexpr int CV_WINDOW = CV_WGROUPS * TC_KCORES * TC_CORE;  // 8704 B
constexpr int CV_TAP = TC_GROUPS * TC_KCORES * TC_CORE;      // 8192 B: 128 x 32 weights of a tap
constexpr int CV_STAGE = CV_WINDOW + 3 * CV_TAP;
constexpr int CV_STAGES = 2;
constexpr uint32_t CV_LBO = CV_WGROUPS * TC_CORE;            // window: next core along K
constexpr int CV_DATA = (CV_STAGES * CV_STAGE > TC_BM * TC_EPI_LD * 4 ? CV_STAGES * CV_STAGE : TC_BM * TC_EPI_LD * 4);
constexpr int CV_SMEM = CV_DATA + 64;
constexpr int CV_WCORES = CV_WGROUPS * TC_KCORES;            // window core matrices a stage
constexpr int CV_WITER = (CV_WCORES + TC_THREADS / 32 - 1) / (TC_THREADS / 32);
static_assert(TC_KCORES * 8 == CV_CK && CV_ROWS % 8 == 0 && CV_ROWS >= TC_BN + 2, "window plan");
static_assert(CV_STAGE % 16 == 0 && CV_WINDOW % 16 == 0 && (3 * CV_TAP / 16) % TC_THREADS == 0, "16-byte copies");

// Wp[((ot * nq + q) * 3 + d) * 4096 + e]: the weights of output-channel tile ot, input-channel
// chunk q and tap d in the core-matrix layout: element e = (j * 16 + g) * 64 + r * 8 + i holds
// W[o][c][d], o = 128 ot + 8 g + r, c = 32 q + 8 j + i (zero outside Co x Ci).
__global__ void pack_conv_weights_kernel(int Co, int Ci, int nq, size_t total, const bf16* __restrict__ W,
                                         bf16* __restrict__ Wp) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int e = static_cast<int>(i & 4095);
    const size_t blk = i >> 12;
    const int d = static_cast<int>(blk % 3);
    const size_t oq = blk / 3;
    const int q = static_cast<int>(oq % nq), ot = static_cast<int>(oq / nq);
    const int core = e >> 6, g = core & 15, j = core >> 4;
    const int o = ot * TC_BM + g * 8 + ((e >> 3) & 7), c = q * CV_CK + j * 8 + (e & 7);
    Wp[i] = (o < Co && c < Ci) ? W[(static_cast<size_t>(o) * Ci + c) * 3 + d] : __float2bfloat16_rn(0.f);
  }
}

__global__ void __launch_bounds__(TC_THREADS) tc_conv_kernel(int Ci, int Co, int Lin, int L, int ush,
                                                              const float* __restrict__ X, const bf16* __restrict__ Wp,
                                                              const float* __restrict__ bias, float* __restrict__ pre,
                                                              float* __restrict__ out, int* err, int stall_test) {
  extern __shared__ __align__(128) uint8_t cv_smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(cv_smem + CV_DATA);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + CV_STAGES);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_ot = (Co + TC_BM - 1) / TC_BM, n_tt = (L + TC_BN - 1) / TC_BN, nq = (Ci + CV_CK - 1) / CV_CK;
  const int ot = blockIdx.x % n_ot;
  const int rest = blockIdx.x / n_ot;
  const int t0 = (rest % n_tt) * TC_BN, b = rest / n_tt;
  const float* xb = X + static_cast<size_t>(b) * Ci * Lin;
  const uint32_t tmem = tc_begin(bars, CV_STAGES, tmem_slot, tid, warp);
  const int r = lane & 7, w = lane >> 3;  // window row in the group, channel pair in the core
  int issued = 0;
  bool late = false;
  if (stall_test && !mbar_wait(smem_addr(&bars[0]), 0, 20000000ull)) late = true;
  if (__syncthreads_or(late)) issued = -1;
  for (int q = 0; q < nq && issued >= 0; ++q) {
    const int buf = q % CV_STAGES;
    if (q >= CV_STAGES && !mbar_wait(smem_addr(&bars[buf]), ((q / CV_STAGES) - 1) & 1)) late = true;
    uint8_t* win = cv_smem + buf * CV_STAGE;
    uint8_t* taps = win + CV_WINDOW;
    if (!late) {
      const uint4* src = reinterpret_cast<const uint4*>(Wp + static_cast<size_t>((ot * nq + q) * 3) * (CV_TAP / 2));
      uint4 wv[3 * CV_TAP / 16 / TC_THREADS];
#pragma unroll
      for (int i = 0; i < 3 * CV_TAP / 16 / TC_THREADS; ++i) wv[i] = src[tid + i * TC_THREADS];
      float v[CV_WITER][2];
#pragma unroll
      for (int i = 0; i < CV_WITER; ++i) {
        const int cidx = warp + i * (TC_THREADS / 32);
        const int g = cidx % CV_WGROUPS, j = cidx / CV_WGROUPS;
        const int s = t0 - 1 + g * 8 + r;
        const int c = q * CV_CK + j * 8 + 2 * w;
        v[i][0] = v[i][1] = 0.f;
        if (cidx < CV_WCORES && static_cast<unsigned>(s) < static_cast<unsigned>(L)) {
          const float* p = xb + static_cast<size_t>(c) * Lin + (s >> ush);
          if (c < Ci) v[i][0] = p[0];
          if (c + 1 < Ci) v[i][1] = p[Lin];
        }
      }
#pragma unroll
      for (int i = 0; i < 3 * CV_TAP / 16 / TC_THREADS; ++i) reinterpret_cast<uint4*>(taps)[tid + i * TC_THREADS] = wv[i];
#pragma unroll
      for (int i = 0; i < CV_WITER; ++i) {
        const int cidx = warp + i * (TC_THREADS / 32);
        if (cidx < CV_WCORES) {
          const int g = cidx % CV_WGROUPS, j = cidx / CV_WGROUPS;
          const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(v[i][0]));
          const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(v[i][1]));
          *reinterpret_cast<uint32_t*>(win + (j * CV_WGROUPS + g) * TC_CORE + r * 16 + w * 4) = lo | (hi << 16);
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (__syncthreads_or(late)) break;
    if (tid == 0) {
      tc_fence_after();
      const uint32_t w_addr = smem_addr(win), a_addr = smem_addr(taps);
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int j = 0; j < TC_KCORES / 2; ++j)
          tc_mma(tmem, tc_desc(a_addr + d * CV_TAP + 2 * j * TC_LBO), tc_desc(w_addr + d * 16 + 2 * j * CV_LBO, CV_LBO),
                 (q | d | j) != 0);
      tc_commit(&bars[buf]);
    }
    ++issued;
  }
  if (issued < 0) issued = 0;
  const bool failed = tc_finish(bars, CV_STAGES, issued, late);
  float* tile = reinterpret_cast<float*>(cv_smem);
  tc_drain_tile(tmem, tile, issued > 0, failed, warp, lane);
  if (failed) {
    if (tid == 0) atomicExch(err, 1);
    return;
  }
  const int o0 = ot * TC_BM;
  for (int idx = tid; idx < TC_BM * TC_BN; idx += TC_THREADS) {
    const int mm = idx / TC_BN, nn = idx - mm * TC_BN;
    const int o = o0 + mm, t = t0 + nn;
    if (o < Co && t < L) {
      const float p = tile[mm * TC_EPI_LD + nn] + bias[o];
      const size_t i = (static_cast<size_t>(b) * Co + o) * L + t;
      pre[i] = p;
      if (out) out[i] = gelu(p);
    }
  }
}

// ---- the convolution's weight gradient on tcgen05 ------------------------------------------
// dW[o][c][d] = sum_{b,t} dZ[b][o][t] X[b][c][(t + d - 1) >> ush] (zero outside [0, L)). A CTA
// owns 128 output channels x 128 input channels of one tap d and the samples of split z of S;
// its K loop runs over those samples' times in chunks of 32, staging dZ (rows o) and the tap's
// shifted input (rows c) as K-major operands, with no index division. The sums go to
// dst[z][o][c * 3 + d]: the split-K workspace (added in split order afterwards) or dW itself.
__global__ void __launch_bounds__(TC_THREADS) tc_conv_wgrad_kernel(int B, int Ci, int Co, int Lin, int L, int ush,
                                                                    int S, const float* __restrict__ dZ,
                                                                    const float* __restrict__ X,
                                                                    float* __restrict__ dst, int* err, int stall_test) {
  extern __shared__ __align__(128) uint8_t wg_smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(wg_smem + TC_DATA);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + TC_STAGES);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_ot = (Co + TC_BM - 1) / TC_BM, n_ct = (Ci + TC_BN - 1) / TC_BN;
  int id = blockIdx.x;
  const int ot = id % n_ot;
  id /= n_ot;
  const int d = id % 3;
  id /= 3;
  const int ct = id % n_ct, z = id / n_ct;
  const int b0 = static_cast<int>(static_cast<long long>(z) * B / S);
  const int b1 = static_cast<int>(static_cast<long long>(z + 1) * B / S);
  const int nchunk = (L + TC_BK - 1) / TC_BK;
  const int nst = (b1 - b0) * nchunk;
  const int o0 = ot * TC_BM, c0 = ct * TC_BN;
  const int r = lane >> 2, w = lane & 3;  // K is contiguous in both operands
  int orow[2], crow[2];
  bool oin[2], cin[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    orow[h] = o0 + (warp + 8 * h) * 8 + r;
    crow[h] = c0 + (warp + 8 * h) * 8 + r;
    oin[h] = orow[h] < Co;
    cin[h] = crow[h] < Ci;
  }
  const uint32_t tmem = tc_begin(bars, TC_STAGES, tmem_slot, tid, warp);
  int issued = 0;
  bool late = false;
  if (stall_test && !mbar_wait(smem_addr(&bars[0]), 0, 20000000ull)) late = true;
  if (__syncthreads_or(late)) issued = -1;
  for (int s = 0; s < nst && issued >= 0; ++s) {
    const int buf = s % TC_STAGES;
    if (s >= TC_STAGES && !mbar_wait(smem_addr(&bars[buf]), ((s / TC_STAGES) - 1) & 1)) late = true;
    uint8_t* a_op = wg_smem + buf * TC_STAGE;
    uint8_t* b_op = a_op + TC_OPERAND;
    if (!late) {
      const int b = b0 + s / nchunk, t0 = (s % nchunk) * TC_BK;
      const float* zb = dZ + static_cast<size_t>(b) * Co * L;
      const float* xb = X + static_cast<size_t>(b) * Ci * Lin;
      float va[2][TC_KCORES][2], vb[2][TC_KCORES][2];
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < TC_KCORES; ++j)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int t = t0 + j * 8 + 2 * w + e;
            const int u = t + d - 1;
            va[h][j][e] = (oin[h] && t < L) ? zb[static_cast<size_t>(orow[h]) * L + t] : 0.f;
            vb[h][j][e] = (cin[h] && t < L && static_cast<unsigned>(u) < static_cast<unsigned>(L))
                              ? xb[static_cast<size_t>(crow[h]) * Lin + (u >> ush)]
                              : 0.f;
          }
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < TC_KCORES; ++j) {
          const int off = (j * TC_GROUPS + warp + 8 * h) * TC_CORE + r * 16 + w * 4;
          *reinterpret_cast<uint32_t*>(a_op + off) =
              static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(va[h][j][0]))) |
              (static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(va[h][j][1]))) << 16);
          *reinterpret_cast<uint32_t*>(b_op + off) =
              static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(vb[h][j][0]))) |
              (static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(vb[h][j][1]))) << 16);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (__syncthreads_or(late)) break;
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a_addr = smem_addr(a_op), b_addr = smem_addr(b_op);
#pragma unroll
      for (int j = 0; j < TC_KCORES / 2; ++j)
        tc_mma(tmem, tc_desc(a_addr + 2 * j * TC_LBO), tc_desc(b_addr + 2 * j * TC_LBO), (s | j) != 0);
      tc_commit(&bars[buf]);
    }
    ++issued;
  }
  if (issued < 0) issued = 0;
  const bool failed = tc_finish(bars, TC_STAGES, issued, late);
  float* tile = reinterpret_cast<float*>(wg_smem);
  tc_drain_tile(tmem, tile, issued > 0, failed, warp, lane);
  if (failed) {
    if (tid == 0) atomicExch(err, 1);
    return;
  }
  float* out = dst + static_cast<size_t>(z) * Co * Ci * 3;
  for (int idx = tid; idx < TC_BM * TC_BN; idx += TC_THREADS) {
    const int mm = idx / TC_BN, nn = idx - mm * TC_BN;
    const int o = o0 + mm, c = c0 + nn;
    if (o < Co && c < Ci) out[(static_cast<size_t>(o) * Ci + c) * 3 + d] = tile[mm * TC_EPI_LD + nn];
  }
}

// Wt[((ct * nq + q) * 3 + d) * 4096 + e]: W[o][c][d] transposed (rows c, K = o) in the
// core-matrix layout: element e = (j * 16 + g) * 64 + r * 8 + i holds c = 128 ct + 8 g + r,
// o = 32 q + 8 j + i (zero outside Co x Ci).
__global__ void pack_conv_weights_t_kernel(int Co, int Ci, int nq, size_t total, const bf16* __restrict__ W,
                                           bf16* __restrict__ Wt) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int e = static_cast<int>(i & 4095);
    const size_t blk = i >> 12;
    const int d = static_cast<int>(blk % 3);
    const size_t cq = blk / 3;
    const int q = static_cast<int>(cq % nq), ct = static_cast<int>(cq / nq);
    const int core = e >> 6, g = core & 15, j = core >> 4;
    const int c = ct * TC_BM + g * 8 + ((e >> 3) & 7), o = q * CV_CK + j * 8 + (e & 7);
    Wt[i] = (o < Co && c < Ci) ? W[(static_cast<size_t>(o) * Ci + c) * 3 + d] : __float2bfloat16_rn(0.f);
  }
}

// ---- the convolution's data gradient on tcgen05 ---------------------------------------------
// dX[b][c][t'] = sum_{o,d,r<UP} W[o][c][d] dZ[b][o][UP t' + r - d + 1] (zero outside [0, L)).
// A CTA owns 128 input channels x 128 times t0' .. t0' + 127 of one sample b. Per chunk of 32
// output channels it stages dZ around the tile as K-major windows of 136 rows (K = output
// channel): UP = 1, one window, row R = time t0' - 1 + R; UP = 2, two, row R = time
// 2 (t0' - 1 + R) + p for parity p. Term (r, d) reads time UP (t0' + n) + e, e = r - d + 1,
// which is row n + 1 + (e - p) / UP of window p = e mod UP: the staged rows through a
// descriptor offset by that many rows. The taps' transposed weights are 16-byte copies.
template <int UP>
struct Dgrad {
  static constexpr int kStage = UP * CV_WINDOW + 3 * CV_TAP;
  static constexpr int kData = (2 * kStage > TC_BM * TC_EPI_LD * 4 ? 2 * kStage : TC_BM * TC_EPI_LD * 4);
  static constexpr int kSmem = kData + 64;
  static constexpr int kCores = UP * CV_WCORES;
  static constexpr int kIter = (kCores + TC_THREADS / 32 - 1) / (TC_THREADS / 32);
};

template <int UP>
__global__ void __launch_bounds__(TC_THREADS) tc_conv_dgrad_kernel(int Ci, int Co, int Lin, int L,
                                                                    const float* __restrict__ dZ,
                                                                    const bf16* __restrict__ Wt, float* __restrict__ dX,
                                                                    int* err, int stall_test) {
  using G = Dgrad<UP>;
  extern __shared__ __align__(128) uint8_t dg_smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(dg_smem + G::kData);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_ct = (Ci + TC_BM - 1) / TC_BM, n_tt = (Lin + TC_BN - 1) / TC_BN, nq = (Co + CV_CK - 1) / CV_CK;
  const int ct = blockIdx.x % n_ct;
  const int rest = blockIdx.x / n_ct;
  const int t0 = (rest % n_tt) * TC_BN, b = rest / n_tt;
  const float* zb = dZ + static_cast<size_t>(b) * Co * L;
  const uint32_t tmem = tc_begin(bars, 2, tmem_slot, tid, warp);
  const int r = lane & 7, w = lane >> 3;  // window row in the group, output-channel pair
  int issued = 0;
  bool late = false;
  if (stall_test && !mbar_wait(smem_addr(&bars[0]), 0, 20000000ull)) late = true;
  if (__syncthreads_or(late)) issued = -1;
  for (int q = 0; q < nq && issued >= 0; ++q) {
    const int buf = q & 1;
    if (q >= 2 && !mbar_wait(smem_addr(&bars[buf]), ((q >> 1) - 1) & 1)) late = true;
    uint8_t* win = dg_smem + buf * G::kStage;
    uint8_t* taps = win + UP * CV_WINDOW;
    if (!late) {
      const uint4* src = reinterpret_cast<const uint4*>(Wt + static_cast<size_t>((ct * nq + q) * 3) * (CV_TAP / 2));
      uint4 wv[3 * CV_TAP / 16 / TC_THREADS];
#pragma unroll
      for (int i = 0; i < 3 * CV_TAP / 16 / TC_THREADS; ++i) wv[i] = src[tid + i * TC_THREADS];
      float v[G::kIter][2];
#pragma unroll
      for (int i = 0; i < G::kIter; ++i) {
        const int cidx = warp + i * (TC_THREADS / 32);
        const int p = cidx / CV_WCORES, within = cidx - p * CV_WCORES;
        const int g = within % CV_WGROUPS, j = within / CV_WGROUPS;
        const int u = UP * (t0 - 1 + g * 8 + r) + p;
        const int o = q * CV_CK + j * 8 + 2 * w;
        v[i][0] = v[i][1] = 0.f;
        if (cidx < G::kCores && static_cast<unsigned>(u) < static_cast<unsigned>(L)) {
          const float* pz = zb + static_cast<size_t>(o) * L + u;
          if (o < Co) v[i][0] = pz[0];
          if (o + 1 < Co) v[i][1] = pz[L];
        }
      }
#pragma unroll
      for (int i = 0; i < 3 * CV_TAP / 16 / TC_THREADS; ++i) reinterpret_cast<uint4*>(taps)[tid + i * TC_THREADS] = wv[i];
#pragma unroll
      for (int i = 0; i < G::kIter; ++i) {
        const int cidx = warp + i * (TC_THREADS / 32);
        if (cidx < G::kCores) {
          const int p = cidx / CV_WCORES, within = cidx - p * CV_WCORES;
          const int g = within % CV_WGROUPS, j = within / CV_WGROUPS;
          const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(v[i][0]));
          const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(v[i][1]));
          *reinterpret_cast<uint32_t*>(win + p * CV_WINDOW + (j * CV_WGROUPS + g) * TC_CORE + r * 16 + w * 4) =
              lo | (hi << 16);
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (__syncthreads_or(late)) break;
    if (tid == 0) {
      tc_fence_after();
      const uint32_t w_addr = smem_addr(win), a_addr = smem_addr(taps);
      bool first = q == 0;
#pragma unroll
      for (int rr = 0; rr < UP; ++rr)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const int e = rr - d + 1;           // -1 .. 2
          const int p = UP == 2 ? (e & 1) : 0;
          const int off = 1 + (UP == 2 ? (e - p) / 2 : e);  // window row of output row 0
#pragma unroll
          for (int j = 0; j < TC_KCORES / 2; ++j) {
            tc_mma(tmem, tc_desc(a_addr + d * CV_TAP + 2 * j * TC_LBO),
                   tc_desc(w_addr + p * CV_WINDOW + off * 16 + 2 * j * CV_LBO, CV_LBO), first ? 0u : 1u);
            first = false;
          }
        }
      tc_commit(&bars[buf]);
    }
    ++issued;
  }
  if (issued < 0) issued = 0;
  const bool failed = tc_finish(bars, 2, issued, late);
  float* tile = reinterpret_cast<float*>(dg_smem);
  tc_drain_tile(tmem, tile, issued > 0, failed, warp, lane);
  if (failed) {
    if (tid == 0) atomicExch(err, 1);
    return;
  }
  const int c0 = ct * TC_BM;
  for (int idx = tid; idx < TC_BM * TC_BN; idx += TC_THREADS) {
    const int mm = idx / TC_BN, nn = idx - mm * TC_BN;
    const int c = c0 + mm, t = t0 + nn;
    if (c < Ci && t < Lin) dX[(static_cast<size_t>(b) * Ci + c) * Lin + t] = tile[mm * TC_EPI_LD + nn];
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

int tile_rows(int M) { return M >= 512 ? 256 : 128; }

// CTAs that fill the GPU once: 152 SMs x resident CTAs of the product kernel
int splits_for(int M, int N, int K, int kind) {
  const int bm = kind == 1 ? TC_BM : tile_rows(M);
  const int bn = kind == 1 ? TC_BN : BN;
  const int fill = kind == 1 ? 152 * 3 : 152 * 4;
  const int tiles = ((M + bm - 1) / bm) * ((N + bn - 1) / bn);
  int s = (fill + tiles - 1) / tiles;
  const int kmax = (K + 255) / 256;
  if (s > kmax) s = kmax;
  if (s > 64) s = 64;
  return s < 1 ? 1 : s;
}

template <class LA, class LB, class EP>
int run_gemm(int M, int N, int K, LA la, LB lb, EP ep, float* ws, bool allow_split, const Products& pr,
             cudaStream_t s) {
  if (M <= 0 || N <= 0) return 0;
  if (pr.kind != 0 && (pr.kind != 1 || !pr.err)) return static_cast<int>(cudaErrorInvalidValue);
  int splits = (allow_split && ws) ? splits_for(M, N, K, pr.kind) : 1;
  const size_t mn = static_cast<size_t>(M) * N;
  if (splits > 1 && static_cast<size_t>(splits) * mn > pr.ws_floats)
    splits = static_cast<int>(std::max<size_t>(1, pr.ws_floats / mn));
  static_assert(BKM == TC_BK, "one K granule for both product kernels");
  int kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + BKM - 1) / BKM * BKM;
  const int used = K > 0 ? (K + kchunk - 1) / kchunk : 1;
  float* part = used > 1 ? ws : nullptr;
  if (pr.kind == 1) {
    const cudaError_t e =
        cudaFuncSetAttribute(tc_gemm_kernel<LA, LB, EP>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return static_cast<int>(e);
    const long long tiles = static_cast<long long>((M + TC_BM - 1) / TC_BM) * ((N + TC_BN - 1) / TC_BN);
    if (tiles > 0x7FFFFFFFLL) return static_cast<int>(cudaErrorInvalidValue);
    tc_gemm_kernel<LA, LB, EP><<<dim3(static_cast<unsigned>(tiles), 1, used), TC_THREADS, TC_SMEM, s>>>(
        M, N, K, kchunk, la, lb, ep, part, pr.err, pr.stall_test);
  } else if (tile_rows(M) == 256) {
    gemm_kernel<256><<<dim3((N + BN - 1) / BN, (M + 255) / 256, used), 512, 0, s>>>(M, N, K, kchunk, la, lb, ep, part);
  } else {
    gemm_kernel<128><<<dim3((N + BN - 1) / BN, (M + 127) / 128, used), 256, 0, s>>>(M, N, K, kchunk, la, lb, ep, part);
  }
  if (used > 1)
    splitk_finalize_kernel<<<grid_for(static_cast<size_t>(M) * N), 256, 0, s>>>(M, N, used, ws, ep);
  return static_cast<int>(cudaGetLastError());
}

// ---- loaders ------------------------------------------------------------------------------
// Each loader reads one operand as float32: A(m, k) or B(k, n). row(i) gathers what depends on
// the row alone (i = m for A, n for B) and at(row, k) reads one element, so the tcgen05 kernel,
// whose lanes keep their rows for the whole K loop, computes the row part once; operator()
// combines the two for the mma.sync kernel. kAlongK / kAlongN: the index that is contiguous in
// memory. In the convolutions up is 1 or 2 and ush = up / 2 shifts the upsampling's index map.

// q = k / d for 0 <= k < 2^24, from a float reciprocal and one correction step (the float
// quotient is within 1 of the exact one there).
struct DivBy {
  int d;
  float inv;
  __device__ __forceinline__ int operator()(int k) const {
    int q = __float2int_rz(__int2float_rn(k) * inv);
    const int r = k - q * d;
    q += (r >= d) - (r < 0);
    return q;
  }
};
DivBy div_by(int d) { return DivBy{d, 1.0f / static_cast<float>(d)}; }

struct RowMajorA {  // A(m, k) = P[m * ld + k]
  static constexpr bool kAlongK = true;
  const float* P;
  int ld;
  using Row = const float*;
  __device__ Row row(int m) const { return P + static_cast<size_t>(m) * ld; }
  __device__ float at(Row p, int k) const { return p[k]; }
  __device__ float operator()(int m, int k) const { return at(row(m), k); }
};
struct ColMajorA {  // A(m, k) = P[k * ld + m]
  static constexpr bool kAlongK = false;
  const float* P;
  int ld;
  using Row = const float*;
  __device__ Row row(int m) const { return P + m; }
  __device__ float at(Row p, int k) const { return p[static_cast<size_t>(k) * ld]; }
  __device__ float operator()(int m, int k) const { return at(row(m), k); }
};
struct RowMajorB {  // B(k, n) = P[k * ld + n]
  static constexpr bool kAlongN = true;
  const float* P;
  int ld;
  using Row = const float*;
  __device__ Row row(int n) const { return P + n; }
  __device__ float at(Row p, int k) const { return p[static_cast<size_t>(k) * ld]; }
  __device__ float operator()(int k, int n) const { return at(row(n), k); }
};
struct WeightRowB {  // B(k, n) = W[k * ld + n], bf16
  static constexpr bool kAlongN = true;
  const bf16* W;
  int ld;
  using Row = const bf16*;
  __device__ Row row(int n) const { return W + n; }
  __device__ float at(Row p, int k) const { return __bfloat162float(p[static_cast<size_t>(k) * ld]); }
  __device__ float operator()(int k, int n) const { return at(row(n), k); }
};
struct WeightColB {  // B(k, n) = W[n * ld + k], bf16
  static constexpr bool kAlongN = false;
  const bf16* W;
  int ld;
  using Row = const bf16*;
  __device__ Row row(int n) const { return W + static_cast<size_t>(n) * ld; }
  __device__ float at(Row p, int k) const { return __bfloat162float(p[k]); }
  __device__ float operator()(int k, int n) const { return at(row(n), k); }
};
struct ConvWeightA {  // A(o, k) = W[o][k], k = c * 3 + d
  static constexpr bool kAlongK = true;
  const bf16* W;
  int ld;
  using Row = const bf16*;
  __device__ Row row(int m) const { return W + static_cast<size_t>(m) * ld; }
  __device__ float at(Row p, int k) const { return __bfloat162float(p[k]); }
  __device__ float operator()(int m, int k) const { return at(row(m), k); }
};
struct ConvInputB {  // B(k = c*3+d, n = b*L+t) = X[b][c][(t + d - 1) / up], zero outside [0, L)
  static constexpr bool kAlongN = true;
  const float* X;
  int Ci, Lin, L, ush;
  DivBy byL;
  struct Row {
    const float* x;  // X[b]
    int t1;          // t - 1
  };
  __device__ Row row(int n) const {
    const int b = byL(n);
    return Row{X + static_cast<size_t>(b) * Ci * Lin, n - b * L - 1};
  }
  __device__ float at(const Row& r, int k) const {
    const int c = k / 3, d = k - 3 * c;
    const int s = r.t1 + d;
    if (static_cast<unsigned>(s) >= static_cast<unsigned>(L)) return 0.f;
    return r.x[static_cast<size_t>(c) * Lin + (s >> ush)];
  }
  __device__ float operator()(int k, int n) const { return at(row(n), k); }
};
struct ConvWeightTA {  // A(c, k = (o*3+d)*up + r) = W[o][c][d]
  static constexpr bool kAlongK = false;
  const bf16* W;
  int Ci, ush;
  using Row = const bf16*;
  __device__ Row row(int m) const { return W + static_cast<size_t>(m) * 3; }
  __device__ float at(Row p, int k) const {
    const int od = k >> ush;
    const int o = od / 3, d = od - 3 * o;
    return __bfloat162float(p[static_cast<size_t>(o) * Ci * 3 + d]);
  }
  __device__ float operator()(int m, int k) const { return at(row(m), k); }
};
struct ConvGradB {  // B(k = (o*3+d)*up + r, n = b*Lin + t') = dZ[b][o][up t' + r - d + 1]
  static constexpr bool kAlongN = true;
  const float* dZ;
  int Co, Lin, L, ush;
  DivBy byLin;
  struct Row {
    const float* z;  // dZ[b]
    int t1;          // up t' + 1
  };
  __device__ Row row(int n) const {
    const int b = byLin(n);
    return Row{dZ + static_cast<size_t>(b) * Co * L, ((n - b * Lin) << ush) + 1};
  }
  __device__ float at(const Row& rw, int k) const {
    const int od = k >> ush, r = k - (od << ush);
    const int o = od / 3, d = od - 3 * o;
    const int t = rw.t1 + r - d;
    if (static_cast<unsigned>(t) >= static_cast<unsigned>(L)) return 0.f;
    return rw.z[static_cast<size_t>(o) * L + t];
  }
  __device__ float operator()(int k, int n) const { return at(row(n), k); }
};
struct ConvGradA {  // A(o, k = b*L + t) = dZ[b][o][t]
  static constexpr bool kAlongK = true;
  const float* dZ;
  int Co, L;
  DivBy byL;
  using Row = const float*;
  __device__ Row row(int m) const { return dZ + static_cast<size_t>(m) * L; }
  __device__ float at(Row p, int k) const {
    const int b = byL(k);
    return p[static_cast<size_t>(b) * Co * L + (k - b * L)];
  }
  __device__ float operator()(int m, int k) const { return at(row(m), k); }
};
struct ConvInputWB {  // B(k = b*L + t, n = c*3 + d) = X[b][c][(t + d - 1) / up]
  static constexpr bool kAlongN = false;
  const float* X;
  int Ci, Lin, L, ush;
  DivBy byL;
  struct Row {
    const float* x;  // X[0][c]
    int dm1;         // d - 1
  };
  __device__ Row row(int n) const {
    const int c = n / 3;
    return Row{X + static_cast<size_t>(c) * Lin, n - 3 * c - 1};
  }
  __device__ float at(const Row& r, int k) const {
    const int b = byL(k);
    const int s = k - b * L + r.dm1;
    if (static_cast<unsigned>(s) >= static_cast<unsigned>(L)) return 0.f;
    return r.x[static_cast<size_t>(b) * Ci * Lin + (s >> ush)];
  }
  __device__ float operator()(int k, int n) const { return at(row(n), k); }
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
  DivBy byL;
  __device__ void operator()(int m, int n, float v) const {
    const int b = byL(n), t = n - b * L;
    const float p = v + bias[m];
    const size_t i = (static_cast<size_t>(b) * Co + m) * L + t;
    pre[i] = p;
    if (out) out[i] = gelu(p);
  }
};
struct ConvDataEp {  // (m = c, n = b*Lin + t')
  float* dX;
  int Ci, Lin;
  DivBy byLin;
  __device__ void operator()(int m, int n, float v) const {
    const int b = byLin(n), tp = n - b * Lin;
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

// db[o] = sum_{b,t} dZ[b][o][t] in two fixed-order passes: block (o, p) sums samples
// [p B / P, (p + 1) B / P) into part[p][o] (a strided sum per thread, then a tree), and
// channel_finish_kernel adds the P parts in order.
__global__ void channel_partials_kernel(int B, int Co, int L, int P, const float* __restrict__ dZ,
                                        float* __restrict__ part) {
  __shared__ float red[256];
  const int o = blockIdx.x, p = blockIdx.y;
  const int b0 = static_cast<int>(static_cast<long long>(p) * B / P);
  const int b1 = static_cast<int>(static_cast<long long>(p + 1) * B / P);
  float s = 0.f;
  for (int b = b0; b < b1; ++b) {
    const float* row = dZ + (static_cast<size_t>(b) * Co + o) * L;
    for (int t = threadIdx.x; t < L; t += blockDim.x) s += row[t];
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[static_cast<size_t>(p) * Co + o] = red[0];
}

__global__ void channel_finish_kernel(int Co, int P, const float* __restrict__ part, float* __restrict__ db) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= Co) return;
  float s = 0.f;
  for (int p = 0; p < P; ++p) s += part[static_cast<size_t>(p) * Co + o];
  db[o] = s;
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
// input features: the moment-tensor entries). Block row y walks samples, x the C*L outputs.
__global__ void contract_forward_kernel(int B, int K, int C, int L, int in_dim, int k0, const float* __restrict__ x,
                                        const float* __restrict__ D, float* __restrict__ y) {
  const size_t CL = static_cast<size_t>(C) * L;
  for (int b = blockIdx.y; b < B; b += gridDim.y) {
    const float* xb = x + static_cast<size_t>(b) * in_dim + k0;
    const float* Db = D + static_cast<size_t>(b) * K * CL;
    float* yb = y + static_cast<size_t>(b) * CL;
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < CL;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
      float s = 0.f;
      for (int k = 0; k < K; ++k) s = fmaf(xb[k], Db[k * CL + i], s);
      yb[i] = s;
    }
  }
}

// dD[b][k*C + c][t] = x[b][k0 + k] dy[b][c][t]; block row y walks the (sample, k) pairs
__global__ void contract_backward_kernel(int B, int K, int C, int L, int in_dim, int k0, const float* __restrict__ x,
                                         const float* __restrict__ dy, float* __restrict__ dD) {
  const size_t CL = static_cast<size_t>(C) * L;
  for (int bk = blockIdx.y; bk < B * K; bk += gridDim.y) {
    const int b = bk / K, k = bk - b * K;
    const float xv = x[static_cast<size_t>(b) * in_dim + k0 + k];
    const float* src = dy + static_cast<size_t>(b) * CL;
    float* dst = dD + static_cast<size_t>(bk) * CL;
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < CL;
         i += static_cast<size_t>(gridDim.x) * blockDim.x)
      dst[i] = xv * src[i];
  }
}

__global__ void to_bf16_kernel(size_t n, const float* __restrict__ p, bf16* __restrict__ pb) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    pb[i] = __float2bfloat16_rn(p[i]);
}

}  // namespace

size_t splitk_floats(int M, int N, int K) {
  const int s = max(splits_for(M, N, K, 0), splits_for(M, N, K, 1));
  return s > 1 ? static_cast<size_t>(s) * M * N : 0;
}

int linear_forward(int B, int K, int N, const float* X, const bf16* W, const float* bias, float* pre, float* out,
                   bool act, const Products& pr, cudaStream_t s) {
  return run_gemm(B, N, K, RowMajorA{X, K}, WeightColB{W, K}, LinearEp{pre, out, bias, N, act}, nullptr, false, pr, s);
}

int linear_backward_data(int B, int K, int N, const float* dZ, const bf16* W, float* dX, float* ws,
                         const Products& pr, cudaStream_t s) {
  return run_gemm(B, K, N, RowMajorA{dZ, N}, WeightRowB{W, K}, StoreEp{dX, K}, ws, true, pr, s);
}

int linear_backward_weight(int B, int K, int N, const float* dZ, const float* X, float* dW, float* db, float* ws,
                           const Products& pr, cudaStream_t s) {
  int r = run_gemm(N, K, B, ColMajorA{dZ, N}, RowMajorB{X, K}, StoreEp{dW, K}, ws, true, pr, s);
  if (r) return r;
  column_sums_kernel<<<grid_for(N), 256, 0, s>>>(B, N, dZ, db);
  return static_cast<int>(cudaGetLastError());
}

size_t conv_pack_bytes(int Ci, int Co) {
  const size_t fwd = static_cast<size_t>((Co + TC_BM - 1) / TC_BM) * ((Ci + CV_CK - 1) / CV_CK) * 3 * CV_TAP;
  const size_t bwd = static_cast<size_t>((Ci + TC_BM - 1) / TC_BM) * ((Co + CV_CK - 1) / CV_CK) * 3 * CV_TAP;
  return fwd > bwd ? fwd : bwd;
}

int conv_forward(int B, int Ci, int Co, int Lin, int up, const float* X, const bf16* W, const float* bias,
                 float* pre, float* out, const Products& pr, cudaStream_t s) {
  const int L = Lin * up;
  if (pr.kind == 1) {
    if (B <= 0) return 0;
    if (!pr.err || !pr.pack || conv_pack_bytes(Ci, Co) > pr.pack_bytes) return static_cast<int>(cudaErrorInvalidValue);
    const int nq = (Ci + CV_CK - 1) / CV_CK;
    const size_t total = static_cast<size_t>((Co + TC_BM - 1) / TC_BM) * nq * 3 * (CV_TAP / 2);
    pack_conv_weights_kernel<<<grid_for(total), 256, 0, s>>>(Co, Ci, nq, total, W, pr.pack);
    const long long tiles =
        static_cast<long long>((Co + TC_BM - 1) / TC_BM) * ((L + TC_BN - 1) / TC_BN) * static_cast<long long>(B);
    if (tiles > 0x7FFFFFFFLL) return static_cast<int>(cudaErrorInvalidValue);
    const cudaError_t e = cudaFuncSetAttribute(tc_conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, CV_SMEM);
    if (e != cudaSuccess) return static_cast<int>(e);
    tc_conv_kernel<<<static_cast<unsigned>(tiles), TC_THREADS, CV_SMEM, s>>>(Ci, Co, Lin, L, up >> 1, X, pr.pack, bias,
                                                                            pre, out, pr.err, pr.stall_test);
    return static_cast<int>(cudaGetLastError());
  }
  return run_gemm(Co, B * L, Ci * 3, ConvWeightA{W, Ci * 3}, ConvInputB{X, Ci, Lin, L, up >> 1, div_by(L)},
                  ConvEp{pre, out, bias, Co, L, div_by(L)}, nullptr, false, pr, s);
}

// db[o] = sum over samples and times of dZ[b][o][t]: P sample slices a channel (P Co <= the
// scratch pr.red holds), parts added in slice order
int channel_sums(int B, int Co, int L, const float* dZ, float* db, const Products& pr, cudaStream_t s) {
  int P = pr.red ? static_cast<int>(pr.red_floats / static_cast<size_t>(Co)) : 1;
  if (P > (608 + Co - 1) / Co) P = (608 + Co - 1) / Co;
  if (P > B) P = B;
  if (P < 1) P = 1;
  float* part = pr.red ? pr.red : db;
  channel_partials_kernel<<<dim3(Co, P), 256, 0, s>>>(B, Co, L, P, dZ, part);
  if (pr.red) channel_finish_kernel<<<(Co + 255) / 256, 256, 0, s>>>(Co, P, part, db);
  return static_cast<int>(cudaGetLastError());
}

int conv_backward_data(int B, int Ci, int Co, int Lin, int up, const float* dZ, const bf16* W, float* dX,
                       const Products& pr, cudaStream_t s) {
  const int L = Lin * up;
  if (pr.kind == 1) {
    if (B <= 0) return 0;
    if (!pr.err || !pr.pack || conv_pack_bytes(Ci, Co) > pr.pack_bytes || (up != 1 && up != 2))
      return static_cast<int>(cudaErrorInvalidValue);
    const int nq = (Co + CV_CK - 1) / CV_CK;
    const size_t total = static_cast<size_t>((Ci + TC_BM - 1) / TC_BM) * nq * 3 * (CV_TAP / 2);
    pack_conv_weights_t_kernel<<<grid_for(total), 256, 0, s>>>(Co, Ci, nq, total, W, pr.pack);
    const long long tiles =
        static_cast<long long>((Ci + TC_BM - 1) / TC_BM) * ((Lin + TC_BN - 1) / TC_BN) * static_cast<long long>(B);
    if (tiles > 0x7FFFFFFFLL) return static_cast<int>(cudaErrorInvalidValue);
    cudaError_t e;
    if (up == 1) {
      e = cudaFuncSetAttribute(tc_conv_dgrad_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, Dgrad<1>::kSmem);
      if (e != cudaSuccess) return static_cast<int>(e);
      tc_conv_dgrad_kernel<1><<<static_cast<unsigned>(tiles), TC_THREADS, Dgrad<1>::kSmem, s>>>(
          Ci, Co, Lin, L, dZ, pr.pack, dX, pr.err, pr.stall_test);
    } else {
      e = cudaFuncSetAttribute(tc_conv_dgrad_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, Dgrad<2>::kSmem);
      if (e != cudaSuccess) return static_cast<int>(e);
      tc_conv_dgrad_kernel<2><<<static_cast<unsigned>(tiles), TC_THREADS, Dgrad<2>::kSmem, s>>>(
          Ci, Co, Lin, L, dZ, pr.pack, dX, pr.err, pr.stall_test);
    }
    return static_cast<int>(cudaGetLastError());
  }
  return run_gemm(Ci, B * Lin, Co * 3 * up, ConvWeightTA{W, Ci, up >> 1},
                  ConvGradB{dZ, Co, Lin, L, up >> 1, div_by(Lin)}, ConvDataEp{dX, Ci, Lin, div_by(Lin)}, nullptr,
                  false, pr, s);
}

int conv_backward_weight(int B, int Ci, int Co, int Lin, int up, const float* dZ, const float* X, float* dW,
                         float* db, float* ws, const Products& pr, cudaStream_t s) {
  const int L = Lin * up;
  int r = 0;
  if (pr.kind == 1 && B > 0) {
    if (!pr.err) return static_cast<int>(cudaErrorInvalidValue);
    int S = ws ? splits_for(Co, Ci * 3, B * L, 1) : 1;
    if (S > B) S = B;
    const size_t mn = static_cast<size_t>(Co) * Ci * 3;
    if (S > 1 && static_cast<size_t>(S) * mn > pr.ws_floats) S = static_cast<int>(std::max<size_t>(1, pr.ws_floats / mn));
    const long long tiles =
        static_cast<long long>((Co + TC_BM - 1) / TC_BM) * 3 * ((Ci + TC_BN - 1) / TC_BN) * static_cast<long long>(S);
    if (tiles > 0x7FFFFFFFLL) return static_cast<int>(cudaErrorInvalidValue);
    const cudaError_t e =
        cudaFuncSetAttribute(tc_conv_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return static_cast<int>(e);
    tc_conv_wgrad_kernel<<<static_cast<unsigned>(tiles), TC_THREADS, TC_SMEM, s>>>(
        B, Ci, Co, Lin, L, up >> 1, S, dZ, X, S > 1 ? ws : dW, pr.err, pr.stall_test);
    if (S > 1)
      splitk_finalize_kernel<<<grid_for(static_cast<size_t>(Co) * Ci * 3), 256, 0, s>>>(Co, Ci * 3, S, ws,
                                                                                        StoreEp{dW, Ci * 3});
    r = static_cast<int>(cudaGetLastError());
  } else {
    r = run_gemm(Co, Ci * 3, B * L, ConvGradA{dZ, Co, L, div_by(L)}, ConvInputWB{X, Ci, Lin, L, up >> 1, div_by(L)},
                 StoreEp{dW, Ci * 3}, ws, true, pr, s);
  }
  if (r) return r;
  return channel_sums(B, Co, L, dZ, db, pr, s);
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
  if (B <= 0) return 0;
  const size_t CL = static_cast<size_t>(C) * L;
  const int gx = static_cast<int>(std::min<size_t>((CL + 255) / 256, 64));
  contract_forward_kernel<<<dim3(gx, std::min(B, 65535)), 256, 0, s>>>(B, K, C, L, in_dim, in_dim - K, x, D, y);
  return static_cast<int>(cudaGetLastError());
}

int contract_backward(int B, int K, int C, int L, int in_dim, const float* x, const float* dy, float* dD,
                      cudaStream_t s) {
  if (B <= 0) return 0;
  const size_t CL = static_cast<size_t>(C) * L;
  const int gx = static_cast<int>(std::min<size_t>((CL + 255) / 256, 64));
  contract_backward_kernel<<<dim3(gx, std::min(B * K, 65535)), 256, 0, s>>>(B, K, C, L, in_dim, in_dim - K, x, dy,
                                                                           dD);
  return static_cast<int>(cudaGetLastError());
}

int to_bf16(size_t n, const float* p, bf16* pb, cudaStream_t s) {
  to_bf16_kernel<<<grid_for(n), 256, 0, s>>>(n, p, pb);
  return static_cast<int>(cudaGetLastError());
}

}  // namespace sgk
