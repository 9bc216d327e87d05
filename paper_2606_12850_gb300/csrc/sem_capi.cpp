// C ABI of libsemgb (declared in include/sem.h): context, set-up, device buffers, the
// time-step sequence and its CUDA-graph capture.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <set>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "sem.h"
#include "sem_sources.h"
#include "sem_internal.h"

using namespace semgb;

namespace {

constexpr int kStepsPerGraph = 10;
thread_local std::string g_err;  // message of the last failed context-free call

}  // namespace

struct sem_ctx {
  int ngll = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t aux = nullptr;      // the adjoint's sensitivity terms run here, one step behind
  cudaEvent_t ev_sweep[2] = {nullptr, nullptr}, ev_sens[2] = {nullptr, nullptr};
  std::string err;

  std::vector<double> xi, w, hprime;

  // mesh (host)
  bool have_mesh = false, have_mat = false, have_dt = false;
  int nspec = 0, nglob = 0, ncolors = 0;
  std::vector<int32_t> ibool;       // caller order
  std::vector<int> order;           // record slot -> caller element (patch sweep order)
  std::vector<int> pos_of;          // caller element -> record slot
  std::vector<int> color_count;     // elements per colour
  std::vector<int> sweep_off;       // element-list ranges, one per (slab, colour) launch
  std::vector<int> pcolor_off;      // patch ranges, one per patch colour
  int npatch = 0, pmax_nodes = 0, ptables = 0;
  int stall_test = 0;               // SEM_OPT_SWEEP_STALL_TEST (one-shot)
  int fuse_newmark = 2;             // SEM_OPT_FUSED_NEWMARK: Newmark update in the patch sweep
                                    // (1 on, 0 off, 2 on for a single shot)
  int shot_pairs = 1;               // SEM_OPT_SHOT_PAIRS: patch CTAs per shot pair (1) or shot (0)
  PatchShape shape_opt{0, 0, 0};    // SEM_OPT_PATCH_SHAPE for the next sem_set_mesh (0: the order's)
  PatchShape shape{0, 0, 0};        // the bricks of the current mesh
  std::vector<PatchDesc> pdesc;     // host copy of the patch descriptors
  std::vector<int> last_patch;      // internal node -> the patch that touches it last
  int assembly = 0;                 // SEM_OPT_ASSEMBLY: 0 patches, one launch per colour,
                                    // 1 elements, 2 persistent patch sweep, 3 atomic ablation
  int slabs = 1;                    // spatial slabs of the sweep order
  int slabs_opt = 0;                // requested slab count (0 = automatic)
  std::vector<float> rec;           // colour-sorted element records (host copy)
  std::vector<double> dxmin;        // per caller element
  std::vector<double> node_xyz;     // [nglob][3], caller node order
  std::vector<int> node_new;        // caller node -> internal node
  std::vector<int> perm;            // internal node -> caller node
  std::vector<double> ctrl;         // [nspec][8][3] corner vertices (caller order)
  std::vector<double> vpmax;        // per caller element
  double dt = 0.0;

  // device
  float* d_rec = nullptr;
  int* d_order = nullptr;         // record slot -> caller element
  int* d_elist = nullptr;         // record slots in element colour order
  int* d_perm = nullptr;          // internal node -> caller node
  int* d_node_new = nullptr;      // caller node -> internal node
  PatchDesc* d_pdesc = nullptr;   // patches in sweep order
  uint16_t* d_pslots = nullptr;   // patch tables: shared patch node -> local points meeting there
  uint16_t* d_pwords = nullptr;   // patch tables: shared patch node -> its first point's ibool word
  int* d_pcolor_end = nullptr;    // per patch colour, the end of its patch range
  SweepSync* d_sync = nullptr;    // counters of the persistent sweep
  PatchSrc* d_psrc = nullptr;     // point sources by the patch that touches their node last
  float *d_u = nullptr, *d_v = nullptr, *d_a = nullptr, *d_minv = nullptr;
  float* d_f = nullptr;           // scratch force buffer for sem_energy
  float *d_lam = nullptr, *d_lam_old = nullptr, *d_lamF = nullptr;  // adjoint fields [nglob][4]
  double* d_grad = nullptr;       // [3][nlocal] sensitivities (rho, kappa, mu), record order
  float* d_grad32 = nullptr;      // [3][nlocal] float32 partial sums, flushed into d_grad
  int since_flush = 0;            // adjoint steps accumulated in d_grad32
  int node_order = 0;             // SEM_OPT_NODE_ORDER: device state arrays in caller (0) or internal (1) order
  PatchRecv* d_precv = nullptr;   // receivers by the patch that touches their node last
  int* d_precv_range = nullptr;   // [npatch][2] first, count into d_precv
  int* d_rnode = nullptr;         // distinct receiver nodes (internal ids)
  int* d_roff = nullptr;          // their receivers: d_rlist[d_roff[t] .. d_roff[t+1])
  int* d_rlist = nullptr;
  int nrnodes = 0;
  bool adjoint = false;
  double* d_partials = nullptr;   // scratch partial sums for sem_energy
  DevCtl* d_ctl = nullptr;
  int* d_src_node = nullptr;
  int* d_src_shot = nullptr;
  double* d_src_force = nullptr;
  int nsrc = 0;
  int shots = 1;  // wavefields [nglob][shots][kNodeStride]
  double f0 = 0.0, t0 = 0.0;
  int* d_rec_node = nullptr;
  int nrec = 0;
  size_t dev_bytes = 0;

  // time stepping
  bool pending = false;  // a_raw holds forces and v the half-step velocity
  long long steps = 0;
  cudaGraphExec_t graph = nullptr;
  bool graph_valid = false;
  bool graph_fused = false;           // the graph holds steps of the fused sweep
  cudaGraphExec_t graph_snap = nullptr;  // fused steps that also store the displacement
  cudaGraphExec_t graph_adj = nullptr;   // adjoint steps indexed by the device counter
  const float* graph_adj_lam = nullptr;  // d_lam when graph_adj was captured
  bool graph_adj_G = false;              // graph_adj injects receiver residuals
  unsigned long long generation = 0;  // bumped whenever launches captured in graphs go stale
  int variant = 0;                    // force-kernel contraction form (sem_autotune)
};

namespace {

int fail(sem_ctx* c, int code, const std::string& msg) {
  if (c)
    c->err = msg;
  else
    g_err = msg;
  return code;
}

int cuda_fail(sem_ctx* c, cudaError_t e, const char* what) {
  return fail(c, SEM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define SEM_CUDA(c, call)                                   \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail((c), e_, #call); \
  } while (0)

#define SEM_LAUNCH(c, call)                                                                    \
  do {                                                                                         \
    int r_ = (call);                                                                           \
    if (r_ != 0) return cuda_fail((c), static_cast<cudaError_t>(r_), #call);                   \
  } while (0)

template <typename T>
int dev_alloc(sem_ctx* c, T** p, size_t count) {
  if (*p) {
    cudaFree(*p);
    *p = nullptr;
  }
  if (count == 0) return SEM_OK;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess) return fail(c, SEM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  *p = static_cast<T*>(q);
  c->dev_bytes += count * sizeof(T);
  return SEM_OK;
}

void free_device(sem_ctx* c) {
  void* ptrs[] = {c->d_rec, c->d_order, c->d_elist, c->d_perm, c->d_node_new, c->d_pdesc, c->d_pslots, c->d_pwords, c->d_pcolor_end, c->d_sync, c->d_psrc, c->d_u, c->d_v,
                  c->d_a, c->d_minv, c->d_f, c->d_partials, c->d_lam, c->d_lam_old, c->d_lamF, c->d_grad,
                  c->d_grad32, c->d_precv, c->d_precv_range, c->d_rnode, c->d_roff, c->d_rlist,
                  c->d_ctl, c->d_src_node, c->d_src_shot, c->d_src_force, c->d_rec_node};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  c->d_rec = nullptr;
  c->d_order = nullptr;
  c->d_elist = nullptr;
  c->d_perm = nullptr;
  c->d_node_new = nullptr;
  c->d_pdesc = nullptr;
  c->d_pslots = nullptr;
  c->d_pwords = nullptr;
  c->d_pcolor_end = nullptr;
  c->d_sync = nullptr;
  c->d_psrc = nullptr;
  c->d_u = c->d_v = c->d_a = c->d_minv = c->d_f = nullptr;
  c->d_lam = c->d_lam_old = c->d_lamF = nullptr;
  c->d_grad = nullptr;
  c->d_grad32 = nullptr;
  c->d_rnode = c->d_roff = c->d_rlist = nullptr;
  c->d_precv = nullptr;
  c->d_precv_range = nullptr;
  c->nrnodes = 0;
  c->adjoint = false;
  c->d_partials = nullptr;
  c->d_ctl = nullptr;
  c->d_src_node = nullptr;
  c->d_src_shot = nullptr;
  c->d_src_force = nullptr;
  c->d_rec_node = nullptr;
  c->dev_bytes = 0;
}

void drop_graph(sem_ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
  if (c->graph_snap) cudaGraphExecDestroy(c->graph_snap);
  c->graph_snap = nullptr;
  if (c->graph_adj) cudaGraphExecDestroy(c->graph_adj);
  c->graph_adj = nullptr;
  c->graph_valid = false;
  ++c->generation;
}

DevProblem problem(const sem_ctx* c) {
  DevProblem p{};
  p.ngll = c->ngll;
  p.nspec = c->nspec;
  p.nglob = c->nglob;
  p.rec = c->d_rec;
  p.u = c->d_u;
  p.v = c->d_v;
  p.a = c->d_a;
  p.minv = c->d_minv;
  p.ctl = c->d_ctl;
  p.nsrc = c->nsrc;
  p.src_node = c->d_src_node;
  p.src_shot = c->d_src_shot;
  p.shots = c->shots;
  p.src_force = c->d_src_force;
  p.f0 = c->f0;
  p.t0 = c->t0;
  p.nrec = c->nrec;
  p.rec_node = c->d_rec_node;
  p.dt = c->dt;
  return p;
}

int set_device(sem_ctx* c) {
  SEM_CUDA(c, cudaSetDevice(c->device));
  return SEM_OK;
}

// f = -K u over all colours (Sec. IV-C: colour by colour, no atomics). On the context's own
// fields the patch kernel takes the patch colours in order (one launch per colour, one CTA
// per patch and shot; patches of a colour share no node). Otherwise (caller arrays, or
// SEM_OPT_ASSEMBLY = 1) the element kernel walks the element list slab by slab and, inside a
// slab, colour by colour: a launch holds elements of one colour only.
// With nm (mode 1 or 2; only on the per-colour patch path, see fused_sweep) the sweep also
// runs the Newmark update of every node at the patch that touches it last.
int forces_all_colors(sem_ctx* c, const float* u, float* f, int node_stride, int shots,
                      const SweepNewmark* nm = nullptr) {
  if ((c->assembly == 0 || c->assembly == 2) && node_stride == kNodeStride && c->npatch > 0) {
    PatchLaunch P{};
    if (nm) P.nm = *nm;
    P.rec = c->d_rec;
    P.desc = c->d_pdesc;
    P.slots = c->d_pslots;
    P.words = c->d_pwords;
    P.u = u;
    P.f = f;
    P.variant = c->variant;
    P.shots = shots;
    P.pairs = c->shot_pairs;
    const int npc = static_cast<int>(c->pcolor_off.size()) - 1;
    if (c->assembly == 2 && shots == 1 && npc <= kMaxSweepColors && P.nm.mode == 0) {
      P.sync = c->d_sync;
      P.color_end = c->d_pcolor_end;
      P.npatch = c->npatch;
      P.ncolors = npc;
      P.stall = c->stall_test;
      c->stall_test = 0;
      SEM_LAUNCH(c, launch_patch_forces(c->ngll, P, c->stream));
      return SEM_OK;
    }
    for (size_t k = 0; k + 1 < c->pcolor_off.size(); ++k) {
      P.p0 = c->pcolor_off[k];
      P.p1 = c->pcolor_off[k + 1];
      SEM_LAUNCH(c, launch_patch_forces(c->ngll, P, c->stream));
    }
    return SEM_OK;
  }
  ForceLaunch L{};
  L.rec = c->d_rec;
  L.elist = c->d_elist;
  L.perm = c->d_perm;
  if (c->assembly == 3 && node_stride == kNodeStride && shots == 1) {  // colouring ablation
    L.u = u;
    L.f = f;
    L.node_stride = node_stride;
    L.shots = 1;
    L.variant = c->variant;
    L.atomic = 1;
    L.e0 = 0;
    L.e1 = c->nspec;
    SEM_CUDA(c, cudaMemsetAsync(f, 0, kNodeStride * static_cast<size_t>(c->nglob) * sizeof(float), c->stream));
    SEM_LAUNCH(c, launch_forces(c->ngll, L, c->stream));
    return SEM_OK;
  }
  L.u = u;
  L.f = f;
  L.node_stride = node_stride;
  L.shots = shots;
  L.variant = c->variant;
  for (size_t k = 0; k + 1 < c->sweep_off.size(); ++k) {
    L.e0 = c->sweep_off[k];
    L.e1 = c->sweep_off[k + 1];
    SEM_LAUNCH(c, launch_forces(c->ngll, L, c->stream));
  }
  return SEM_OK;
}

// Whether time steps run the fused sweep: the per-colour patch sweep (SEM_OPT_ASSEMBLY 0)
// with SEM_OPT_FUSED_NEWMARK on (by default for a single shot only: with several shots the
// separate pass over the [nglob][S][4] fields is faster on GB300, 48^3 at NGLL 5 with 32
// shots: 11.8 ms per step against 13.1 ms).
bool fused_sweep(const sem_ctx* c) {
  return (c->fuse_newmark == 1 || (c->fuse_newmark == 2 && c->shots == 1)) && c->assembly == 0 && c->npatch > 0;
}

SweepNewmark sweep_newmark(const sem_ctx* c, int mode) {
  SweepNewmark nm{};
  nm.mode = mode;
  nm.u = c->d_u;
  nm.v = c->d_v;
  nm.a = c->d_a;
  nm.minv = c->d_minv;
  nm.src = c->d_psrc;
  nm.step = &c->d_ctl->step;
  nm.f0 = c->f0;
  nm.t0 = c->t0;
  nm.dtd = c->dt;
  nm.dt = static_cast<float>(c->dt);
  nm.hdt = static_cast<float>(0.5 * c->dt);
  nm.hdt2 = static_cast<float>(0.5 * c->dt * c->dt);
  return nm;
}

// One step of the fused sweep from u_{n+1} (predicted) and the half-step velocity: the
// receivers sample u_{n+1} and the step counter advances to n+1, then the sweep assembles
// the forces and, at each node's last touch, adds the step's point sources and runs the
// corrector of step n fused with the predictor of step n+1 (mode 1), or the corrector alone
// (mode 2, the last step of a run: the state is complete afterwards).
int enqueue_fused_step(sem_ctx* c, int mode) {
  DevProblem p = problem(c);
  p.nsrc = 0;  // the sweep adds the sources
  SEM_LAUNCH(c, launch_sources_record(p, c->stream));
  const SweepNewmark nm = sweep_newmark(c, mode);
  return forces_all_colors(c, c->d_u, c->d_a, kNodeStride, c->shots, &nm);
}

// One time step in the "pending" representation (a holds M a_raw of the previous step, v
// the half-step velocity): corrector(n-1) fused with predictor(n), forces, sources,
// receivers. The first step from a complete state uses the predictor alone.
int enqueue_step(sem_ctx* c, bool first) {
  const DevProblem p = problem(c);
  if (first)
    SEM_LAUNCH(c, launch_predictor(p, c->stream));
  else
    SEM_LAUNCH(c, launch_fused_newmark(p, c->stream));
  int r = forces_all_colors(c, c->d_u, c->d_a, kNodeStride, c->shots);
  if (r) return r;
  SEM_LAUNCH(c, launch_sources_record(p, c->stream));
  return SEM_OK;
}
int enqueue_pending_step(sem_ctx* c) { return enqueue_step(c, false); }
int enqueue_first_step(sem_ctx* c) { return enqueue_step(c, true); }

int build_graph(sem_ctx* c) {
  drop_graph(c);
  cudaGraph_t g = nullptr;
  const bool fused = fused_sweep(c);
  SEM_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  int r = SEM_OK;
  for (int s = 0; s < kStepsPerGraph && r == SEM_OK; ++s) r = fused ? enqueue_fused_step(c, 1) : enqueue_pending_step(c);
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  if (r != SEM_OK) {
    if (g) cudaGraphDestroy(g);
    return r;
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
  c->graph_valid = true;
  c->graph_fused = fused;
  return SEM_OK;
}

int finish_state(sem_ctx* c);

// nsteps steps of the fused sweep from a complete state, which they leave complete: the
// predictor, nsteps - 1 steps of mode 1 (in graphs of kStepsPerGraph steps), one of mode 2.
int advance_fused(sem_ctx* c, int nsteps) {
  int r = finish_state(c);  // a pending state left by steps of another assembly
  if (r) return r;
  SEM_LAUNCH(c, launch_predictor(problem(c), c->stream));
  int left = nsteps - 1;
  if (left >= kStepsPerGraph && (!c->graph_valid || !c->graph_fused))
    if ((r = build_graph(c))) return r;
  for (; left >= kStepsPerGraph; left -= kStepsPerGraph) SEM_CUDA(c, cudaGraphLaunch(c->graph, c->stream));
  for (; left > 0; --left)
    if ((r = enqueue_fused_step(c, 1))) return r;
  return enqueue_fused_step(c, 2);
}

int check_ready(sem_ctx* c) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (!c->have_mesh) return fail(c, SEM_ESTATE, "sem_set_mesh has not been called");
  if (!c->have_mat) return fail(c, SEM_ESTATE, "sem_set_material has not been called");
  if (!c->have_dt) return fail(c, SEM_ESTATE, "sem_set_dt has not been called");
  return SEM_OK;
}

// nsteps time steps; fused false keeps the separate Newmark passes (the state is then left
// pending), as the group step needs.
int advance(sem_ctx* c, int nsteps, float* seis_dev, bool fused = true) {
  int r = check_ready(c);
  if (r) return r;
  if (nsteps < 0) return fail(c, SEM_EINVAL, "nsteps must be >= 0");
  if ((r = set_device(c))) return r;
  SEM_LAUNCH(c, launch_set_ctl(c->d_ctl, c->steps, seis_dev ? nsteps : 0, seis_dev, c->stream));
  if (fused && fused_sweep(c)) {
    if (nsteps > 0 && (r = advance_fused(c, nsteps))) return r;
    c->steps += nsteps;
    return SEM_OK;
  }
  int left = nsteps;
  if (left > 0 && !c->pending) {
    if ((r = enqueue_first_step(c))) return r;
    c->pending = true;
    --left;
  }
  if (left >= kStepsPerGraph && (!c->graph_valid || c->graph_fused))
    if ((r = build_graph(c))) return r;
  while (left >= kStepsPerGraph) {
    SEM_CUDA(c, cudaGraphLaunch(c->graph, c->stream));
    left -= kStepsPerGraph;
  }
  while (left > 0) {
    if ((r = enqueue_pending_step(c))) return r;
    --left;
  }
  c->steps += nsteps;
  return SEM_OK;
}

// After the stream is idle: SEM_ETIMEOUT (and the flag cleared) if a wait of the persistent
// sweep gave up since the last check.
int check_sweep_timeout(sem_ctx* c) {
  if (!c->d_sync) return SEM_OK;
  int err = 0;
  SEM_CUDA(c, cudaMemcpyAsync(&err, &c->d_sync->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  SEM_CUDA(c, cudaStreamSynchronize(c->stream));
  if (!err) return SEM_OK;
  SEM_CUDA(c, cudaMemsetAsync(&c->d_sync->err, 0, sizeof(int), c->stream));
  SEM_CUDA(c, cudaStreamSynchronize(c->stream));
  return fail(c, SEM_ETIMEOUT, "a bounded wait of the force sweep gave up (the forces of that sweep are incomplete)");
}

// The float32 sensitivity partials of the steps since the last flush, added into the float64
// accumulators (every kFlushEvery adjoint steps, at the end of a segment, and before the
// gradients are read: a float32 sum of a few dozen terms keeps about six digits).
constexpr int kFlushEvery = 60;  // a multiple of kStepsPerGraph
int flush_gradients(sem_ctx* c) {
  if (!c->since_flush) return SEM_OK;
  const long long n = 3ll * c->nspec * c->ngll * c->ngll * c->ngll;
  SEM_LAUNCH(c, launch_flush_partials(c->d_grad32, c->d_grad, n, c->stream));
  c->since_flush = 0;
  return SEM_OK;
}

// Completes a pending state: a = M^-1 a_raw, v = v_half + dt/2 a.
int finish_state(sem_ctx* c) {
  if (!c->pending) return SEM_OK;
  SEM_LAUNCH(c, launch_corrector(problem(c), c->stream));
  c->pending = false;
  return SEM_OK;
}


}  // namespace

namespace semgb {

int ctx_view(sem_ctx* c, CtxView* out) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (!c->have_mat) return fail(c, SEM_ESTATE, "sem_set_material has not been called");
  out->device = c->device;
  out->stream = c->stream;
  out->nglob = c->nglob;
  out->minv = c->d_minv;
  out->node_new = c->d_node_new;
  return SEM_OK;
}

int ctx_fail(sem_ctx* c, int code, const char* message) { return fail(c, code, message); }

}  // namespace semgb

extern "C" {

int sem_version(void) { return 100; }

int sem_gll(int ngll, double* xi, double* w, double* hprime) {
  std::string err;
  if (gll_basis(ngll, xi, w, hprime, &err)) return fail(nullptr, SEM_EINVAL, err);
  return SEM_OK;
}

int sem_color_elements(int nspec, int ngll, int nglob, const int32_t* ibool, int32_t* color, int* ncolors) {
  if (nspec < 1 || nglob < 1 || !ibool || !color || !ncolors || ngll < kMinNgll || ngll > kMaxNgll)
    return fail(nullptr, SEM_EINVAL, "sem_color_elements: bad arguments");
  const size_t nloc = static_cast<size_t>(nspec) * ngll * ngll * ngll;
  for (size_t q = 0; q < nloc; ++q)
    if (ibool[q] < 0 || ibool[q] >= nglob) return fail(nullptr, SEM_EINVAL, "ibool entry out of range");
  std::vector<int32_t> col;
  std::string err;
  if (color_elements(nspec, ngll, nglob, ibool, &col, ncolors, &err)) return fail(nullptr, SEM_EINVAL, err);
  std::memcpy(color, col.data(), sizeof(int32_t) * nspec);
  return SEM_OK;
}

int sem_patch_plan(int ngll, int nspec, int nglob, const int32_t* ibool, int32_t* patch_of, int32_t* color_of,
                   int64_t* info) {
  if (nspec < 1 || nglob < 1 || !ibool || ngll < kMinNgll || ngll > kMaxNgll)
    return fail(nullptr, SEM_EINVAL, "sem_patch_plan: bad arguments");
  const int np = ngll * ngll * ngll;
  const size_t nloc = static_cast<size_t>(nspec) * np;
  for (size_t q = 0; q < nloc; ++q)
    if (ibool[q] < 0 || ibool[q] >= nglob) return fail(nullptr, SEM_EINVAL, "ibool entry out of range");
  PatchShape shape;
  PatchPlan plan;
  std::string err;
  if (patch_shape(ngll, &shape) || build_patches(nspec, ngll, nglob, ibool, shape, &plan, &err))
    return fail(nullptr, SEM_EINVAL, "sem_patch_plan: " + err);
  for (int c = 0; c < plan.ncolors; ++c)
    for (int P = plan.color_off[c]; P < plan.color_off[c + 1]; ++P) {
      if (color_of) color_of[P] = c;
      if (patch_of)
        for (int s = plan.patch_off[P]; s < plan.patch_off[P + 1]; ++s) patch_of[plan.elem[s]] = P;
    }
  if (info) {
    info[0] = plan.npatch;
    info[1] = plan.ncolors;
    info[2] = plan.max_nodes;
    info[3] = static_cast<int64_t>(plan.tab_nelem.size());
    info[4] = shape.bx;
    info[5] = shape.by;
    info[6] = shape.bz;
  }
  return SEM_OK;
}

int sem_geometry(int ngll, int nspec, const double* ctrl, double* xyz, double* dxi_dx, double* jac) {
  if (nspec < 1 || !ctrl || ngll < kMinNgll || ngll > kMaxNgll)
    return fail(nullptr, SEM_EINVAL, "sem_geometry: bad arguments");
  for (size_t q = 0; q < static_cast<size_t>(nspec) * 24; ++q)
    if (!std::isfinite(ctrl[q])) return fail(nullptr, SEM_EINVAL, "non-finite corner coordinate");
  std::vector<double> xi(ngll), w(ngll), h(static_cast<size_t>(ngll) * ngll);
  std::string err;
  if (gll_basis(ngll, xi.data(), w.data(), h.data(), &err)) return fail(nullptr, SEM_EINVAL, err);
  const size_t np = static_cast<size_t>(ngll) * ngll * ngll;
  std::vector<double> X(3 * np), G(9 * np), J(np);
  int bad = -1;
  for (int e = 0; e < nspec; ++e) {
    const size_t e0 = static_cast<size_t>(e) * np;
    if (!element_geometry(ngll, xi.data(), h.data(), ctrl + 24 * static_cast<size_t>(e), X.data(), G.data(),
                          J.data()) &&
        bad < 0)
      bad = e;
    if (xyz) std::memcpy(xyz + 3 * e0, X.data(), sizeof(double) * 3 * np);
    if (dxi_dx) std::memcpy(dxi_dx + 9 * e0, G.data(), sizeof(double) * 9 * np);
    if (jac) std::memcpy(jac + e0, J.data(), sizeof(double) * np);
  }
  if (bad >= 0)
    return fail(nullptr, SEM_EINVAL, "element " + std::to_string(bad) + " has a Jacobian determinant <= 0");
  return SEM_OK;
}

int sem_geometry_points(int ngll, int nspec, const double* xyz, double* dxi_dx, double* jac) {
  if (nspec < 1 || !xyz || ngll < kMinNgll || ngll > kMaxNgll)
    return fail(nullptr, SEM_EINVAL, "sem_geometry_points: bad arguments");
  const size_t np = static_cast<size_t>(ngll) * ngll * ngll;
  for (size_t q = 0; q < 3 * np * nspec; ++q)
    if (!std::isfinite(xyz[q])) return fail(nullptr, SEM_EINVAL, "non-finite point coordinate");
  std::vector<double> xi(ngll), w(ngll), h(static_cast<size_t>(ngll) * ngll);
  std::string err;
  if (gll_basis(ngll, xi.data(), w.data(), h.data(), &err)) return fail(nullptr, SEM_EINVAL, err);
  std::vector<double> G(9 * np), J(np);
  int bad = -1;
  for (int e = 0; e < nspec; ++e) {
    const size_t e0 = static_cast<size_t>(e) * np;
    if (!geometry_from_positions(ngll, h.data(), xyz + 3 * e0, G.data(), J.data()) && bad < 0) bad = e;
    if (dxi_dx) std::memcpy(dxi_dx + 9 * e0, G.data(), sizeof(double) * 9 * np);
    if (jac) std::memcpy(jac + e0, J.data(), sizeof(double) * np);
  }
  if (bad >= 0)
    return fail(nullptr, SEM_EINVAL, "element " + std::to_string(bad) + " has a Jacobian determinant <= 0");
  return SEM_OK;
}

int sem_locate_points(int nspec, const double* ctrl, int npts, const double* xyz, int32_t* elem_out,
                      double* ref_out) {
  if (nspec < 1 || npts < 0 || !ctrl || (npts > 0 && (!xyz || !elem_out)))
    return fail(nullptr, SEM_EINVAL, "sem_locate_points: bad arguments");
  for (size_t q = 0; q < static_cast<size_t>(nspec) * 24; ++q)
    if (!std::isfinite(ctrl[q])) return fail(nullptr, SEM_EINVAL, "non-finite corner coordinate");
  for (size_t q = 0; q < static_cast<size_t>(npts) * 3; ++q)
    if (!std::isfinite(xyz[q])) return fail(nullptr, SEM_EINVAL, "non-finite point coordinate");
  std::vector<double> ref(3 * static_cast<size_t>(npts));
  locate_points(nspec, ctrl, npts, xyz, elem_out, ref.data());
  if (ref_out) std::copy(ref.begin(), ref.end(), ref_out);
  return SEM_OK;
}

int sem_point_source_forces(int ngll, const double* ctrl_e, const double* ref, const double* force,
                            const double* moment, double* f_out) {
  if (ngll < kMinNgll || ngll > kMaxNgll || !ctrl_e || !ref || !f_out || (!force) == (!moment))
    return fail(nullptr, SEM_EINVAL, "sem_point_source_forces: bad arguments (give exactly one of force, moment)");
  for (int q = 0; q < 24; ++q)
    if (!std::isfinite(ctrl_e[q])) return fail(nullptr, SEM_EINVAL, "non-finite corner coordinate");
  for (int q = 0; q < 3; ++q)
    if (!(std::fabs(ref[q]) <= 1.0)) return fail(nullptr, SEM_EINVAL, "reference coordinate outside [-1, 1]");
  const double* v = force ? force : moment;
  for (int q = 0; q < (force ? 3 : 6); ++q)
    if (!std::isfinite(v[q])) return fail(nullptr, SEM_EINVAL, "non-finite source value");
  std::vector<double> xi(ngll), w(ngll), h(static_cast<size_t>(ngll) * ngll);
  std::string err;
  if (gll_basis(ngll, xi.data(), w.data(), h.data(), &err)) return fail(nullptr, SEM_EINVAL, err);
  point_source_forces(ngll, xi.data(), h.data(), ctrl_e, ref, force, moment, f_out);
  return SEM_OK;
}

int sem_create(sem_ctx** out, int ngll, int device, void* cuda_stream) {
  if (!out) return fail(nullptr, SEM_EINVAL, "sem_create: out is NULL");
  *out = nullptr;
  if (ngll < kMinNgll || ngll > kMaxNgll) return fail(nullptr, SEM_EINVAL, "ngll must be in [2, 10]");
  sem_ctx* c = new (std::nothrow) sem_ctx();
  if (!c) return fail(nullptr, SEM_ENOMEM, "out of host memory");
  c->ngll = ngll;
  c->device = device;
  c->xi.resize(ngll);
  c->w.resize(ngll);
  c->hprime.resize(ngll * ngll);
  std::string err;
  gll_basis(ngll, c->xi.data(), c->w.data(), c->hprime.data(), &err);
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) {
    if (cuda_stream) {
      c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
      e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
      c->own_stream = (e == cudaSuccess);
    }
  }
  if (e == cudaSuccess) {
    int r = upload_basis(ngll, c->w.data(), c->hprime.data(), c->stream);
    if (r) e = static_cast<cudaError_t>(r);
  }
  if (e == cudaSuccess) {
    void* q = nullptr;
    e = cudaMalloc(&q, sizeof(DevCtl));
    c->d_ctl = static_cast<DevCtl*>(q);
    if (e == cudaSuccess) e = cudaMemset(c->d_ctl, 0, sizeof(DevCtl));
  }
  if (e != cudaSuccess) {
    g_err = std::string("sem_create: ") + cudaGetErrorString(e);
    sem_destroy(c);
    return SEM_ECUDA;
  }
  *out = c;
  return SEM_OK;
}

int sem_destroy(sem_ctx* c) {
  if (!c) return SEM_OK;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graph(c);
  free_device(c);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  if (c->aux) cudaStreamDestroy(c->aux);
  for (int k = 0; k < 2; ++k) {
    if (c->ev_sweep[k]) cudaEventDestroy(c->ev_sweep[k]);
    if (c->ev_sens[k]) cudaEventDestroy(c->ev_sens[k]);
  }
  delete c;
  return SEM_OK;
}

int sem_set_option(sem_ctx* c, int option, long long value) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  switch (option) {
    case SEM_OPT_SWEEP_SLABS:
      if (value < 0 || value > (1 << 20)) return fail(c, SEM_EINVAL, "slab count out of range");
      c->slabs_opt = static_cast<int>(value);
      return SEM_OK;
    case SEM_OPT_CONTRACTION:
      if (value < 0 || value > 2) return fail(c, SEM_EINVAL, "contraction form must be 0, 1 or 2");
      c->variant = static_cast<int>(value);
      drop_graph(c);
      return SEM_OK;
    case SEM_OPT_NODE_ORDER:
      if (value < 0 || value > 1) return fail(c, SEM_EINVAL, "node order must be 0 (caller) or 1 (internal)");
      c->node_order = static_cast<int>(value);
      drop_graph(c);  // the snapshot graph maps nodes in this order
      return SEM_OK;
    case SEM_OPT_SWEEP_STALL_TEST:
      if (value < 0 || value > 1) return fail(c, SEM_EINVAL, "stall test must be 0 or 1");
      c->stall_test = static_cast<int>(value);
      return SEM_OK;
    case SEM_OPT_SHOT_PAIRS:
      if (value < 0 || value > 1) return fail(c, SEM_EINVAL, "shot pairs must be 0 or 1");
      c->shot_pairs = static_cast<int>(value);
      drop_graph(c);
      return SEM_OK;
    case SEM_OPT_PATCH_SHAPE: {
      PatchShape def;
      if (patch_shape(c->ngll, &def)) return fail(c, SEM_EINVAL, "no patch kernel for this order");
      if (value == 0) {
        c->shape_opt = PatchShape{0, 0, 0};
        return SEM_OK;
      }
      const int bx = static_cast<int>(value & 0xFF), by = static_cast<int>((value >> 8) & 0xFF),
                bz = static_cast<int>((value >> 16) & 0xFF);
      if (value < 0 || (value >> 24) != 0 || bx < 1 || by < 1 || bz < 1 || bx * by * bz > def.bx * def.by * def.bz)
        return fail(c, SEM_EINVAL,
                    "patch shape must be bx | by << 8 | bz << 16 with bx, by, bz >= 1 and bx*by*bz <= " +
                        std::to_string(def.bx * def.by * def.bz) + " (the elements a patch CTA holds at this order)");
      c->shape_opt = PatchShape{bx, by, bz};
      return SEM_OK;
    }
    case SEM_OPT_FUSED_NEWMARK:
      if (value < 0 || value > 2) return fail(c, SEM_EINVAL, "fused Newmark must be 0, 1 or 2");
      c->fuse_newmark = static_cast<int>(value);
      drop_graph(c);
      return SEM_OK;
    case SEM_OPT_ASSEMBLY:
      if (value < 0 || value > 3)
        return fail(c, SEM_EINVAL,
                    "assembly must be 0 (patch colours), 1 (elements), 2 (persistent patch sweep) or 3 (atomic "
                    "ablation)");
      c->assembly = static_cast<int>(value);
      drop_graph(c);
      return SEM_OK;
    default:
      return fail(c, SEM_EINVAL, "unknown option " + std::to_string(option));
  }
}

// Mesh set-up shared by sem_set_mesh (per-point positions pts[nspec][np][3]) and
// sem_set_mesh_corners (trilinear corners ctrl[nspec][8][3]); exactly one is non-null.
static int set_mesh_impl(sem_ctx* c, int nspec, int nglob, const int32_t* ibool, const double* ctrl_in,
                         const double* pts) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (nspec < 1 || nglob < 1 || !ibool || (!ctrl_in) == (!pts)) return fail(c, SEM_EINVAL, "sem_set_mesh: bad arguments");
  const int n = c->ngll, np = n * n * n;
  const size_t nloc = static_cast<size_t>(nspec) * np;
  if (nloc > (1ull << 31) - 1 || nglob > kMaxNodes) return fail(c, SEM_EINVAL, "mesh too large for int32 indexing");
  std::vector<char> seen(nglob, 0);
  for (size_t q = 0; q < nloc; ++q) {
    if (ibool[q] < 0 || ibool[q] >= nglob)
      return fail(c, SEM_EINVAL, "ibool entry " + std::to_string(q) + " out of range");
    seen[ibool[q]] = 1;
  }
  for (int g = 0; g < nglob; ++g)
    if (!seen[g]) return fail(c, SEM_EINVAL, "global node " + std::to_string(g) + " is not referenced by ibool");
  // corner vertices: given, or the corner GLL points of the per-point positions (used by
  // point location and by sources between nodes, which take the trilinear map of the
  // corners)
  std::vector<double> corners;
  const double* ctrl = ctrl_in;
  if (pts) {
    for (size_t q = 0; q < 3 * nloc; ++q)
      if (!std::isfinite(pts[q])) return fail(c, SEM_EINVAL, "non-finite point coordinate");
    corners.resize(static_cast<size_t>(nspec) * 24);
    const int N = n - 1;
    for (int e = 0; e < nspec; ++e)
      for (int v = 0; v < 8; ++v) {
        const int p = ((v & 1) ? N : 0) + n * (((v >> 1) & 1) ? N : 0) + n * n * (((v >> 2) & 1) ? N : 0);
        for (int d = 0; d < 3; ++d)
          corners[24 * static_cast<size_t>(e) + 3 * v + d] = pts[3 * (static_cast<size_t>(e) * np + p) + d];
      }
    ctrl = corners.data();
  }
  for (size_t q = 0; q < static_cast<size_t>(nspec) * 24; ++q)
    if (!std::isfinite(ctrl[q])) return fail(c, SEM_EINVAL, "non-finite corner coordinate");

  std::vector<int32_t> color;
  int ncolors = 0;
  std::string err;
  if (color_elements(nspec, n, nglob, ibool, &color, &ncolors, &err)) return fail(c, SEM_EINVAL, err);

  // geometry per element (caller order)
  std::vector<double> xyz(3 * np), G(9 * np), J(np);
  c->dxmin.assign(nspec, 0.0);
  c->node_xyz.assign(3 * static_cast<size_t>(nglob), 0.0);
  std::vector<float> geom(static_cast<size_t>(nspec) * 10 * np);  // [e][10][p] in caller p order
  for (int e = 0; e < nspec; ++e) {
    bool ok;
    if (pts) {
      std::memcpy(xyz.data(), pts + 3 * static_cast<size_t>(e) * np, sizeof(double) * 3 * np);
      ok = geometry_from_positions(n, c->hprime.data(), xyz.data(), G.data(), J.data());
    } else {
      ok = element_geometry(n, c->xi.data(), c->hprime.data(), ctrl + 24 * static_cast<size_t>(e), xyz.data(),
                            G.data(), J.data());
    }
    if (!ok) return fail(c, SEM_EINVAL, "element " + std::to_string(e) + " has a Jacobian determinant <= 0");
    double dmin = 1e300;
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          const int p = i + n * (j + n * k);
          const int nb[3] = {i + 1 < n ? p + 1 : -1, j + 1 < n ? p + n : -1, k + 1 < n ? p + n * n : -1};
          for (int d = 0; d < 3; ++d) {
            if (nb[d] < 0) continue;
            const double dx = xyz[3 * nb[d]] - xyz[3 * p], dy = xyz[3 * nb[d] + 1] - xyz[3 * p + 1],
                         dz = xyz[3 * nb[d] + 2] - xyz[3 * p + 2];
            dmin = std::min(dmin, std::sqrt(dx * dx + dy * dy + dz * dz));
          }
        }
    c->dxmin[e] = dmin;
    for (int p = 0; p < np; ++p) {
      const size_t q = static_cast<size_t>(e) * np + p;
      for (int d = 0; d < 3; ++d) c->node_xyz[3 * static_cast<size_t>(ibool[q]) + d] = xyz[3 * p + d];
      float* gq = geom.data() + static_cast<size_t>(e) * 10 * np;
      for (int a = 0; a < 9; ++a) gq[a * np + p] = static_cast<float>(G[9 * p + a]);
      gq[9 * np + p] = static_cast<float>(J[p]);
    }
  }

  // patches (bricks of the lattice coordinates, coloured) give the record order
  PatchShape shape;
  PatchPlan plan;
  if (patch_shape(n, &shape)) return fail(c, SEM_EINVAL, "no patch kernel for this order");
  if (c->shape_opt.bx > 0) shape = c->shape_opt;
  if (build_patches(nspec, n, nglob, ibool, shape, &plan, &err)) return fail(c, SEM_EINVAL, "patches: " + err);
  c->shape = shape;
  c->order = plan.elem;
  c->node_new = plan.node_new;
  c->perm.assign(nglob, 0);
  for (int g = 0; g < nglob; ++g) c->perm[c->node_new[g]] = g;
  c->pos_of.assign(nspec, 0);
  for (int s = 0; s < nspec; ++s) c->pos_of[c->order[s]] = s;

  // element list for the element kernel: spatial slabs along the longest axis of the
  // element centroids (equal element counts), colour by colour inside a slab, caller order
  // inside a colour
  const int K = std::max(1, std::min(c->slabs_opt, nspec));
  std::vector<int> slab(nspec, 0);
  if (K > 1) {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    std::vector<double> cen(3 * static_cast<size_t>(nspec), 0.0);
    for (int e = 0; e < nspec; ++e)
      for (int d = 0; d < 3; ++d) {
        double m = 0.0;
        for (int v = 0; v < 8; ++v) m += ctrl[24 * static_cast<size_t>(e) + 3 * v + d];
        cen[3 * static_cast<size_t>(e) + d] = m / 8.0;
        lo[d] = std::min(lo[d], m / 8.0);
        hi[d] = std::max(hi[d], m / 8.0);
      }
    int ax = 0;
    for (int d = 1; d < 3; ++d)
      if (hi[d] - lo[d] > hi[ax] - lo[ax]) ax = d;
    std::vector<int> byc(nspec);
    for (int e = 0; e < nspec; ++e) byc[e] = e;
    std::stable_sort(byc.begin(), byc.end(), [&](int a, int b) { return cen[3 * static_cast<size_t>(a) + ax] < cen[3 * static_cast<size_t>(b) + ax]; });
    for (int r = 0; r < nspec; ++r) slab[byc[r]] = static_cast<int>(static_cast<long long>(r) * K / nspec);
  }
  c->color_count.assign(ncolors, 0);
  for (int e = 0; e < nspec; ++e) c->color_count[color[e]]++;
  std::vector<int> cnt(static_cast<size_t>(K) * ncolors, 0);
  for (int e = 0; e < nspec; ++e) cnt[static_cast<size_t>(slab[e]) * ncolors + color[e]]++;
  std::vector<int> off(cnt.size() + 1, 0);
  for (size_t k = 0; k < cnt.size(); ++k) off[k + 1] = off[k] + cnt[k];
  c->sweep_off.assign(1, 0);
  for (size_t k = 0; k < cnt.size(); ++k)
    if (cnt[k] > 0) c->sweep_off.push_back(off[k + 1]);
  c->slabs = K;
  std::vector<int> elist(nspec, 0);
  {
    std::vector<int> fillp(off.begin(), off.end() - 1);
    for (int e = 0; e < nspec; ++e) elist[fillp[static_cast<size_t>(slab[e]) * ncolors + color[e]]++] = c->pos_of[e];
  }

  // element records in patch sweep order; the ibool words carry the first-touch flag of the
  // element kernel's order (the patch kernel has its own, in the patch node lists)
  const int RW = rec_words(n);
  c->rec.assign(static_cast<size_t>(nspec) * RW, 0.f);
  std::vector<char> touched(nglob, 0);
  for (int t = 0; t < nspec; ++t) {
    const int s = elist[t];
    const int e = c->order[s];
    float* r = c->rec.data() + static_cast<size_t>(s) * RW;
    const float* gq = geom.data() + static_cast<size_t>(e) * 10 * np;
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          const int p = i + n * (j + n * k);
          const int q = rec_pos(n, i, j, k);
          uint32_t g = static_cast<uint32_t>(c->node_new[ibool[static_cast<size_t>(e) * np + p]]);
          if (!touched[g]) {
            touched[g] = 1;
            g |= kFirstTouchBit;
          }
          std::memcpy(&r[kIbool * np + p], &g, sizeof(uint32_t));
          for (int a = 0; a < 9; ++a) r[(kG + a) * np + q] = gq[a * np + p];
          r[kJac * np + q] = gq[9 * np + p];
        }
  }
  // patch descriptors; the first touch of every node in patch-colour order is flagged on the
  // ibool word of its first local point in that patch's table, the points alone at their
  // patch node on their own words; the slot tables become shared-memory offsets of the
  // patch kernel's workspaces
  int ES = 0, TS = 0, EPT = 0;
  if (patch_layout(n, &ES, &TS, &EPT)) return fail(c, SEM_EINVAL, "no patch layout for this order");
  auto ws_float = [&](int le) { return (le / EPT) * TS + (le % EPT) * ES; };
  std::vector<uint16_t> slots(plan.csr.size(), kPatchNoSlot), words;
  std::vector<int> word_off(plan.tab_nelem.size(), 0);
  for (size_t t = 0; t < plan.tab_nelem.size(); ++t) {
    const size_t g0 = plan.tab_csr_off[t];
    const size_t g1 = t + 1 < plan.tab_nelem.size() ? plan.tab_csr_off[t + 1] : plan.csr.size();
    word_off[t] = static_cast<int>(words.size());
    for (size_t q = g0; q < g1; ++q) {
      const uint16_t v = plan.csr[q];
      if (v == kPatchNoSlot || (v & kPatchChain)) {
        slots[q] = v;
        continue;
      }
      const int le = v / np, pp = v % np;
      const int off = ws_float(le) + 3 * pp;
      if (off >= kPatchChain) return fail(c, SEM_EINVAL, "patch workspace offsets exceed the slot range");
      slots[q] = static_cast<uint16_t>(off);
      if ((q - g0) % kPatchSlots == 0 && (q - g0) / kPatchSlots < static_cast<size_t>(plan.tab_nshared[t])) {
        const int wo = ws_float(le) + 9 * np + pp;  // a shared node's first slot
        if (wo > 0xFFFF) return fail(c, SEM_EINVAL, "patch workspace offsets exceed the word range");
        words.push_back(static_cast<uint16_t>(wo));
      }
    }
  }
  std::vector<PatchDesc> pdesc(plan.npatch);
  auto flag_word = [&](int slot, int pp, uint32_t bit) {
    float* r = c->rec.data() + static_cast<size_t>(slot) * RW;
    uint32_t wd;
    std::memcpy(&wd, &r[kIbool * np + pp], sizeof(uint32_t));
    wd |= bit;
    std::memcpy(&r[kIbool * np + pp], &wd, sizeof(uint32_t));
  };
  // the patch that touches each node last in the sweep (patches are in sweep order); its
  // local points at the node carry kPatchLastBit
  std::vector<int> last_patch(nglob, -1);
  for (int P = 0; P < plan.npatch; ++P)
    for (int k = plan.node_off[P]; k < plan.node_off[P + 1]; ++k) last_patch[plan.nodes[k] & ~kFirstTouchBit] = P;
  for (int P = 0; P < plan.npatch; ++P) {
    PatchDesc& d = pdesc[P];
    const int t = plan.table_of[P];
    d.slot0 = plan.patch_off[P];
    d.nelem = plan.patch_off[P + 1] - plan.patch_off[P];
    d.nshared = plan.tab_nshared[t];
    d.slot_off = plan.tab_csr_off[t];
    d.word_off = word_off[t];
    d.src_off = d.nsrc = d.pad = 0;
    const uint16_t* lid = plan.lid.data() + plan.tab_lid_off[t];
    for (int q = 0; q < d.nelem * np; ++q)
      if (last_patch[plan.nodes[plan.node_off[P] + lid[q]] & ~kFirstTouchBit] == P)
        flag_word(d.slot0 + q / np, q % np, kPatchLastBit);
    const int nnode = plan.node_off[P + 1] - plan.node_off[P];
    for (int k = 0; k < nnode; ++k) {
      if (!(plan.nodes[plan.node_off[P] + k] & kFirstTouchBit)) continue;
      const int q0 = plan.first_q[static_cast<size_t>(plan.tab_first_off[t]) + k];
      flag_word(d.slot0 + q0 / np, q0 % np, kPatchFirstBit);
    }
    const uint32_t* ex = plan.excl.data() + plan.tab_excl_off[t];
    for (int q = 0; q < d.nelem * np; ++q)
      if ((ex[q / 32] >> (q % 32)) & 1u) flag_word(d.slot0 + q / np, q % np, kAloneBit);
  }
  c->last_patch.assign(nglob, -1);
  for (int g = 0; g < nglob; ++g) c->last_patch[plan.node_new[g]] = last_patch[g];
  c->pdesc = pdesc;
  c->pcolor_off = plan.color_off;
  c->npatch = plan.npatch;
  c->pmax_nodes = plan.max_nodes;
  c->ptables = static_cast<int>(plan.tab_nelem.size());

  c->ibool.assign(ibool, ibool + nloc);
  c->ctrl.assign(ctrl, ctrl + 24 * static_cast<size_t>(nspec));
  c->nspec = nspec;
  c->nglob = nglob;
  c->ncolors = ncolors;
  c->have_mesh = true;
  c->have_mat = false;
  c->have_dt = false;
  c->pending = false;
  c->steps = 0;
  drop_graph(c);

  int r = set_device(c);
  if (r) return r;
  cudaStreamSynchronize(c->stream);
  DevCtl* keep_ctl = c->d_ctl;
  c->d_ctl = nullptr;
  free_device(c);
  c->d_ctl = keep_ctl;
  c->dev_bytes = sizeof(DevCtl);
  const size_t nf = kNodeStride * static_cast<size_t>(nglob) * c->shots;
  if ((r = dev_alloc(c, &c->d_rec, c->rec.size())) || (r = dev_alloc(c, &c->d_order, c->order.size())) ||
      (r = dev_alloc(c, &c->d_elist, elist.size())) || (r = dev_alloc(c, &c->d_pdesc, pdesc.size())) ||
      (r = dev_alloc(c, &c->d_perm, c->perm.size())) || (r = dev_alloc(c, &c->d_node_new, c->node_new.size())) ||
      (r = dev_alloc(c, &c->d_pslots, std::max<size_t>(slots.size(), kPatchSlots))) ||
      (r = dev_alloc(c, &c->d_pwords, std::max<size_t>(words.size(), 1))) ||
      (r = dev_alloc(c, &c->d_pcolor_end, static_cast<size_t>(plan.ncolors))) || (r = dev_alloc(c, &c->d_sync, 1)) ||
      (r = dev_alloc(c, &c->d_u, nf)) ||
      (r = dev_alloc(c, &c->d_v, nf)) || (r = dev_alloc(c, &c->d_a, nf)) ||
      (r = dev_alloc(c, &c->d_minv, static_cast<size_t>(nglob))))
    return r;
  // geometry and ibool travel once; the material fields are written on the device
  SEM_CUDA(c, cudaMemcpyAsync(c->d_rec, c->rec.data(), c->rec.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  SEM_CUDA(c, cudaMemcpyAsync(c->d_order, c->order.data(), c->order.size() * sizeof(int), cudaMemcpyHostToDevice,
                              c->stream));
  SEM_CUDA(c, cudaMemcpyAsync(c->d_elist, elist.data(), elist.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  SEM_CUDA(c, cudaMemcpyAsync(c->d_perm, c->perm.data(), c->perm.size() * sizeof(int), cudaMemcpyHostToDevice,
                              c->stream));
  SEM_CUDA(c, cudaMemcpyAsync(c->d_node_new, c->node_new.data(), c->node_new.size() * sizeof(int),
                              cudaMemcpyHostToDevice, c->stream));
  SEM_CUDA(c, cudaMemcpyAsync(c->d_pdesc, pdesc.data(), pdesc.size() * sizeof(PatchDesc), cudaMemcpyHostToDevice,
                              c->stream));
  if (!slots.empty())
    SEM_CUDA(c, cudaMemcpyAsync(c->d_pslots, slots.data(), slots.size() * sizeof(uint16_t), cudaMemcpyHostToDevice,
                                c->stream));
  if (!words.empty())
    SEM_CUDA(c, cudaMemcpyAsync(c->d_pwords, words.data(), words.size() * sizeof(uint16_t), cudaMemcpyHostToDevice,
                                c->stream));
  SEM_CUDA(c, cudaMemcpyAsync(c->d_pcolor_end, plan.color_off.data() + 1, plan.ncolors * sizeof(int),
                              cudaMemcpyHostToDevice, c->stream));
  SEM_CUDA(c, cudaMemsetAsync(c->d_sync, 0, sizeof(SweepSync), c->stream));
  SEM_CUDA(c, cudaMemsetAsync(c->d_u, 0, nf * sizeof(float), c->stream));
  SEM_CUDA(c, cudaMemsetAsync(c->d_v, 0, nf * sizeof(float), c->stream));
  SEM_CUDA(c, cudaMemsetAsync(c->d_a, 0, nf * sizeof(float), c->stream));
  SEM_CUDA(c, cudaMemsetAsync(c->d_minv, 0, nglob * sizeof(float), c->stream));
  SEM_CUDA(c, cudaStreamSynchronize(c->stream));
  std::vector<float>().swap(c->rec);  // the device copy is the only one from here on
  c->nsrc = 0;
  c->nrec = 0;
  return SEM_OK;
}

int sem_set_mesh(sem_ctx* c, int nspec, int nglob, const int32_t* ibool, const double* xyz) {
  if (!xyz) return fail(c, SEM_EINVAL, "sem_set_mesh: NULL coordinates");
  return set_mesh_impl(c, nspec, nglob, ibool, nullptr, xyz);
}

int sem_set_mesh_corners(sem_ctx* c, int nspec, int nglob, const int32_t* ibool, const double* ctrl) {
  if (!ctrl) return fail(c, SEM_EINVAL, "sem_set_mesh_corners: NULL corners");
  return set_mesh_impl(c, nspec, nglob, ibool, ctrl, nullptr);
}

// Writes kappa and mu into the element records, assembles the mass and its inverse and the
// per-element largest vp, all on the device, from per-point arrays already on the device.
static int material_apply(sem_ctx* c, const float* rho, const float* p1, const float* p2, bool moduli) {
  MaterialLaunch m{};
  m.rec = c->d_rec;
  m.order = c->d_order;
  m.elist = c->d_elist;
  m.rho = rho;
  m.p1 = p1;
  m.p2 = p2;
  m.moduli = moduli ? 1 : 0;
  m.ngll = c->ngll;
  m.nspec = c->nspec;
  m.nglob = c->nglob;
  for (int i = 0; i < c->ngll; ++i) m.w[i] = c->w[i];
  double *mass = nullptr, *vpmax = nullptr;
  SEM_CUDA(c, cudaMallocAsync(reinterpret_cast<void**>(&mass), c->nglob * sizeof(double), c->stream));
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&vpmax), c->nspec * sizeof(double), c->stream);
  if (e == cudaSuccess)
    e = static_cast<cudaError_t>(launch_material_apply(m, c->sweep_off.data(), static_cast<int>(c->sweep_off.size()) - 1, mass, c->d_minv, vpmax,
                                                       c->stream));
  c->vpmax.assign(c->nspec, 0.0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->vpmax.data(), vpmax, c->nspec * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  cudaFreeAsync(mass, c->stream);
  if (vpmax) cudaFreeAsync(vpmax, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "material upload");
  SEM_CUDA(c, cudaStreamSynchronize(c->stream));
  c->have_mat = true;
  drop_graph(c);
  return SEM_OK;
}

// Shared by sem_set_material and sem_set_moduli: per local point rho and (kappa, mu), either
// given or derived from (vp, vs); checked on the host, then applied on the device.
static int set_material_impl(sem_ctx* c, const float* rho, const float* p1, const float* p2, bool moduli) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (!c->have_mesh) return fail(c, SEM_ESTATE, "sem_set_mesh has not been called");
  if (!rho || !p1 || !p2) return fail(c, SEM_EINVAL, "material: NULL array");
  const int n = c->ngll, np = n * n * n;
  const size_t nloc = static_cast<size_t>(c->nspec) * np;
  for (size_t q = 0; q < nloc; ++q) {
    if (!std::isfinite(rho[q]) || !std::isfinite(p1[q]) || !std::isfinite(p2[q]))
      return fail(c, SEM_EINVAL, "non-finite material value");
    const bool ok = moduli ? (rho[q] > 0.f && p2[q] >= 0.f && p1[q] > 0.f) : (rho[q] > 0.f && p2[q] >= 0.f && p1[q] > p2[q]);
    if (!ok)
      return fail(c, SEM_EINVAL,
                  std::string(moduli ? "moduli need rho > 0, kappa > 0, mu >= 0" : "material needs rho > 0, vs >= 0, vp > vs") +
                      " (local point " + std::to_string(q) + ")");
  }
  int r = set_device(c);
  if (r) return r;
  float* tmp = nullptr;
  SEM_CUDA(c, cudaMallocAsync(reinterpret_cast<void**>(&tmp), 3 * nloc * sizeof(float), c->stream));
  const float* src[3] = {rho, p1, p2};
  cudaError_t e = cudaSuccess;
  for (int f = 0; f < 3 && e == cudaSuccess; ++f)
    e = cudaMemcpyAsync(tmp + f * nloc, src[f], nloc * sizeof(float), cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) {
    cudaFreeAsync(tmp, c->stream);
    return cuda_fail(c, e, "material upload");
  }
  r = material_apply(c, tmp, tmp + nloc, tmp + 2 * nloc, moduli);
  cudaFreeAsync(tmp, c->stream);
  return r;
}

int sem_set_material(sem_ctx* c, const float* rho, const float* vp, const float* vs) {
  return set_material_impl(c, rho, vp, vs, false);
}

int sem_set_moduli(sem_ctx* c, const float* rho, const float* kappa, const float* mu) {
  return set_material_impl(c, rho, kappa, mu, true);
}

int sem_set_moduli_dev(sem_ctx* c, const float* rho, const float* kappa, const float* mu) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (!c->have_mesh) return fail(c, SEM_ESTATE, "sem_set_mesh has not been called");
  if (!rho || !kappa || !mu) return fail(c, SEM_EINVAL, "material: NULL array");
  int r = set_device(c);
  if (r) return r;
  MaterialLaunch m{};
  m.rho = rho;
  m.p1 = kappa;
  m.p2 = mu;
  m.moduli = 1;
  m.ngll = c->ngll;
  m.nspec = c->nspec;
  m.nglob = c->nglob;
  unsigned long long* d_bad = nullptr;
  unsigned long long bad = ~0ull;
  SEM_CUDA(c, cudaMallocAsync(reinterpret_cast<void**>(&d_bad), sizeof(unsigned long long), c->stream));
  cudaError_t e = cudaMemsetAsync(d_bad, 0xff, sizeof(unsigned long long), c->stream);
  if (e == cudaSuccess) e = static_cast<cudaError_t>(launch_material_check(m, d_bad, c->stream));
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, c->stream);
  cudaFreeAsync(d_bad, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "material check");
  SEM_CUDA(c, cudaStreamSynchronize(c->stream));
  if (bad != ~0ull)
    return fail(c, SEM_EINVAL, "moduli need finite rho > 0, kappa > 0, mu >= 0 (local point " + std::to_string(bad) + ")");
  return material_apply(c, rho, kappa, mu, true);
}

int sem_suggest_dt(sem_ctx* c, double courant, double* dt_out) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (!c->have_mat) return fail(c, SEM_ESTATE, "sem_set_material has not been called");
  if (!dt_out || !(courant > 0.0)) return fail(c, SEM_EINVAL, "sem_suggest_dt: bad arguments");
  double best = 1e300;
  for (int e = 0; e < c->nspec; ++e) best = std::min(best, c->dxmin[e] / c->vpmax[e]);
  *dt_out = courant * best;
  return SEM_OK;
}

int sem_set_dt(sem_ctx* c, double dt) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (!c->have_mat) return fail(c, SEM_ESTATE, "sem_set_material has not been called");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, SEM_EINVAL, "dt must be positive and finite");
  if (c->pending) {  // complete the state with the old dt before switching
    int r = set_device(c);
    if (r || (r = finish_state(c))) return r;
  }
  c->dt = dt;
  c->have_dt = true;
  drop_graph(c);
  return SEM_OK;
}

int sem_node_xyz(sem_ctx* c, int npts, const int32_t* node, double* xyz_out) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (!c->have_mesh) return fail(c, SEM_ESTATE, "sem_set_mesh has not been called");
  if (npts < 0 || (npts > 0 && (!node || !xyz_out))) return fail(c, SEM_EINVAL, "sem_node_xyz: bad arguments");
  for (int i = 0; i < npts; ++i) {
    if (node[i] < 0 || node[i] >= c->nglob) return fail(c, SEM_EINVAL, "node out of range");
    for (int d = 0; d < 3; ++d) xyz_out[3 * i + d] = c->node_xyz[3 * static_cast<size_t>(node[i]) + d];
  }
  return SEM_OK;
}

int sem_locate_nodes(sem_ctx* c, int npts, const double* xyz, const double* surface_z, int32_t* node_out) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (!c->have_mesh) return fail(c, SEM_ESTATE, "sem_set_mesh has not been called");
  if (npts < 0 || (npts > 0 && (!xyz || !node_out))) return fail(c, SEM_EINVAL, "sem_locate_nodes: bad arguments");
  if (locate_nodes(c->nglob, c->node_xyz.data(), npts, xyz, surface_z, node_out))
    return fail(c, SEM_EINVAL, "no node lies on the requested surface");
  return SEM_OK;
}

// The point sources of the fused sweep: entry s (internal node, shot, force) goes to the patch
// that touches its node last; the descriptors name each patch's range.
static int set_patch_sources(sem_ctx* c, const std::vector<int>& nodes, const std::vector<int>& shots,
                             const std::vector<double>& forces) {
  if (c->npatch <= 0) return SEM_OK;
  std::vector<std::pair<int, int>> by_patch;  // (patch, entry), in entry order within a patch
  for (size_t s = 0; s < nodes.size(); ++s) by_patch.emplace_back(c->last_patch[nodes[s]], static_cast<int>(s));
  std::stable_sort(by_patch.begin(), by_patch.end(),
                   [](const std::pair<int, int>& x, const std::pair<int, int>& y) { return x.first < y.first; });
  std::vector<PatchSrc> list(by_patch.size());
  for (PatchDesc& d : c->pdesc) d.src_off = d.nsrc = 0;
  for (size_t k = 0; k < by_patch.size(); ++k) {
    const int P = by_patch[k].first, s = by_patch[k].second;
    PatchSrc& e = list[k];
    e.node = nodes[s];
    e.shot = shots[s];
    for (int d = 0; d < 3; ++d) e.f[d] = forces[3 * static_cast<size_t>(s) + d];
    PatchDesc& d = c->pdesc[P];
    if (d.nsrc == 0) d.src_off = static_cast<int>(k);
    ++d.nsrc;
  }
  int r = dev_alloc(c, &c->d_psrc, list.size());
  if (r) return r;
  if (!list.empty())
    SEM_CUDA(c, cudaMemcpy(c->d_psrc, list.data(), list.size() * sizeof(PatchSrc), cudaMemcpyHostToDevice));
  SEM_CUDA(c, cudaMemcpy(c->d_pdesc, c->pdesc.data(), c->pdesc.size() * sizeof(PatchDesc), cudaMemcpyHostToDevice));
  return SEM_OK;
}

static int set_sources_impl(sem_ctx* c, int nsrc, const int32_t* shot, const int32_t* node, const double* force,
                            double f0, double t0) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (!c->have_mesh) return fail(c, SEM_ESTATE, "sem_set_mesh has not been called");
  if (nsrc < 0 || (nsrc > 0 && (!node || !force)) || !std::isfinite(f0) || !std::isfinite(t0))
    return fail(c, SEM_EINVAL, "sem_set_sources: bad arguments");
  // one entry per (shot, node); sources sharing both merge (same time function, forces add);
  // without a shot index a source acts in every shot
  std::vector<int> nodes, shots;
  std::vector<double> forces;
  std::unordered_map<int64_t, size_t> entry;  // (shot, node) -> index of its entry
  for (int s = 0; s < nsrc; ++s) {
    if (node[s] < 0 || node[s] >= c->nglob) return fail(c, SEM_EINVAL, "source node out of range");
    if (shot && (shot[s] < 0 || shot[s] >= c->shots)) return fail(c, SEM_EINVAL, "source shot out of range");
    for (int d = 0; d < 3; ++d)
      if (!std::isfinite(force[3 * s + d])) return fail(c, SEM_EINVAL, "non-finite source force");
    const int first = shot ? shot[s] : 0, last = shot ? shot[s] : c->shots - 1;
    for (int sh = first; sh <= last; ++sh) {
      const int g = c->node_new[node[s]];  // internal node
      const int64_t key = static_cast<int64_t>(sh) * c->nglob + g;
      const auto found = entry.find(key);
      const size_t m = found == entry.end() ? nodes.size() : found->second;
      if (m == nodes.size()) {
        entry.emplace(key, m);
        nodes.push_back(g);
        shots.push_back(sh);
        forces.insert(forces.end(), force + 3 * s, force + 3 * s + 3);
      } else {
        for (int d = 0; d < 3; ++d) forces[3 * m + d] += force[3 * s + d];
      }
    }
  }
  int r = set_device(c);
  if (r) return r;
  cudaStreamSynchronize(c->stream);
  c->dev_bytes -= c->nsrc * (2 * sizeof(int) + 3 * sizeof(double));
  c->nsrc = static_cast<int>(nodes.size());
  if ((r = dev_alloc(c, &c->d_src_node, nodes.size())) || (r = dev_alloc(c, &c->d_src_shot, shots.size())) ||
      (r = dev_alloc(c, &c->d_src_force, forces.size())))
    return r;
  if (!nodes.empty()) {
    SEM_CUDA(c, cudaMemcpy(c->d_src_node, nodes.data(), nodes.size() * sizeof(int), cudaMemcpyHostToDevice));
    SEM_CUDA(c, cudaMemcpy(c->d_src_shot, shots.data(), shots.size() * sizeof(int), cudaMemcpyHostToDevice));
    SEM_CUDA(c, cudaMemcpy(c->d_src_force, forces.data(), forces.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  if ((r = set_patch_sources(c, nodes, shots, forces))) return r;
  c->f0 = f0;
  c->t0 = t0;
  drop_graph(c);
  return SEM_OK;
}

int sem_set_source_nodes(sem_ctx* c, int nsrc, const int32_t* node, const double* force, double f0, double t0) {
  return set_sources_impl(c, nsrc, nullptr, node, force, f0, t0);
}

int sem_set_sources(sem_ctx* c, int nsrc, const double* xyz, const double* force, double f0, double t0) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (!c->have_mesh) return fail(c, SEM_ESTATE, "sem_set_mesh has not been called");
  if (nsrc < 0 || (nsrc > 0 && (!xyz || !force))) return fail(c, SEM_EINVAL, "sem_set_sources: bad arguments");
  for (size_t q = 0; q < 3 * static_cast<size_t>(nsrc); ++q)
    if (!std::isfinite(xyz[q])) return fail(c, SEM_EINVAL, "non-finite source position");
  std::vector<int32_t> node(nsrc > 0 ? nsrc : 1);
  if (nsrc > 0) locate_nodes(c->nglob, c->node_xyz.data(), nsrc, xyz, nullptr, node.data());
  return set_sources_impl(c, nsrc, nullptr, node.data(), force, f0, t0);
}

int sem_set_shot_sources(sem_ctx* c, int nsrc, const int32_t* shot, const int32_t* node, const double* force,
                         double f0, double t0) {
  if (nsrc > 0 && !shot) return fail(c, SEM_EINVAL, "sem_set_shot_sources: NULL shot array");
  return set_sources_impl(c, nsrc, shot, node, force, f0, t0);
}

int sem_set_shot_sources_at(sem_ctx* c, int nsrc, const int32_t* shot, const double* xyz, const double* force,
                            const double* moment, double f0, double t0) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (!c->have_mesh) return fail(c, SEM_ESTATE, "sem_set_mesh has not been called");
  if (nsrc < 0 || (nsrc > 0 && (!xyz || (!force) == (!moment))))
    return fail(c, SEM_EINVAL, "sem_set_shot_sources_at: bad arguments (give xyz and exactly one of force, moment)");
  const int n = c->ngll, np = n * n * n, nv = force ? 3 : 6;
  for (int s = 0; s < nsrc; ++s) {
    const double* v = (force ? force : moment) + static_cast<size_t>(nv) * s;
    for (int q = 0; q < 3; ++q)
      if (!std::isfinite(xyz[3 * static_cast<size_t>(s) + q])) return fail(c, SEM_EINVAL, "non-finite source position");
    for (int q = 0; q < nv; ++q)
      if (!std::isfinite(v[q])) return fail(c, SEM_EINVAL, "non-finite source value");
    if (shot && (shot[s] < 0 || shot[s] >= c->shots)) return fail(c, SEM_EINVAL, "source shot out of range");
  }
  std::vector<int32_t> elem(nsrc > 0 ? nsrc : 1);
  std::vector<double> refs(3 * static_cast<size_t>(nsrc > 0 ? nsrc : 1));
  if (nsrc > 0) locate_points(c->nspec, c->ctrl.data(), nsrc, xyz, elem.data(), refs.data());
  std::vector<int32_t> shots, nodes;
  std::vector<double> forces, f(3 * static_cast<size_t>(np));
  for (int s = 0; s < nsrc; ++s) {
    const double* v = (force ? force : moment) + static_cast<size_t>(nv) * s;
    const int e = elem[s];
    if (e < 0) return fail(c, SEM_EINVAL, "source " + std::to_string(s) + " lies outside the mesh");
    point_source_forces(n, c->xi.data(), c->hprime.data(), c->ctrl.data() + 24 * static_cast<size_t>(e),
                        refs.data() + 3 * static_cast<size_t>(s), force ? v : nullptr, moment ? v : nullptr, f.data());
    for (int p = 0; p < np; ++p) {
      const double* fp = f.data() + 3 * p;
      if (fp[0] == 0.0 && fp[1] == 0.0 && fp[2] == 0.0) continue;
      if (shot) shots.push_back(shot[s]);
      nodes.push_back(c->ibool[static_cast<size_t>(e) * np + p]);
      forces.insert(forces.end(), fp, fp + 3);
    }
  }
  return set_sources_impl(c, static_cast<int>(nodes.size()), shot ? shots.data() : nullptr, nodes.data(),
                          forces.data(), f0, t0);
}

int sem_set_shot_moment_sources(sem_ctx* c, int nsrc, const int32_t* shot, const int32_t* node, const double* moment,
                                double f0, double t0) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (!c->have_mesh) return fail(c, SEM_ESTATE, "sem_set_mesh has not been called");
  if (nsrc < 0 || (nsrc > 0 && (!shot || !node || !moment)))
    return fail(c, SEM_EINVAL, "sem_set_shot_moment_sources: bad arguments");
  const int n = c->ngll, np = n * n * n;
  std::vector<int> owner_e(c->nglob, -1), owner_p(c->nglob, -1);  // lowest element holding a node
  for (int e = c->nspec - 1; e >= 0; --e)
    for (int p = 0; p < np; ++p) {
      const int g = c->ibool[static_cast<size_t>(e) * np + p];
      owner_e[g] = e;
      owner_p[g] = p;
    }
  std::vector<double> xyz(3 * np), G(9 * np), J(np);
  std::vector<int32_t> shots, nodes;
  std::vector<double> forces;
  for (int s = 0; s < nsrc; ++s) {
    if (node[s] < 0 || node[s] >= c->nglob) return fail(c, SEM_EINVAL, "source node out of range");
    if (shot[s] < 0 || shot[s] >= c->shots) return fail(c, SEM_EINVAL, "source shot out of range");
    for (int q = 0; q < 6; ++q)
      if (!std::isfinite(moment[6 * s + q])) return fail(c, SEM_EINVAL, "non-finite moment tensor");
    const int e = owner_e[node[s]], p0 = owner_p[node[s]];
    const int i0 = p0 % n, j0 = (p0 / n) % n, k0 = p0 / (n * n);
    element_geometry(n, c->xi.data(), c->hprime.data(), c->ctrl.data() + 24 * static_cast<size_t>(e), xyz.data(),
                     G.data(), J.data());
    const double* m6 = moment + 6 * s;  // Mxx Myy Mzz Mxy Mxz Myz
    const double M[3][3] = {{m6[0], m6[3], m6[4]}, {m6[3], m6[1], m6[5]}, {m6[4], m6[5], m6[2]}};
    const double* g0 = G.data() + 9 * static_cast<size_t>(p0);  // dxi_r/dx_d at 3r + d
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          // reference gradient of psi_(i,j,k) at the source point (i0, j0, k0)
          const double dr[3] = {(j == j0 && k == k0) ? c->hprime[i0 * n + i] : 0.0,
                                (i == i0 && k == k0) ? c->hprime[j0 * n + j] : 0.0,
                                (i == i0 && j == j0) ? c->hprime[k0 * n + k] : 0.0};
          if (dr[0] == 0.0 && dr[1] == 0.0 && dr[2] == 0.0) continue;
          double grad[3];
          for (int d = 0; d < 3; ++d) grad[d] = dr[0] * g0[d] + dr[1] * g0[3 + d] + dr[2] * g0[6 + d];
          shots.push_back(shot[s]);
          nodes.push_back(c->ibool[static_cast<size_t>(e) * np + i + n * (j + n * k)]);
          for (int a = 0; a < 3; ++a) forces.push_back(M[a][0] * grad[0] + M[a][1] * grad[1] + M[a][2] * grad[2]);
        }
  }
  return set_sources_impl(c, static_cast<int>(nodes.size()), shots.data(), nodes.data(), forces.data(), f0, t0);
}

int sem_set_shots(sem_ctx* c, int nshots) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (!c->have_mesh) return fail(c, SEM_ESTATE, "sem_set_mesh has not been called");
  if (nshots < 1 || static_cast<long long>(nshots) * c->nglob > (1ll << 31) - 1)
    return fail(c, SEM_EINVAL, "sem_set_shots: nshots must be >= 1 and nglob * nshots < 2^31");
  int r = set_device(c);
  if (r) return r;
  cudaStreamSynchronize(c->stream);
  const size_t old = kNodeStride * static_cast<size_t>(c->nglob) * c->shots * sizeof(float);
  c->dev_bytes -= 3 * old;
  if (c->d_f) {
    c->dev_bytes -= old;
    cudaFree(c->d_f);
    c->d_f = nullptr;
  }
  c->shots = nshots;
  const size_t nf = kNodeStride * static_cast<size_t>(c->nglob) * nshots;
  if ((r = dev_alloc(c, &c->d_u, nf)) || (r = dev_alloc(c, &c->d_v, nf)) || (r = dev_alloc(c, &c->d_a, nf))) return r;
  SEM_CUDA(c, cudaMemsetAsync(c->d_u, 0, nf * sizeof(float), c->stream));
  SEM_CUDA(c, cudaMemsetAsync(c->d_v, 0, nf * sizeof(float), c->stream));
  SEM_CUDA(c, cudaMemsetAsync(c->d_a, 0, nf * sizeof(float), c->stream));
  SEM_CUDA(c, cudaStreamSynchronize(c->stream));
  c->pending = false;
  c->steps = 0;
  c->nsrc = 0;  // sources name shots: set them again
  int rs = set_patch_sources(c, {}, {}, {});
  if (rs) return rs;
  drop_graph(c);
  return SEM_OK;
}

int sem_set_receivers(sem_ctx* c, int nrec, const double* xyz, int32_t* node_out) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (!c->have_mesh) return fail(c, SEM_ESTATE, "sem_set_mesh has not been called");
  if (nrec < 0 || (nrec > 0 && !xyz)) return fail(c, SEM_EINVAL, "sem_set_receivers: bad arguments");
  for (size_t q = 0; q < 3 * static_cast<size_t>(nrec); ++q)
    if (!std::isfinite(xyz[q])) return fail(c, SEM_EINVAL, "non-finite receiver position");
  std::vector<int32_t> node(nrec > 0 ? nrec : 1);
  if (nrec > 0) locate_nodes(c->nglob, c->node_xyz.data(), nrec, xyz, nullptr, node.data());
  const int r = sem_set_receiver_nodes(c, nrec, node.data());
  if (r == SEM_OK && node_out && nrec > 0) std::memcpy(node_out, node.data(), sizeof(int32_t) * nrec);
  return r;
}

int sem_set_receiver_nodes(sem_ctx* c, int nrec, const int32_t* node) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (!c->have_mesh) return fail(c, SEM_ESTATE, "sem_set_mesh has not been called");
  if (nrec < 0 || (nrec > 0 && !node)) return fail(c, SEM_EINVAL, "sem_set_receiver_nodes: bad arguments");
  for (int r = 0; r < nrec; ++r)
    if (node[r] < 0 || node[r] >= c->nglob) return fail(c, SEM_EINVAL, "receiver node out of range");
  int r = set_device(c);
  if (r) return r;
  cudaStreamSynchronize(c->stream);
  c->dev_bytes -= c->nrec * sizeof(int) + (2 * c->nrnodes + 1 + c->nrec) * sizeof(int);
  c->nrec = nrec;
  std::vector<int> internal(nrec);
  for (int k = 0; k < nrec; ++k) internal[k] = c->node_new[node[k]];
  // distinct receiver nodes and their receivers in ascending order (adjoint injection)
  std::vector<int> byn(nrec);
  for (int k = 0; k < nrec; ++k) byn[k] = k;
  std::stable_sort(byn.begin(), byn.end(), [&](int x, int y) { return internal[x] < internal[y]; });
  std::vector<int> rnode, roff(1, 0);
  for (int k = 0; k < nrec; ++k) {
    if (k == 0 || internal[byn[k]] != internal[byn[k - 1]]) {
      if (k > 0) roff.push_back(k);
      rnode.push_back(internal[byn[k]]);
    }
  }
  if (nrec > 0) roff.push_back(nrec);
  c->nrnodes = static_cast<int>(rnode.size());
  if ((r = dev_alloc(c, &c->d_rec_node, static_cast<size_t>(nrec))) ||
      (r = dev_alloc(c, &c->d_rnode, rnode.size())) || (r = dev_alloc(c, &c->d_roff, rnode.empty() ? 0 : roff.size())) ||
      (r = dev_alloc(c, &c->d_rlist, byn.size())))
    return r;
  if (nrec > 0) {
    SEM_CUDA(c, cudaMemcpy(c->d_rec_node, internal.data(), nrec * sizeof(int), cudaMemcpyHostToDevice));
    SEM_CUDA(c, cudaMemcpy(c->d_rnode, rnode.data(), rnode.size() * sizeof(int), cudaMemcpyHostToDevice));
    SEM_CUDA(c, cudaMemcpy(c->d_roff, roff.data(), roff.size() * sizeof(int), cudaMemcpyHostToDevice));
    SEM_CUDA(c, cudaMemcpy(c->d_rlist, byn.data(), byn.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  // the same receivers by the patch that touches their node last (the fused adjoint sweep),
  // ascending receiver index within a patch
  if (c->npatch > 0) {
    std::vector<std::pair<int, int>> by_patch;  // (patch, receiver)
    for (int k = 0; k < nrec; ++k) by_patch.emplace_back(c->last_patch[internal[k]], k);
    std::sort(by_patch.begin(), by_patch.end());
    std::vector<PatchRecv> list(by_patch.size());
    std::vector<int> range(2 * static_cast<size_t>(c->npatch), 0);
    for (size_t k = 0; k < by_patch.size(); ++k) {
      const int P = by_patch[k].first, rr = by_patch[k].second;
      list[k] = PatchRecv{internal[rr], rr};
      if (range[2 * P + 1] == 0) range[2 * P] = static_cast<int>(k);
      ++range[2 * P + 1];
    }
    if ((r = dev_alloc(c, &c->d_precv, list.size())) || (r = dev_alloc(c, &c->d_precv_range, range.size()))) return r;
    if (!list.empty())
      SEM_CUDA(c, cudaMemcpy(c->d_precv, list.data(), list.size() * sizeof(PatchRecv), cudaMemcpyHostToDevice));
    SEM_CUDA(c, cudaMemcpy(c->d_precv_range, range.data(), range.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  drop_graph(c);
  return SEM_OK;
}

// Host arrays pass through a stream-ordered staging buffer in the caller layout, so every
// transfer is one contiguous copy; the layout change is a kernel on the device.
static int set_state_impl(sem_ctx* c, const float* u, const float* v, const float* a, cudaMemcpyKind kind) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (!c->have_mesh) return fail(c, SEM_ESTATE, "sem_set_mesh has not been called");
  int r = set_device(c);
  if (r) return r;
  const size_t n3 = 3 * static_cast<size_t>(c->nglob) * c->shots;
  const bool host = kind == cudaMemcpyHostToDevice;
  const float* src[3] = {u, v, a};
  float* dst[3] = {c->d_u, c->d_v, c->d_a};
  float* stage = nullptr;
  if (host && (u || v || a)) SEM_CUDA(c, cudaMallocAsync(reinterpret_cast<void**>(&stage), n3 * sizeof(float), c->stream));
  int rc = SEM_OK;
  for (int q = 0; q < 3 && rc == SEM_OK; ++q) {
    cudaError_t e = cudaSuccess;
    if (!src[q]) {
      e = cudaMemsetAsync(dst[q], 0, kNodeStride * static_cast<size_t>(c->nglob) * c->shots * sizeof(float), c->stream);
    } else {
      const float* from = src[q];
      if (host) {
        e = cudaMemcpyAsync(stage, src[q], n3 * sizeof(float), cudaMemcpyHostToDevice, c->stream);
        from = stage;
      }
      const int* perm = (!host && c->node_order == 1) ? nullptr : c->d_perm;
      if (e == cudaSuccess) e = static_cast<cudaError_t>(launch_unpack(from, dst[q], perm, c->nglob, c->shots, c->stream));
    }
    if (e != cudaSuccess) rc = cuda_fail(c, e, "sem_set_state copy");
  }
  if (stage) cudaFreeAsync(stage, c->stream);
  if (rc) return rc;
  c->pending = false;
  c->steps = 0;
  if (host) {  // values from the host are checked on the device (one pass over the state)
    int* flag = &c->d_ctl->err;
    int bad = 0;
    SEM_CUDA(c, cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
    SEM_LAUNCH(c, launch_nonfinite_check(problem(c), flag, c->stream));
    SEM_CUDA(c, cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    SEM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (bad) {
      for (float* d : dst)
        SEM_CUDA(c, cudaMemsetAsync(d, 0, kNodeStride * static_cast<size_t>(c->nglob) * c->shots * sizeof(float), c->stream));
      SEM_CUDA(c, cudaStreamSynchronize(c->stream));
      return fail(c, SEM_EINVAL, "non-finite state value (the state was reset to zero)");
    }
  }
  return SEM_OK;
}

int sem_set_state(sem_ctx* c, const float* u, const float* v, const float* a) {
  return set_state_impl(c, u, v, a, cudaMemcpyHostToDevice);
}

int sem_set_state_dev(sem_ctx* c, const float* u, const float* v, const float* a) {
  return set_state_impl(c, u, v, a, cudaMemcpyDeviceToDevice);
}

static int get_state_impl(sem_ctx* c, float* u, float* v, float* a, cudaMemcpyKind kind) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (!c->have_mesh) return fail(c, SEM_ESTATE, "sem_set_mesh has not been called");
  int r = set_device(c);
  if (r || ((v || a) && (r = finish_state(c)))) return r;  // u is complete at any step
  const size_t n3 = 3 * static_cast<size_t>(c->nglob) * c->shots;
  const bool host = kind == cudaMemcpyDeviceToHost;
  float* dst[3] = {u, v, a};
  const float* src[3] = {c->d_u, c->d_v, c->d_a};
  float* stage = nullptr;
  if (host && (u || v || a)) SEM_CUDA(c, cudaMallocAsync(reinterpret_cast<void**>(&stage), n3 * sizeof(float), c->stream));
  int rc = SEM_OK;
  for (int q = 0; q < 3 && rc == SEM_OK; ++q) {
    if (!dst[q]) continue;
    const int* perm = (!host && c->node_order == 1) ? nullptr : c->d_perm;
    cudaError_t e =
        static_cast<cudaError_t>(launch_pack(src[q], host ? stage : dst[q], perm, c->nglob, c->shots, c->stream));
    if (e == cudaSuccess && host) e = cudaMemcpyAsync(dst[q], stage, n3 * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) rc = cuda_fail(c, e, "sem_get_state copy");
  }
  if (stage) cudaFreeAsync(stage, c->stream);
  if (rc) return rc;
  if (host) SEM_CUDA(c, cudaStreamSynchronize(c->stream));
  return SEM_OK;
}

int sem_set_step(sem_ctx* c, long long step) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (step < 0) return fail(c, SEM_EINVAL, "step must be >= 0");
  c->steps = step;
  return SEM_OK;
}

int sem_get_state(sem_ctx* c, float* u, float* v, float* a) { return get_state_impl(c, u, v, a, cudaMemcpyDeviceToHost); }

int sem_get_state_dev(sem_ctx* c, float* u, float* v, float* a) {
  return get_state_impl(c, u, v, a, cudaMemcpyDeviceToDevice);
}

int sem_step(sem_ctx* c, int nsteps) { return advance(c, nsteps, nullptr); }

int sem_run_dev(sem_ctx* c, int nsteps, float* seis_dev) { return advance(c, nsteps, seis_dev); }

int sem_run_record_snapshots(sem_ctx* c, int nsteps, float* seis_dev, float* u_dev) {
  int r = check_ready(c);
  if (r) return r;
  if (nsteps < 0) return fail(c, SEM_EINVAL, "nsteps must be >= 0");
  if (nsteps > 0 && !u_dev) return fail(c, SEM_EINVAL, "sem_run_snapshots: NULL snapshot buffer");
  if ((r = set_device(c))) return r;
  const size_t per = 3 * static_cast<size_t>(c->nglob) * c->shots;
  const int* perm = c->node_order == 1 ? nullptr : c->d_perm;
  if (!fused_sweep(c)) {
    SEM_LAUNCH(c, launch_set_ctl(c->d_ctl, c->steps, seis_dev ? nsteps : 0, seis_dev, c->stream));
    for (int k = 0; k < nsteps; ++k) {
      if (!c->pending) {
        if ((r = enqueue_first_step(c))) return r;
        c->pending = true;
      } else if ((r = enqueue_pending_step(c))) {
        return r;
      }
      SEM_LAUNCH(c, launch_pack(c->d_u, u_dev + k * per, perm, c->nglob, c->shots, c->stream));
    }
    c->steps += nsteps;
    return SEM_OK;
  }
  // fused sweep: the predictor once, then per step the receivers sample u^{n+1}, which is
  // also the snapshot (the sweep overwrites it with the next prediction), then the sweep; the
  // snapshot slot comes from the device's step counter, so the steps replay as graphs
  if (nsteps == 0) return SEM_OK;
  if ((r = finish_state(c))) return r;
  SEM_LAUNCH(c, launch_set_ctl(c->d_ctl, c->steps, seis_dev ? nsteps : 0, seis_dev, c->stream, u_dev,
                               static_cast<long long>(per)));
  SEM_LAUNCH(c, launch_predictor(problem(c), c->stream));
  auto snap_step = [&](int mode) -> int {
    DevProblem q = problem(c);
    q.nsrc = 0;
    SEM_LAUNCH(c, launch_sources_record(q, c->stream));
    SweepNewmark nm = sweep_newmark(c, mode);
    if (c->shots == 1) {  // the sweep stores u^{n+1} at each node's last touch
      nm.snap_ctl = c->d_ctl;
      nm.snap_perm = perm;
    } else {
      SEM_LAUNCH(c, launch_snapshot(c->d_u, c->d_ctl, perm, c->nglob, c->shots, c->stream));
    }
    return forces_all_colors(c, c->d_u, c->d_a, kNodeStride, c->shots, &nm);
  };
  int left = nsteps - 1;
  if (left >= kStepsPerGraph && !c->graph_snap) {
    cudaGraph_t g = nullptr;
    SEM_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int rc = SEM_OK;
    for (int s = 0; s < kStepsPerGraph && rc == SEM_OK; ++s) rc = snap_step(1);
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (rc == SEM_OK && e == cudaSuccess) e = cudaGraphInstantiate(&c->graph_snap, g, 0);
    if (g) cudaGraphDestroy(g);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(c, e, "snapshot graph");
  }
  for (; left >= kStepsPerGraph; left -= kStepsPerGraph) SEM_CUDA(c, cudaGraphLaunch(c->graph_snap, c->stream));
  for (; left > 0; --left)
    if ((r = snap_step(1))) return r;
  if ((r = snap_step(2))) return r;
  SEM_LAUNCH(c, launch_set_ctl(c->d_ctl, c->steps + nsteps, 0, nullptr, c->stream));  // forget the buffers
  c->steps += nsteps;
  return SEM_OK;
}

int sem_run_snapshots(sem_ctx* c, int nsteps, float* u_dev) {
  return sem_run_record_snapshots(c, nsteps, nullptr, u_dev);
}

int sem_check_finite(sem_ctx* c) {
  int r = check_ready(c);
  if (r) return r;
  if ((r = set_device(c))) return r;
  int* flag = &c->d_ctl->err;
  SEM_CUDA(c, cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
  SEM_LAUNCH(c, launch_nonfinite_check(problem(c), flag, c->stream));
  int bad = 0;
  SEM_CUDA(c, cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  SEM_CUDA(c, cudaStreamSynchronize(c->stream));
  if ((r = check_sweep_timeout(c))) return r;
  if (bad)
    return fail(c, SEM_EDIVERGED,
                "non-finite displacement, velocity or acceleration after " + std::to_string(c->steps) +
                    " steps (is dt above the stability limit?)");
  return SEM_OK;
}

int sem_run(sem_ctx* c, int nsteps, float* seis) {
  int r = check_ready(c);
  if (r) return r;
  if (nsteps < 0) return fail(c, SEM_EINVAL, "nsteps must be >= 0");
  if ((r = set_device(c))) return r;
  float* d_seis = nullptr;
  const size_t count = static_cast<size_t>(c->shots) * c->nrec * 3 * nsteps;
  if (seis && count) {
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d_seis), count * sizeof(float), c->stream);
    if (e != cudaSuccess) return fail(c, SEM_ENOMEM, std::string("seismogram buffer: ") + cudaGetErrorString(e));
  }
  r = advance(c, nsteps, d_seis);
  if (r == SEM_OK && d_seis) {
    cudaError_t e = cudaMemcpyAsync(seis, d_seis, count * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) r = cuda_fail(c, e, "seismogram copy");
  }
  if (d_seis) cudaFreeAsync(d_seis, c->stream);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (r == SEM_OK && e != cudaSuccess) r = cuda_fail(c, e, "sem_run");
  if (r == SEM_OK) r = sem_check_finite(c);
  return r;
}

int sem_apply_stiffness_strided(sem_ctx* c, const float* u_dev, float* f_dev, int node_stride) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (!c->have_mat) return fail(c, SEM_ESTATE, "sem_set_material has not been called");
  if (!u_dev || !f_dev) return fail(c, SEM_EINVAL, "sem_apply_stiffness: NULL pointer");
  if (node_stride != 3 && node_stride != 4) return fail(c, SEM_EINVAL, "node_stride must be 3 or 4");
  if (node_stride == 4 && ((reinterpret_cast<uintptr_t>(u_dev) | reinterpret_cast<uintptr_t>(f_dev)) & 15))
    return fail(c, SEM_EINVAL, "node_stride 4 needs 16-byte aligned arrays");
  const size_t bytes = node_stride * static_cast<size_t>(c->nglob) * sizeof(float);
  const char* a = reinterpret_cast<const char*>(u_dev);
  const char* b = reinterpret_cast<const char*>(f_dev);
  if (a < b + bytes && b < a + bytes) return fail(c, SEM_EINVAL, "u_dev and f_dev overlap");
  int r = set_device(c);
  if (r) return r;
  return forces_all_colors(c, u_dev, f_dev, node_stride, 1);
}

int sem_node_order(sem_ctx* c, int32_t* perm) {
  if (!c || !perm) return fail(c, SEM_EINVAL, "sem_node_order: bad arguments");
  if (!c->have_mesh) return fail(c, SEM_ESTATE, "sem_set_mesh has not been called");
  std::memcpy(perm, c->perm.data(), c->perm.size() * sizeof(int32_t));
  return SEM_OK;
}

int sem_init_acceleration(sem_ctx* c) {
  int r = check_ready(c);
  if (r) return r;
  if ((r = set_device(c)) || (r = finish_state(c))) return r;
  if ((r = forces_all_colors(c, c->d_u, c->d_a, kNodeStride, c->shots))) return r;  // a = -K u
  DevProblem p = problem(c);
  p.dt = 0.0;  // the corrector with dt = 0 only scales a by 1/M and leaves v as it is
  SEM_LAUNCH(c, launch_corrector(p, c->stream));
  return SEM_OK;
}

int sem_apply_stiffness(sem_ctx* c, const float* u_dev, float* f_dev) {
  return sem_apply_stiffness_strided(c, u_dev, f_dev, 3);
}

int sem_energy(sem_ctx* c, double* out) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (!c->have_mat) return fail(c, SEM_ESTATE, "sem_set_material has not been called");
  if (!out) return fail(c, SEM_EINVAL, "sem_energy: NULL output");
  int r = set_device(c);
  if (r || (r = finish_state(c))) return r;
  const size_t nf = kNodeStride * static_cast<size_t>(c->nglob) * c->shots;
  if (!c->d_f) {
    if ((r = dev_alloc(c, &c->d_f, nf)) || (r = dev_alloc(c, &c->d_partials, 2 * static_cast<size_t>(kEnergyBlocks))))
      return r;
    SEM_CUDA(c, cudaMemsetAsync(c->d_f, 0, nf * sizeof(float), c->stream));
  }
  if ((r = forces_all_colors(c, c->d_u, c->d_f, kNodeStride, c->shots))) return r;
  SEM_LAUNCH(c, launch_energy_partials(c->d_u, c->d_v, c->d_f, c->d_minv, c->nglob, c->shots, c->d_partials,
                                       kEnergyBlocks,
                                       c->stream));
  std::vector<double> part(2 * kEnergyBlocks);
  SEM_CUDA(c, cudaMemcpyAsync(part.data(), c->d_partials, part.size() * sizeof(double), cudaMemcpyDeviceToHost,
                              c->stream));
  SEM_CUDA(c, cudaStreamSynchronize(c->stream));
  double kin = 0.0, pot = 0.0;
  for (int b = 0; b < kEnergyBlocks; ++b) {
    kin += part[2 * b];
    pot += part[2 * b + 1];
  }
  out[0] = 0.5 * kin;
  out[1] = -0.5 * pot;  // f = -K u
  return SEM_OK;
}

int sem_sync(sem_ctx* c) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  int r = set_device(c);
  if (r) return r;
  SEM_CUDA(c, cudaStreamSynchronize(c->stream));
  return check_sweep_timeout(c);
}

int sem_info(sem_ctx* c, int64_t* out) {
  if (!c || !out) return fail(c, SEM_EINVAL, "sem_info: bad arguments");
  out[0] = c->nspec;
  out[1] = c->nglob;
  out[2] = c->ngll;
  out[3] = c->ncolors;
  out[4] = c->steps;
  out[5] = static_cast<int64_t>(c->dev_bytes);
  out[6] = c->shots;
  out[7] = c->slabs;
  out[8] = static_cast<int64_t>(c->sweep_off.size()) - 1;
  return SEM_OK;
}

int sem_patch_info(sem_ctx* c, int64_t* out) {
  if (!c || !out) return fail(c, SEM_EINVAL, "sem_patch_info: bad arguments");
  if (!c->have_mesh) return fail(c, SEM_ESTATE, "sem_set_mesh has not been called");
  const PatchShape shape = c->shape;
  out[0] = c->npatch;
  out[1] = static_cast<int64_t>(c->pcolor_off.size()) - 1;
  out[2] = c->pmax_nodes;
  out[3] = c->ptables;
  out[4] = shape.bx;
  out[5] = shape.by;
  out[6] = shape.bz;
  out[7] = c->assembly;
  return SEM_OK;
}

int sem_color_counts(sem_ctx* c, int32_t* counts) {
  if (!c || !counts) return fail(c, SEM_EINVAL, "sem_color_counts: bad arguments");
  if (!c->have_mesh) return fail(c, SEM_ESTATE, "sem_set_mesh has not been called");
  for (int k = 0; k < c->ncolors; ++k) counts[k] = c->color_count[k];
  return SEM_OK;
}

int sem_adjoint_begin(sem_ctx* c) {
  int r = check_ready(c);
  if (r) return r;
  if (c->shots != 1) return fail(c, SEM_EINVAL, "the adjoint runs one shot at a time (sem_set_shots(ctx, 1))");
  if ((r = set_device(c))) return r;
  const size_t nf = kNodeStride * static_cast<size_t>(c->nglob);
  const size_t nloc = static_cast<size_t>(c->nspec) * c->ngll * c->ngll * c->ngll;
  if (!c->d_lam) {
    if ((r = dev_alloc(c, &c->d_lam, nf)) || (r = dev_alloc(c, &c->d_lam_old, nf)) ||
        (r = dev_alloc(c, &c->d_lamF, nf)) || (r = dev_alloc(c, &c->d_grad, 3 * nloc)) ||
        (r = dev_alloc(c, &c->d_grad32, 3 * nloc)))
      return r;
  }
  SEM_CUDA(c, cudaMemsetAsync(c->d_lam, 0, nf * sizeof(float), c->stream));
  SEM_CUDA(c, cudaMemsetAsync(c->d_lam_old, 0, nf * sizeof(float), c->stream));
  SEM_CUDA(c, cudaMemsetAsync(c->d_grad, 0, 3 * nloc * sizeof(double), c->stream));
  SEM_CUDA(c, cudaMemsetAsync(c->d_grad32, 0, 3 * nloc * sizeof(float), c->stream));
  c->since_flush = 0;
  c->adjoint = true;
  return SEM_OK;
}

// Whether adjoint steps run the leapfrog inside the sweep of lam (the per-colour patch
// sweep with SEM_OPT_FUSED_NEWMARK not 0, and the receivers' patch lists built).
bool fused_adjoint(const sem_ctx* c) {
  return c->fuse_newmark != 0 && c->assembly == 0 && c->npatch > 0 && (c->nrec == 0 || c->d_precv_range);
}

// One adjoint step: the sweep of lam with, at each node's last touch, the residual injection
// and the leapfrog (or, unfused, the sweep, then the injection and leapfrog passes). G_dev is
// the residual [nrec][3]; with idx it is taken from the device's adjoint counter (G_dev then
// only says whether there is one).
static int adjoint_sweep_step(sem_ctx* c, const float* G_dev, const DevCtl* idx) {
  if (fused_adjoint(c)) {
    SweepNewmark nm{};
    nm.mode = 3;
    nm.u = c->d_lam;
    nm.lam_old = c->d_lam_old;
    nm.minv = c->d_minv;
    nm.recv_range = c->nrec > 0 && G_dev ? c->d_precv_range : nullptr;
    nm.recv = c->d_precv;
    nm.G = idx ? nullptr : G_dev;
    nm.idx = G_dev ? idx : nullptr;
    nm.inv_dt2 = static_cast<float>(1.0 / (c->dt * c->dt));
    nm.dt2 = static_cast<float>(c->dt * c->dt);
    if (int r = forces_all_colors(c, c->d_lam, c->d_lamF, kNodeStride, 1, &nm)) return r;
  } else {
    if (int r = forces_all_colors(c, c->d_lam, c->d_lamF, kNodeStride, 1)) return r;
    SEM_LAUNCH(c, launch_adjoint_update(c->d_lamF, G_dev, c->d_rnode, c->d_roff, c->d_rlist, c->nrnodes, c->d_lam,
                                        c->d_lam_old, c->d_minv, c->nglob, c->dt, c->stream, idx));
  }
  std::swap(c->d_lam, c->d_lam_old);  // lam <- lam^{m-1}, lam_old <- lam^m
  return SEM_OK;
}

int sem_adjoint_step(sem_ctx* c, const float* G_dev) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (!c->adjoint) return fail(c, SEM_ESTATE, "sem_adjoint_begin has not been called");
  int r = set_device(c);
  if (r) return r;
  return adjoint_sweep_step(c, G_dev, nullptr);
}

int sem_adjoint_accumulate(sem_ctx* c, const float* u_lo, const float* u_mid, const float* u_hi) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (!c->adjoint) return fail(c, SEM_ESTATE, "sem_adjoint_begin has not been called");
  if (!u_lo || !u_mid || !u_hi) return fail(c, SEM_EINVAL, "sem_adjoint_accumulate: NULL snapshot");
  int r = set_device(c);
  if (r) return r;
  const size_t nloc = static_cast<size_t>(c->nspec) * c->ngll * c->ngll * c->ngll;
  SEM_LAUNCH(c, launch_sensitivity(c->ngll, c->d_rec, c->node_order == 1 ? nullptr : c->d_perm, c->d_lam, u_lo, u_mid,
                                    u_hi, c->d_grad32, c->d_grad32 + nloc, c->d_grad32 + 2 * nloc, c->nspec, -1.0,
                                    -c->dt * c->dt, c->stream));
  if (++c->since_flush >= kFlushEvery) return flush_gradients(c);
  return SEM_OK;
}

// One adjoint step (sweep of lam, residual injection and leapfrog, sensitivity terms) with
// its residual and snapshots named by the device's adjoint counter, which it then lowers.
// Step k of a run of indexed adjoint steps: the sweep of lam on the context's stream, the
// sensitivity terms on the auxiliary stream as soon as the sweep is done, so that they overlap
// the next step's sweep. That sweep only writes the buffer of lam^{m+1}, which these terms do
// not read; the sweep after it overwrites lam^{m-1}, so it waits for them (ev_sens ring).
static int adjoint_indexed_step(sem_ctx* c, bool hasG, int k) {
  if (k >= 2) SEM_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_sens[k & 1], 0));
  // (with the counter the residual comes from it; the pointer only marks that there is one)
  if (int r = adjoint_sweep_step(c, hasG ? c->d_lamF : nullptr, c->d_ctl)) return r;
  SEM_LAUNCH(c, launch_adjoint_next(c->d_ctl, c->stream));
  SEM_CUDA(c, cudaEventRecord(c->ev_sweep[k & 1], c->stream));
  SEM_CUDA(c, cudaStreamWaitEvent(c->aux, c->ev_sweep[k & 1], 0));
  const size_t nloc = static_cast<size_t>(c->nspec) * c->ngll * c->ngll * c->ngll;
  SEM_LAUNCH(c, launch_sensitivity(c->ngll, c->d_rec, c->node_order == 1 ? nullptr : c->d_perm, c->d_lam, nullptr,
                                    nullptr, nullptr, c->d_grad32, c->d_grad32 + nloc, c->d_grad32 + 2 * nloc,
                                    c->nspec, -1.0, -c->dt * c->dt, c->aux, c->d_ctl));
  SEM_LAUNCH(c, launch_adjoint_next(c->d_ctl, c->aux, true));
  SEM_CUDA(c, cudaEventRecord(c->ev_sens[k & 1], c->aux));
  return SEM_OK;
}

// The auxiliary stream and events of the overlapped adjoint steps.
static int adjoint_aux(sem_ctx* c) {
  if (c->aux) return SEM_OK;
  SEM_CUDA(c, cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking));
  for (int k = 0; k < 2; ++k) {
    SEM_CUDA(c, cudaEventCreateWithFlags(&c->ev_sweep[k], cudaEventDisableTiming));
    SEM_CUDA(c, cudaEventCreateWithFlags(&c->ev_sens[k], cudaEventDisableTiming));
  }
  return SEM_OK;
}

static int adjoint_segment_steps(sem_ctx* c, int count, const float* G_dev, const float* u_dev) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (!c->adjoint) return fail(c, SEM_ESTATE, "sem_adjoint_begin has not been called");
  if (count < 0) return fail(c, SEM_EINVAL, "count must be >= 0");
  if (count > 0 && !u_dev) return fail(c, SEM_EINVAL, "sem_adjoint_segment: NULL snapshots");
  const size_t n3 = 3 * static_cast<size_t>(c->nglob);
  const size_t gstep = 3 * static_cast<size_t>(c->nrec);
  int j0 = count;
  if (count >= kStepsPerGraph) {
    // steps in graphs of kStepsPerGraph (an even count: the lam buffers end in their roles),
    // residuals and snapshots named by the device counter; the same kernels and sums as the
    // steps one by one below
    const bool hasG = G_dev != nullptr;
    if (int r = adjoint_aux(c)) return r;
    SEM_LAUNCH(c, launch_adjoint_index(c->d_ctl, G_dev, u_dev, static_cast<long long>(n3), static_cast<int>(gstep),
                                       count, c->stream));
    if (c->graph_adj && (c->graph_adj_lam != c->d_lam || c->graph_adj_G != hasG)) {
      cudaGraphExecDestroy(c->graph_adj);
      c->graph_adj = nullptr;
    }
    if (!c->graph_adj) {
      c->graph_adj_lam = c->d_lam;
      c->graph_adj_G = hasG;
      cudaGraph_t g = nullptr;
      SEM_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
      int rc = SEM_OK;
      for (int s = 0; s < kStepsPerGraph && rc == SEM_OK; ++s) rc = adjoint_indexed_step(c, hasG, s);
      // join the auxiliary branch (its last terms) before the graph ends
      if (rc == SEM_OK && cudaStreamWaitEvent(c->stream, c->ev_sens[(kStepsPerGraph - 1) & 1], 0) != cudaSuccess)
        rc = fail(c, SEM_ECUDA, "adjoint graph join");
      cudaError_t e = cudaStreamEndCapture(c->stream, &g);
      if (rc == SEM_OK && e == cudaSuccess) e = cudaGraphInstantiate(&c->graph_adj, g, 0);
      if (g) cudaGraphDestroy(g);
      if (rc) return rc;
      if (e != cudaSuccess) return cuda_fail(c, e, "adjoint graph");
    }
    for (; j0 >= kStepsPerGraph; j0 -= kStepsPerGraph) {
      SEM_CUDA(c, cudaGraphLaunch(c->graph_adj, c->stream));
      c->since_flush += kStepsPerGraph;
      if (c->since_flush >= kFlushEvery)
        if (int r = flush_gradients(c)) return r;
    }
  }
  for (int j = j0; j >= 1; --j) {
    int r = sem_adjoint_step(c, G_dev ? G_dev + (j - 1) * gstep : nullptr);
    if (r) return r;
    if ((r = sem_adjoint_accumulate(c, u_dev + (j - 1) * n3, u_dev + j * n3, u_dev + (j + 1) * n3))) return r;
  }
  return SEM_OK;
}

int sem_adjoint_segment(sem_ctx* c, int count, const float* G_dev, const float* u_dev) {
  int rs = adjoint_segment_steps(c, count, G_dev, u_dev);
  if (rs) return rs;
  return flush_gradients(c);
}

int sem_adjoint_gradients(sem_ctx* c, double* g_rho, double* g_kappa, double* g_mu) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (!c->adjoint) return fail(c, SEM_ESTATE, "sem_adjoint_begin has not been called");
  int r = set_device(c);
  if (r || (r = flush_gradients(c))) return r;
  const int n = c->ngll, np = n * n * n, nl = n * n;
  const size_t nloc = static_cast<size_t>(c->nspec) * np;
  std::vector<double> h(3 * nloc);
  SEM_CUDA(c, cudaMemcpyAsync(h.data(), c->d_grad, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  SEM_CUDA(c, cudaStreamSynchronize(c->stream));
  double* outs[3] = {g_rho, g_kappa, g_mu};
  for (int f = 0; f < 3; ++f) {
    if (!outs[f]) continue;
    for (int s = 0; s < c->nspec; ++s) {
      const size_t caller = static_cast<size_t>(c->order[s]) * np;
      const double* src = h.data() + f * nloc + static_cast<size_t>(s) * np;
      for (int q = 0; q < np; ++q) {
        const int i = q / nl, line = q - i * nl;
        outs[f][caller + i + n * line] = src[q];
      }
    }
  }
  return SEM_OK;
}

int sem_tune_patch_shape(sem_ctx* c, int nspec, int nglob, const int32_t* ibool, const double* xyz,
                         const double* ctrl, const float* rho, const float* vp, const float* vs, int reps,
                         int max_shapes, int32_t* shapes_out, double* ms_out, int* nshapes_out) {
  if (!c) return fail(nullptr, SEM_EINVAL, "null context");
  if (reps < 1 || !ibool || (!xyz) == (!ctrl) || !rho || !vp || !vs)
    return fail(c, SEM_EINVAL, "sem_tune_patch_shape: bad arguments");
  PatchShape def;
  if (patch_shape(c->ngll, &def)) return fail(c, SEM_EINVAL, "no patch kernel for this order");
  const int pe = def.bx * def.by * def.bz;  // elements a patch CTA holds at this order
  std::vector<PatchShape> cand;
  for (int bz = 1; bz <= pe; ++bz)
    for (int by = 1; by <= pe; ++by)
      for (int bx = 1; bx <= pe; ++bx)
        if (bx * by * bz == pe && bx <= 16 && by <= 16 && bz <= 16) cand.push_back(PatchShape{bx, by, bz});
  std::vector<double> ms(cand.size(), 0.0);
  int best = -1;
  for (size_t k = 0; k < cand.size(); ++k) {
    sem_ctx* t = nullptr;
    int r = sem_create(&t, c->ngll, c->device, c->stream);
    if (r) return fail(c, r, "sem_tune_patch_shape: " + g_err);
    const long long code = cand[k].bx | (cand[k].by << 8) | (cand[k].bz << 16);
    double dt = 0.0, prof[2] = {0.0, 0.0};
    if (!r) r = sem_set_option(t, SEM_OPT_PATCH_SHAPE, code);
    if (!r) r = xyz ? sem_set_mesh(t, nspec, nglob, ibool, xyz) : sem_set_mesh_corners(t, nspec, nglob, ibool, ctrl);
    if (!r) r = sem_set_material(t, rho, vp, vs);
    if (!r) r = sem_suggest_dt(t, 0.4, &dt);
    if (!r) r = sem_set_dt(t, dt);
    if (!r) r = sem_set_state(t, nullptr, nullptr, nullptr);
    if (!r) r = sem_profile_steps(t, 2, prof);  // warm-up
    if (!r) r = sem_profile_steps(t, reps, prof);
    const std::string msg = r ? t->err : std::string();
    sem_destroy(t);
    if (r) return fail(c, r, "sem_tune_patch_shape: " + msg);
    ms[k] = prof[0];
    if (best < 0 || ms[k] < ms[best]) best = static_cast<int>(k);
  }
  c->shape_opt = cand[best];
  const int nout = std::min<int>(max_shapes, static_cast<int>(cand.size()));
  for (int k = 0; k < nout; ++k) {
    if (shapes_out) shapes_out[k] = cand[k].bx | (cand[k].by << 8) | (cand[k].bz << 16);
    if (ms_out) ms_out[k] = ms[k];
  }
  if (nshapes_out) *nshapes_out = static_cast<int>(cand.size());
  return SEM_OK;
}

int sem_profile_steps(sem_ctx* c, int nsteps, double* ms_out) {
  int r = check_ready(c);
  if (r) return r;
  if (nsteps < 1 || !ms_out) return fail(c, SEM_EINVAL, "sem_profile_steps: nsteps >= 1 and ms_out required");
  if ((r = set_device(c))) return r;
  const bool fused = fused_sweep(c);
  if (fused && (r = finish_state(c))) return r;
  SEM_LAUNCH(c, launch_set_ctl(c->d_ctl, c->steps, 0, nullptr, c->stream));
  std::vector<cudaEvent_t> ev(2 * static_cast<size_t>(nsteps) + 2, nullptr);
  int rc = SEM_OK;
  for (cudaEvent_t& e : ev)
    if (rc == SEM_OK && cudaEventCreate(&e) != cudaSuccess) rc = fail(c, SEM_ECUDA, "cudaEventCreate");
  auto mark = [&](size_t k) {
    if (rc == SEM_OK && cudaEventRecord(ev[k], c->stream) != cudaSuccess) rc = fail(c, SEM_ECUDA, "cudaEventRecord");
  };
  // event 0: the start, 1 + 2s: before step s's force sweep, 2 + 2s: after it, the last: the end
  const DevProblem p = problem(c);
  mark(0);
  if (rc == SEM_OK && fused) rc = launch_predictor(p, c->stream) ? fail(c, SEM_ECUDA, "predictor launch") : SEM_OK;
  if (rc == SEM_OK && !fused && !c->pending)
    rc = launch_predictor(p, c->stream) ? fail(c, SEM_ECUDA, "predictor launch") : SEM_OK;
  for (int s = 0; s < nsteps && rc == SEM_OK; ++s) {
    if (fused) {
      DevProblem q = p;
      q.nsrc = 0;
      if (launch_sources_record(q, c->stream)) rc = fail(c, SEM_ECUDA, "receiver launch");
      mark(1 + 2 * s);
      const SweepNewmark nm = sweep_newmark(c, s + 1 < nsteps ? 1 : 2);
      if (rc == SEM_OK) rc = forces_all_colors(c, c->d_u, c->d_a, kNodeStride, c->shots, &nm);
      mark(2 + 2 * s);
    } else {
      if (s > 0 || c->pending)
        if (launch_fused_newmark(p, c->stream)) rc = fail(c, SEM_ECUDA, "Newmark launch");
      mark(1 + 2 * s);
      if (rc == SEM_OK) rc = forces_all_colors(c, c->d_u, c->d_a, kNodeStride, c->shots);
      mark(2 + 2 * s);
      if (rc == SEM_OK && launch_sources_record(p, c->stream)) rc = fail(c, SEM_ECUDA, "source launch");
    }
  }
  mark(ev.size() - 1);
  double sweep = 0.0, total = 0.0;
  if (rc == SEM_OK && cudaEventSynchronize(ev.back()) != cudaSuccess) rc = fail(c, SEM_ECUDA, "sem_profile_steps");
  for (int s = 0; s < nsteps && rc == SEM_OK; ++s) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, ev[1 + 2 * s], ev[2 + 2 * s]) != cudaSuccess) rc = fail(c, SEM_ECUDA, "event time");
    sweep += t;
  }
  float t = 0.f;
  if (rc == SEM_OK && cudaEventElapsedTime(&t, ev[0], ev.back()) != cudaSuccess) rc = fail(c, SEM_ECUDA, "event time");
  total = t;
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  if (rc != SEM_OK) return rc;
  if (!fused) c->pending = true;
  c->steps += nsteps;
  ms_out[0] = sweep / nsteps;
  ms_out[1] = (total - sweep) / nsteps;
  return SEM_OK;
}

int sem_autotune(sem_ctx* c, int reps, double* ms_out, int* choice_out) {
  int r = check_ready(c);
  if (r) return r;
  if (reps < 1) return fail(c, SEM_EINVAL, "sem_autotune: reps must be >= 1");
  if ((r = set_device(c))) return r;
  if ((r = finish_state(c))) return r;  // the timing sweeps read u and write scratch only
  const size_t nf = kNodeStride * static_cast<size_t>(c->nglob) * c->shots;
  float* f = nullptr;
  SEM_CUDA(c, cudaMallocAsync(reinterpret_cast<void**>(&f), nf * sizeof(float), c->stream));
  cudaEvent_t ev[2] = {nullptr, nullptr};
  double ms[2] = {0.0, 0.0};
  const int keep = c->variant;
  int rc = SEM_OK;
  for (int k = 0; k < 2 && rc == SEM_OK; ++k) if (cudaEventCreate(&ev[k]) != cudaSuccess) rc = fail(c, SEM_ECUDA, "cudaEventCreate");
  for (int v = 1; v <= 2 && rc == SEM_OK; ++v) {  // 1 line owners, 2 per point
    c->variant = v;
    rc = forces_all_colors(c, c->d_u, f, kNodeStride, c->shots);  // warm-up
    if (rc == SEM_OK && cudaEventRecord(ev[0], c->stream) != cudaSuccess) rc = fail(c, SEM_ECUDA, "cudaEventRecord");
    for (int i = 0; i < reps && rc == SEM_OK; ++i) rc = forces_all_colors(c, c->d_u, f, kNodeStride, c->shots);
    float t = 0.f;
    if (rc == SEM_OK && (cudaEventRecord(ev[1], c->stream) != cudaSuccess || cudaEventSynchronize(ev[1]) != cudaSuccess ||
                         cudaEventElapsedTime(&t, ev[0], ev[1]) != cudaSuccess))
      rc = fail(c, SEM_ECUDA, "sem_autotune timing");
    ms[v - 1] = static_cast<double>(t) / reps;
  }
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  cudaFreeAsync(f, c->stream);
  if (rc != SEM_OK) {
    c->variant = keep;
    return rc;
  }
  c->variant = ms[0] <= ms[1] ? 1 : 2;
  drop_graph(c);
  if (ms_out) {
    ms_out[0] = ms[0];
    ms_out[1] = ms[1];
  }
  if (choice_out) *choice_out = c->variant;
  return SEM_OK;
}

}  // extern "C"

// ---- groups of contexts stepped together ------------------------------------------------
struct sem_group {
  std::vector<sem_ctx*> ctx;
  int device = 0;
  cudaStream_t stream = nullptr;           // the group's launch stream
  std::vector<cudaStream_t> branch;        // one per context, used while capturing
  std::vector<cudaEvent_t> ev;             // fork/join events: [0] fork, [1 + i] join of branch i
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // kStepsPerGraph steps of every context; one step
  std::vector<unsigned long long> gen;     // the contexts' generations the graphs were built on
  std::string err;
  int mode = 0;                            // SEM_GROUP_MODE: 0 graph branches, 1 persistent sweeps
  unsigned int stall = 0;                  // SEM_GROUP_STALL_TEST (one-shot, eager steps only)
  bool persistent = false;                 // the graphs hold persistent sweeps
  struct Sweep {                           // one persistent sweep: the contexts of one order and form
    int ngll = 0, variant = 0, nseg = 0, nitems = 0, nmodels = 0;
    GroupModel* d_models = nullptr;
    GroupSeg* d_segs = nullptr;
  };
  std::vector<Sweep> sweeps;
  GroupSync* d_sync = nullptr;
};

namespace {

int group_fail(sem_group* g, int code, const std::string& msg) {
  if (g)
    g->err = msg;
  else
    g_err = msg;
  return code;
}

void group_drop(sem_group* g) {
  for (auto& x : g->graph)
    if (x) {
      cudaGraphExecDestroy(x);
      x = nullptr;
    }
  for (auto& sw : g->sweeps) {
    if (sw.d_models) cudaFree(sw.d_models);
    if (sw.d_segs) cudaFree(sw.d_segs);
  }
  g->sweeps.clear();
}

// Whether the group's steps can run as persistent sweeps: every context one shot on the
// per-colour patch assembly, at most kMaxSweepColors patch colours.
bool group_persistent_ok(const sem_group* g) {
  if (g->mode != 1 || g->ctx.size() > static_cast<size_t>(kMaxGroupModels)) return false;
  for (const sem_ctx* c : g->ctx)
    if (c->shots != 1 || c->assembly != 0 || c->npatch <= 0 ||
        c->pcolor_off.size() > static_cast<size_t>(kMaxSweepColors) + 1)
      return false;
  return true;
}

// The device tables of the persistent sweeps: contexts grouped by (order, contraction form);
// per sweep its models and its runs of items, colour-major (colour c of every model before
// colour c + 1).
int group_tables(sem_group* g) {
  std::map<std::pair<int, int>, std::vector<int>> by;
  for (size_t i = 0; i < g->ctx.size(); ++i) by[{g->ctx[i]->ngll, g->ctx[i]->variant}].push_back(static_cast<int>(i));
  for (const auto& kv : by) {
    sem_group::Sweep sw;
    sw.ngll = kv.first.first;
    sw.variant = kv.first.second;
    std::vector<GroupModel> models;
    int maxc = 0;
    for (int i : kv.second) {
      const sem_ctx* c = g->ctx[i];
      GroupModel m{};
      m.rec = c->d_rec;
      m.desc = c->d_pdesc;
      m.slots = c->d_pslots;
      m.words = c->d_pwords;
      m.u = c->d_u;
      m.f = c->d_a;
      m.color_end = c->d_pcolor_end;
      m.ncolors = static_cast<int>(c->pcolor_off.size()) - 1;
      maxc = std::max(maxc, m.ncolors);
      models.push_back(m);
    }
    std::vector<GroupSeg> segs;
    int items = 0;
    for (int col = 0; col < maxc; ++col)
      for (size_t k = 0; k < kv.second.size(); ++k) {
        const sem_ctx* c = g->ctx[kv.second[k]];
        if (col >= models[k].ncolors) continue;
        const int n = c->pcolor_off[col + 1] - c->pcolor_off[col];
        if (n <= 0) continue;
        segs.push_back(GroupSeg{items, static_cast<int>(k), col, c->pcolor_off[col]});
        items += n;
      }
    sw.nmodels = static_cast<int>(models.size());
    sw.nseg = static_cast<int>(segs.size());
    sw.nitems = items;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&sw.d_models), models.size() * sizeof(GroupModel));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&sw.d_segs), std::max<size_t>(1, segs.size()) * sizeof(GroupSeg));
    if (e == cudaSuccess)
      e = cudaMemcpy(sw.d_models, models.data(), models.size() * sizeof(GroupModel), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !segs.empty())
      e = cudaMemcpy(sw.d_segs, segs.data(), segs.size() * sizeof(GroupSeg), cudaMemcpyHostToDevice);
    g->sweeps.push_back(sw);
    if (e != cudaSuccess) return group_fail(g, SEM_ECUDA, std::string("group tables: ") + cudaGetErrorString(e));
  }
  if (!g->d_sync) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&g->d_sync), sizeof(GroupSync));
    if (e == cudaSuccess) e = cudaMemset(g->d_sync, 0, sizeof(GroupSync));
    if (e != cudaSuccess) return group_fail(g, SEM_ECUDA, std::string("group counters: ") + cudaGetErrorString(e));
  }
  return SEM_OK;
}

// One pending step of every context on the group's stream with the force sweeps persistent:
// the contexts' Newmark passes, one sweep launch per (order, form), the contexts' sources.
int group_enqueue_persistent_step(sem_group* g, unsigned int stall) {
  for (sem_ctx* c : g->ctx)
    if (launch_fused_newmark(problem(c), g->stream)) return group_fail(g, SEM_ECUDA, "group Newmark pass");
  for (const auto& sw : g->sweeps) {
    GroupLaunch L{};
    L.models = sw.d_models;
    L.segs = sw.d_segs;
    L.nseg = sw.nseg;
    L.nitems = sw.nitems;
    L.nmodels = sw.nmodels;
    L.variant = sw.variant;
    L.stall = stall;
    L.sync = g->d_sync;
    if (launch_group_sweep(sw.ngll, L, g->stream)) return group_fail(g, SEM_ECUDA, "group sweep launch");
  }
  for (sem_ctx* c : g->ctx)
    if (launch_sources_record(problem(c), g->stream)) return group_fail(g, SEM_ECUDA, "group sources");
  return SEM_OK;
}

// A graph of `steps` persistent group steps.
int group_build_persistent(sem_group* g, int which, int steps) {
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return group_fail(g, SEM_ECUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
  int rc = SEM_OK;
  for (int s = 0; s < steps && rc == SEM_OK; ++s) rc = group_enqueue_persistent_step(g, 0u);
  e = cudaStreamEndCapture(g->stream, &graph);
  if (rc == SEM_OK && e != cudaSuccess) rc = group_fail(g, SEM_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
  if (rc == SEM_OK) {
    e = cudaGraphInstantiate(&g->graph[which], graph, 0);
    if (e != cudaSuccess) rc = group_fail(g, SEM_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  }
  if (graph) cudaGraphDestroy(graph);
  return rc;
}

// One graph advancing every context by `steps` pending steps, each context on a branch of
// its own so that the contexts' kernels may run side by side.
int group_build(sem_group* g, int which, int steps) {
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return group_fail(g, SEM_ECUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
  int rc = SEM_OK;
  if (cudaEventRecord(g->ev[0], g->stream) != cudaSuccess) rc = group_fail(g, SEM_ECUDA, "fork event");
  for (size_t i = 0; i < g->ctx.size() && rc == SEM_OK; ++i) {
    sem_ctx* c = g->ctx[i];
    if (cudaStreamWaitEvent(g->branch[i], g->ev[0], 0) != cudaSuccess) {
      rc = group_fail(g, SEM_ECUDA, "branch wait");
      break;
    }
    cudaStream_t own = c->stream;
    c->stream = g->branch[i];
    for (int s = 0; s < steps && rc == SEM_OK; ++s)
      if (enqueue_pending_step(c) != SEM_OK) rc = group_fail(g, SEM_ECUDA, "capture of a step: " + c->err);
    c->stream = own;
    if (rc == SEM_OK && (cudaEventRecord(g->ev[1 + i], g->branch[i]) != cudaSuccess ||
                         cudaStreamWaitEvent(g->stream, g->ev[1 + i], 0) != cudaSuccess))
      rc = group_fail(g, SEM_ECUDA, "join event");
  }
  e = cudaStreamEndCapture(g->stream, &graph);
  if (rc == SEM_OK && e != cudaSuccess) rc = group_fail(g, SEM_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
  if (rc == SEM_OK) {
    e = cudaGraphInstantiate(&g->graph[which], graph, 0);
    if (e != cudaSuccess) rc = group_fail(g, SEM_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  }
  if (graph) cudaGraphDestroy(graph);
  return rc;
}

}  // namespace

extern "C" {

int sem_group_create(sem_group** out, int n, sem_ctx* const* ctxs) {
  if (!out || n < 1 || !ctxs) return group_fail(nullptr, SEM_EINVAL, "sem_group_create: bad arguments");
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return group_fail(nullptr, SEM_EINVAL, "sem_group_create: NULL context");
    if (ctxs[i]->device != ctxs[0]->device)
      return group_fail(nullptr, SEM_EINVAL, "sem_group_create: contexts on different devices");
    for (int k = 0; k < i; ++k)
      if (ctxs[k] == ctxs[i]) return group_fail(nullptr, SEM_EINVAL, "sem_group_create: a context appears twice");
  }
  sem_group* g = new sem_group();
  g->ctx.assign(ctxs, ctxs + n);
  g->device = ctxs[0]->device;
  cudaError_t e = cudaSetDevice(g->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
  g->branch.assign(n, nullptr);
  g->ev.assign(n + 1, nullptr);
  for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&g->branch[i], cudaStreamNonBlocking);
  for (int i = 0; i <= n && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&g->ev[i], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    std::string msg = std::string("sem_group_create: ") + cudaGetErrorString(e);
    sem_group_destroy(g);
    return group_fail(nullptr, SEM_ECUDA, msg);
  }
  *out = g;
  return SEM_OK;
}

int sem_group_destroy(sem_group* g) {
  if (!g) return SEM_OK;
  cudaSetDevice(g->device);
  if (g->stream) cudaStreamSynchronize(g->stream);
  group_drop(g);
  if (g->d_sync) cudaFree(g->d_sync);
  for (cudaEvent_t e : g->ev)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t s : g->branch)
    if (s) cudaStreamDestroy(s);
  if (g->stream) cudaStreamDestroy(g->stream);
  delete g;
  return SEM_OK;
}

int sem_group_step(sem_group* g, int nsteps) {
  if (!g) return group_fail(nullptr, SEM_EINVAL, "null group");
  if (nsteps < 0) return group_fail(g, SEM_EINVAL, "nsteps must be >= 0");
  if (nsteps == 0) return SEM_OK;
  cudaError_t e = cudaSetDevice(g->device);
  if (e != cudaSuccess) return group_fail(g, SEM_ECUDA, cudaGetErrorString(e));
  const size_t n = g->ctx.size();
  // each context: step counter, then one eager step on its own stream (a first step from a
  // complete state, or a pending one), so that all of them continue in pending form
  for (size_t i = 0; i < n; ++i) {
    sem_ctx* c = g->ctx[i];
    int r = check_ready(c);
    if (r) return group_fail(g, r, "context " + std::to_string(i) + ": " + c->err);
    if ((r = advance(c, 1, nullptr, false))) return group_fail(g, r, "context " + std::to_string(i) + ": " + c->err);
    if (cudaEventRecord(g->ev[1 + i], c->stream) != cudaSuccess || cudaStreamWaitEvent(g->stream, g->ev[1 + i], 0) != cudaSuccess)
      return group_fail(g, SEM_ECUDA, "ordering the group after its contexts");
  }
  int left = nsteps - 1;
  const bool persistent = group_persistent_ok(g);
  bool stale = g->gen.size() != n || g->persistent != persistent;
  for (size_t i = 0; i < n && !stale; ++i) stale = g->gen[i] != g->ctx[i]->generation;
  if (stale) {
    group_drop(g);
    g->gen.clear();
    for (sem_ctx* c : g->ctx) g->gen.push_back(c->generation);
    g->persistent = persistent;
    if (persistent) {
      int r = group_tables(g);
      if (r) return r;
    }
  }
  if (persistent && g->stall && left > 0) {  // failure-detection test: one eager step whose waits give up
    int r = group_enqueue_persistent_step(g, g->stall);
    g->stall = 0;
    if (r) return r;
    --left;
  }
  if (left >= kStepsPerGraph && !g->graph[0]) {
    int r = persistent ? group_build_persistent(g, 0, kStepsPerGraph) : group_build(g, 0, kStepsPerGraph);
    if (r) return r;
  }
  if (left % kStepsPerGraph && !g->graph[1]) {
    int r = persistent ? group_build_persistent(g, 1, 1) : group_build(g, 1, 1);
    if (r) return r;
  }
  for (; left >= kStepsPerGraph; left -= kStepsPerGraph)
    if ((e = cudaGraphLaunch(g->graph[0], g->stream)) != cudaSuccess) return group_fail(g, SEM_ECUDA, cudaGetErrorString(e));
  for (; left > 0; --left)
    if ((e = cudaGraphLaunch(g->graph[1], g->stream)) != cudaSuccess) return group_fail(g, SEM_ECUDA, cudaGetErrorString(e));
  // later work of every context waits for the group
  if (cudaEventRecord(g->ev[0], g->stream) != cudaSuccess) return group_fail(g, SEM_ECUDA, "group completion event");
  for (size_t i = 0; i < n; ++i) {
    if (cudaStreamWaitEvent(g->ctx[i]->stream, g->ev[0], 0) != cudaSuccess)
      return group_fail(g, SEM_ECUDA, "ordering a context after the group");
    g->ctx[i]->steps += nsteps - 1;  // advance() counted the eager step
  }
  return SEM_OK;
}

int sem_group_sync(sem_group* g) {
  if (!g) return group_fail(nullptr, SEM_EINVAL, "null group");
  cudaSetDevice(g->device);
  cudaError_t e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return group_fail(g, SEM_ECUDA, cudaGetErrorString(e));
  if (g->d_sync) {
    int err = 0;
    e = cudaMemcpy(&err, &g->d_sync->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return group_fail(g, SEM_ECUDA, cudaGetErrorString(e));
    if (err) {
      cudaMemset(&g->d_sync->err, 0, sizeof(int));
      return group_fail(g, SEM_ETIMEOUT,
                        "a bounded wait of the group sweep gave up (the forces of that step are incomplete)");
    }
  }
  return SEM_OK;
}

int sem_group_set_option(sem_group* g, int option, long long value) {
  if (!g) return group_fail(nullptr, SEM_EINVAL, "null group");
  switch (option) {
    case SEM_GROUP_MODE:
      if (value < 0 || value > 1) return group_fail(g, SEM_EINVAL, "group mode must be 0 (graph branches) or 1 (persistent)");
      g->mode = static_cast<int>(value);
      return SEM_OK;
    case SEM_GROUP_STALL_TEST:
      if (value < 0 || value > 1) return group_fail(g, SEM_EINVAL, "stall test must be 0 or 1");
      g->stall = static_cast<unsigned int>(value);
      return SEM_OK;
    default:
      return group_fail(g, SEM_EINVAL, "unknown group option " + std::to_string(option));
  }
}

int sem_group_info(sem_group* g, int* out) {
  if (!g || !out) return group_fail(g, SEM_EINVAL, "sem_group_info: bad arguments");
  out[0] = group_persistent_ok(g) ? 1 : 0;
  std::set<std::pair<int, int>> keys;
  for (const sem_ctx* c : g->ctx) keys.insert({c->ngll, c->variant});
  out[1] = out[0] ? static_cast<int>(keys.size()) : 0;
  return SEM_OK;
}

const char* sem_group_last_error(const sem_group* g) { return g ? g->err.c_str() : g_err.c_str(); }

const char* sem_last_error(const sem_ctx* c) { return c ? c->err.c_str() : g_err.c_str(); }

}  // extern "C"
