// Internal declarations shared by the host set-up (sem_setup.cpp), the C ABI
// (sem_capi.cpp) and the CUDA kernels (sem_kernels.cu) of libsemgb.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

struct sem_ctx;

namespace semgb {

using sem_ctx_fwd = ::sem_ctx;

constexpr int kMaxNgll = 10;
constexpr int kMinNgll = 2;

// Words per local point in the element record: ibool, nine inverse-Jacobian terms
// dxi_r/dx_d (r-major: xix xiy xiz etax etay etaz gammax gammay gammaz), J kappa, J mu, J.
// The force kernels read the first kForceFields fields only (J sigma from J kappa and J mu
// needs no separate J); J serves the mass and the material sensitivities.
constexpr int kRecFields = 13;
constexpr int kForceFields = 12;
enum RecField { kIbool = 0, kG = 1, kJKappa = 10, kJMu = 11, kJac = 12 };

// The context's own wavefields u, v, a are float32 [nglob][kNodeStride]: x, y, z and a zero
// pad, so that every node is one aligned 16-byte access in the gather, the scatter and the
// Newmark passes. Caller-facing arrays stay [nglob][3]; copies at the boundary are strided.
constexpr int kNodeStride = 4;

// Bit 31 of a record's ibool word marks the first contribution to that node in the
// colour-by-colour processing order: the force kernel stores instead of adding there,
// so the assembled array needs no zeroing pass.
constexpr uint32_t kFirstTouchBit = 0x80000000u;
// Bit 30 marks the same for the patch kernel's order (patch colour by patch colour), on the
// word of the first local point (in patch-table order) of each patch node. Bit 29 marks a
// local point that is the only one of its patch at its node (its element's team writes it
// alone). Bit 28 marks, on every local point of a patch node, that this patch is the node's
// last toucher in the sweep (its force is complete there: the Newmark update of the node can
// run in the same pass). Node ids are below 2^28.
constexpr uint32_t kPatchFirstBit = 0x40000000u;
constexpr uint32_t kAloneBit = 0x20000000u;
constexpr uint32_t kPatchLastBit = 0x10000000u;
constexpr uint32_t kNodeMask = 0x0FFFFFFFu;
constexpr int kMaxNodes = 1 << 28;

inline int rec_words(int ngll) {
  const int np = ngll * ngll * ngll;
  return (kRecFields * np + 3) / 4 * 4;  // 16-byte aligned element records
}

// Position of local point (i, j, k) inside a geometry or material field of an element
// record: points are stored i-major so that the NGLL^2 threads owning the xi-lines (j, k)
// of an element read consecutive words for a fixed i. The ibool field keeps the natural
// order p = i + NGLL*j + NGLL^2*k, which the gather and scatter threads walk.
inline int rec_pos(int ngll, int i, int j, int k) { return i * ngll * ngll + j + ngll * k; }

// ---- host set-up (sem_setup.cpp) -------------------------------------------------------
int gll_basis(int ngll, double* xi, double* w, double* hprime, std::string* err);

// Positions, inverse Jacobian and determinant at every GLL point of one trilinear element;
// xyz[np][3], G[np][9] (dxi_r/dx_d at 3r+d), J[np]; returns false if some J <= 0.
bool element_geometry(int ngll, const double* xi, const double* hprime, const double* ctrl,
                      double* xyz, double* G, double* J);
// The same from the positions xyz[np][3] of the element's GLL points (any geometry).
bool geometry_from_positions(int ngll, const double* hprime, const double* xyz, double* G, double* J);

int color_elements(int nspec, int ngll, int nglob, const int32_t* ibool,
                   std::vector<int32_t>* color, int* ncolors, std::string* err);

int locate_nodes(int nglob, const double* node_xyz, int npts, const double* xyz,
                 const double* surface_z, int32_t* out);

// Patches for the force sweep (sem_patches.cpp): bricks of bx x by x bz elements of the
// mesh's lattice coordinates, coloured so that no two patches of a colour share a node.
struct PatchShape {
  int bx = 1, by = 1, bz = 1;
};
struct PatchPlan {
  int ngll = 0;
  int npatch = 0;
  int ncolors = 0;
  int max_nodes = 0;              // largest patch node count
  int max_elems = 0;              // largest patch element count
  std::vector<int> elem;          // caller elements in sweep order, patch after patch
  std::vector<int> patch_off;     // [npatch + 1] into elem (sweep order)
  std::vector<int> color_off;     // [ncolors + 1] patch ranges of the sweep order
  std::vector<int> node_off;      // [npatch + 1] into nodes
  std::vector<uint32_t> nodes;    // patch node lists: caller node | kFirstTouchBit
  std::vector<int> table_of;      // per patch: its table
  std::vector<int> tab_nelem, tab_nnode, tab_nshared, tab_lid_off, tab_csr_off, tab_excl_off, tab_first_off;
  std::vector<uint16_t> lid;      // per table: [nelem][np] patch-local node of each local point
  std::vector<int> node_new;      // [nglob] internal id of every caller node
  std::vector<uint16_t> csr;      // per table: per shared patch node (one met by several local
                                  // points) kPatchSlots slots holding those local points
                                  // (le*np + p, ascending)
  std::vector<uint32_t> excl;     // per table: bit le*np + p set when that local point is the
                                  // only one at its patch node
  std::vector<uint16_t> first_q;  // per table: per patch node, its first local point
};
// Contribution slots per patch node: 8 (the elements meeting at a vertex of a structured
// hexahedral mesh), read as one 16-byte word. An unused slot holds kPatchNoSlot; a node met
// by more local points continues in another group of slots, named by its last slot as
// kPatchChain | group.
constexpr int kPatchSlots = 8;
constexpr uint16_t kPatchNoSlot = 0xFFFFu;
constexpr uint16_t kPatchChain = 0x8000u;
int build_patches(int nspec, int ngll, int nglob, const int32_t* ibool, const PatchShape& shape, PatchPlan* plan,
                  std::string* err);

// ---- device side (sem_kernels.cu) ------------------------------------------------------
struct DevCtl {
  long long step;  // steps taken since the state was set
  int col;         // next seismogram column
  int ncols;       // columns in the seismogram buffer (0: no recording)
  float* seis;     // [nrec][3][ncols] or null
  int err;
  int pad;
  float* snap;          // displacement snapshots [col][shots][nglob][3], or null
  long long snap_per;   // floats per snapshot
  // adjoint steps replayed from a graph: step j reads residual adj_G + (j - 1) adj_gstep and
  // snapshots adj_u + (j - 1 .. j + 1) adj_n3; j counts down
  const float* adj_G;
  const float* adj_u;
  long long adj_n3;
  int adj_gstep;
  int adj_j;   // the step the sweep of lam is at (residual injection)
  int adj_js;  // the step the sensitivity terms are at (they may run one step behind)
  int pad3;
};

struct DevProblem {
  int ngll;
  int nspec;
  int nglob;
  int shots;  // wavefields are [nglob][shots][kNodeStride]
  const float* rec;
  float* u;
  float* v;
  float* a;
  const float* minv;
  DevCtl* ctl;
  int nsrc;
  const int* src_node;   // per source: global node
  const int* src_shot;   // per source: shot it acts in
  const double* src_force;
  double f0, t0;
  int nrec;
  const int* rec_node;
  double dt;
};

// Copies hprime, hprime*w and w for this ngll into the kernels' constant banks.
int upload_basis(int ngll, const double* w, const double* hprime, void* stream);

// One colour's worth of elements [e0, e1) of the colour-sorted order: f (=|+=) -K u; a node
// is stored at its first touch in colour order and accumulated afterwards.
struct ForceLaunch {
  const float* rec;
  const int* elist;  // record slots in colour order; e0, e1 index this list
  const int* perm;   // internal -> caller node (caller arrays, node_stride 3)
  const float* u;
  float* f;
  int e0, e1;
  int node_stride;  // floats per node in u and f: kNodeStride (internal order), or 3 for caller
                    // arrays in caller order
  int shots;        // > 1: u and f are [nglob][shots][kNodeStride], items (element, shot)
  int variant;      // contraction form: 0 the order's default, 1 line owners, 2 per point
  int atomic;       // colouring ablation: float atomic adds into a zeroed f, any element order
};
int launch_forces(int ngll, const ForceLaunch& launch, void* stream);

// One patch colour [p0, p1) of the patch sweep order on the context's own [nglob][shots][4]
// fields: f (=|+=) -K u.
struct alignas(16) PatchDesc {
  int slot0;     // record slot of the patch's first element (its elements are consecutive)
  int nelem;
  int nshared;   // patch nodes met by several of its local points
  int slot_off;  // its table: per shared node, kPatchSlots slots (shared-memory offsets of the
                 // forces of the local points meeting there)
  int word_off;  // its table: per shared node, the shared-memory offset of its first local
                 // point's ibool word
  int src_off;   // its point sources (PatchSrc entries [src_off, src_off + nsrc)): the ones at
  int nsrc;      // nodes it touches last, added there to the complete force
  int pad;
};
// A receiver in the adjoint sweep: internal node, receiver index (its residual G[3 r + c]).
struct PatchRecv {
  int node;
  int r;
};
struct DevCtl;
// A point source in the patch sweep: internal node, shot, force vector (Sec. V-C).
struct PatchSrc {
  int node;
  int shot;
  double f[3];
};
// The explicit Newmark update (Sec. I) run by the patch sweep at each node's last toucher:
// mode 1 corrector of step n fused with the predictor of step n+1
//   a = M^-1 f ; v = v_half + dt/2 a ; u <- u + dt v + dt^2/2 a ; v_half <- v + dt/2 a
// (f is then not stored), mode 2 the corrector alone (v <- v_half + dt/2 a, a stored), mode 0
// none (f stored). The point sources of the step, at t = ctl->step dt, are added to f first.
struct SweepNewmark {
  int mode;           // 3: the adjoint leapfrog (u = lam^m; lam_old: lam^{m+1} in, lam^{m-1} out)
  float* u;           // [nglob][shots][4], written at last touch (mode 1)
  float* v;           // [nglob][shots][4], half-step velocity in, out as above
  float* a;           // [nglob][shots][4], acceleration out (mode 2)
  const float* minv;  // [nglob]
  const PatchSrc* src;
  const long long* step;  // the step counter (t_{n+1} = step dt)
  double f0, t0, dtd;     // Ricker centre frequency and delay, step (double)
  float dt, hdt, hdt2;
  // adjoint (mode 3): the receivers at the nodes each patch touches last (recv_range[2 P],
  // recv_range[2 P + 1] = first, count into recv, ascending receiver within a patch), the
  // residual G [nrec][3]
  // (or, with idx, the one the device's adjoint counter names), 1/dt^2 and dt^2
  // snapshot run (modes 1, 2): u^{n+1} also stored at each node's last touch into
  // ctl->snap + (ctl->col - 1) ctl->snap_per, [nglob][3] in the order snap_perm maps to
  const DevCtl* snap_ctl;
  const int* snap_perm;
  float* lam_old;
  const int* recv_range;
  const PatchRecv* recv;
  const float* G;
  const DevCtl* idx;
  float inv_dt2, dt2;
};
// Counters of a persistent sweep (all patch colours in one launch): patches taken, CTAs
// that have left, a wait that gave up, patches finished per colour. Zero between sweeps.
constexpr int kMaxSweepColors = 64;
struct SweepSync {
  unsigned int next;
  unsigned int exited;
  int err;
  int pad;
  unsigned int done[kMaxSweepColors];
};
// One persistent sweep over the patches of several models of one order (a group step):
// items are the patches of every model, colour-major (colour 0 of every model, then colour
// 1, ...); a patch of colour c writes once every patch of colour c - 1 of its own model has
// finished. Models and runs of items live in device memory.
constexpr int kMaxGroupModels = 64;
struct GroupModel {
  const float* rec;
  const PatchDesc* desc;
  const uint16_t* slots;
  const uint16_t* words;
  const float* u;        // [nglob][4]
  float* f;              // [nglob][4]
  const int* color_end;  // per colour, the end of its patch range (model-local patches)
  int ncolors;
  int pad;
};
struct GroupSeg {  // a run of consecutive items: patches [p0, p0 + count) of one (model, colour)
  int item0;
  int model;
  int color;
  int p0;
};
struct GroupSync {
  unsigned int next;
  unsigned int exited;
  int err;
  int pad;
  unsigned int done[kMaxGroupModels * kMaxSweepColors];  // [model][colour] finished patches
};
struct GroupLaunch {
  const GroupModel* models;
  const GroupSeg* segs;
  int nseg;
  int nitems;
  int nmodels;
  int variant;       // contraction form as in ForceLaunch
  unsigned int stall;  // a count that never arrives (tests)
  GroupSync* sync;
};
int launch_group_sweep(int ngll, const GroupLaunch& launch, void* stream);

struct PatchLaunch {
  const float* rec;
  const PatchDesc* desc;
  const uint16_t* slots;
  const uint16_t* words;
  SweepSync* sync;        // non-null: one persistent launch over all colours
  const int* color_end;   // per colour, the end of its patch range (persistent launch)
  int npatch, ncolors;    // (persistent launch)
  int stall;              // (persistent launch) wait for a count that never arrives (tests)
  const float* u;
  float* f;
  int p0, p1;
  int variant;  // contraction form as in ForceLaunch
  int shots;    // > 1: fields [nglob][shots][kNodeStride]
  int pairs;    // with shots > 1: one CTA per (patch, shot pair) (else one per (patch, shot))
  SweepNewmark nm;  // mode 0: forces only
};
int launch_patch_forces(int ngll, const PatchLaunch& launch, void* stream);
// Shared-memory layout of the patch kernel for this order: workspace floats per element,
// per team, and elements per team (the slot tables hold offsets into it).
int patch_layout(int ngll, int* es, int* ts, int* e);
// the brick each order's patch kernel is compiled for
int patch_shape(int ngll, PatchShape* out);
int forces_kernel_smem_bytes(int ngll);
int forces_elements_per_cta(int ngll);

int launch_set_ctl(DevCtl* ctl, long long step, int ncols, float* seis, void* stream, float* snap = nullptr,
                   long long snap_per = 0);
// the displacement into snapshot ctl->col - 1 (the column the receivers just sampled)
int launch_snapshot(const float* u, DevCtl* ctl, const int* perm, int nglob, int shots, void* stream);
int launch_predictor(const DevProblem& p, void* stream);
int launch_fused_newmark(const DevProblem& p, void* stream);
int launch_corrector(const DevProblem& p, void* stream);
int launch_sources_record(const DevProblem& p, void* stream);
// u_lo, u_mid, u_hi: [nglob][3] in caller order (perm: internal -> caller node) or in
// internal order (perm null); the terms are added to float32 partials g_* [nlocal]
// (idx non-null: the snapshots are idx->adj_u + (j - 1 .. j + 1) idx->adj_n3, j = idx->adj_j)
int launch_sensitivity(int ngll, const float* rec, const int* perm, const float* lam, const float* u_lo,
                       const float* u_mid, const float* u_hi, float* g_rho, float* g_kappa, float* g_mu, int nspec,
                       double c_m, double c_k, void* stream, const DevCtl* idx = nullptr);
// solver layout [nglob][shots][kNodeStride] in internal node order <-> caller layout
// [shots][nglob][3] in caller node order (perm: internal -> caller node)
int launch_pack(const float* u, float* out, const int* perm, int nglob, int shots, void* stream);
int launch_unpack(const float* in, float* u, const int* perm, int nglob, int shots, void* stream);
// rnode[nnodes]: distinct receiver nodes; rlist[roff[t] .. roff[t+1]): their receivers
// (idx non-null: G_dev is taken from idx->adj_G at step idx->adj_j; G_dev then only says
// whether there is one)
int launch_adjoint_update(float* F, const float* G_dev, const int* rnode, const int* roff, const int* rlist,
                          int nnodes, const float* lam, float* lam_old, const float* minv, int nglob, double dt,
                          void* stream, const DevCtl* idx = nullptr);
int launch_adjoint_index(DevCtl* ctl, const float* G, const float* u, long long n3, int gstep, int j, void* stream);
int launch_adjoint_next(DevCtl* ctl, void* stream, bool sensitivity = false);  // adj_j (or adj_js) -= 1
// acc[t] += part[t] (float64), part[t] = 0, for t < n
int launch_flush_partials(float* part, double* acc, long long n, void* stream);
// Material on the device (Sec. II-B moduli, Sec. I diagonal mass). rho, p1, p2: per local
// point in caller order [nspec][ngll^3]; moduli: (p1, p2) = (kappa, mu), else (vp, vs).
struct MaterialLaunch {
  float* rec;          // colour-sorted element records
  const int* order;    // record slot -> caller element
  const int* elist;    // record slots in element colour order (the ranges below index it)
  const float* rho;
  const float* p1;
  const float* p2;
  int moduli;
  int ngll;
  int nspec;
  int nglob;
  double w[kMaxNgll];  // GLL weights
};
// index of the first local point that breaks rho > 0, mu (vs) >= 0, kappa > 0 (vp > vs) or
// is not finite, as an atomic minimum into *first_bad (caller presets it to ~0ull)
int launch_material_check(const MaterialLaunch& m, unsigned long long* first_bad, void* stream);
// kappa and mu into the records, the mass range by range of the sweep order (one colour per
// range, so no races), 1/mass,
// and the largest vp of every caller element (for the CFL suggestion)
int launch_material_apply(const MaterialLaunch& m, const int* sweep_off, int nranges, double* mass, float* minv,
                          double* vpmax, void* stream);
int launch_nonfinite_check(const DevProblem& p, int* flag, void* stream);
int launch_energy_partials(const float* u, const float* v, const float* f, const float* minv,
                           int nglob, int shots, double* partials, int nblocks, void* stream);
constexpr int kEnergyBlocks = 608;  // 4 CTAs per SM on 152 SMs

// ---- context access for entry points defined outside sem_capi.cpp ----------------------
struct CtxView {
  int device;
  void* stream;
  int nglob;
  const float* minv;     // internal node order
  const int* node_new;   // caller node -> internal node
};
// SEM_OK and the view when the material is set; otherwise an error code (message set).
int ctx_view(sem_ctx_fwd* c, CtxView* out);
int ctx_fail(sem_ctx_fwd* c, int code, const char* message);

}  // namespace semgb
