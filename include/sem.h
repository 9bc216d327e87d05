/*
 * sem.h -- C ABI of libsemgb, a GB300 (sm_103a) spectral-element solver for the 3D
 * isotropic elastic wave equation (arXiv 2606.12850, "High-Order Spectral Element Methods
 * for Wave Propagation on ARM Multicore CPU with SME").
 *
 * The library evaluates the hot path of Sec. II-B and IV-C on one GPU:
 *   - matrix-free internal forces  f = -K u  (Sec. II-B: reference derivatives along
 *     xi/eta/zeta as small products with the 1D GLL derivative matrix, Jacobian map,
 *     isotropic Hooke stress, weighted transposed products);
 *   - deterministic assembly through ibool, colour by colour with no atomics (Sec. IV-C:
 *     elements sharing a node never share a colour);
 *   - explicit second-order Newmark stepping with the diagonal GLL mass (Sec. I, II-B,
 *     V-C), a Ricker point force and receiver recording (Sec. V-C).
 *
 * Conventions used by every call:
 *   ngll     points per direction, NGLL = N + 1, 2 <= ngll <= 10.
 *   local point index p = i + ngll*j + ngll*ngll*k (i along xi, j along eta, k along zeta).
 *   ibool    int32 [nspec][ngll^3], 0-based global node of every local point.
 *   ctrl     float64 [nspec][8][3] corner vertices of each (trilinear) hexahedron; corner
 *            c = a + 2b + 4d sits at reference (xi, eta, zeta) = (2a-1, 2b-1, 2d-1).
 *   fields   float32 [shots][nglob][3] (x, y, z per node), metres, m/s, m/s^2; shots = 1
 *            unless sem_set_shots chose more.
 *   seis     float32 [shots][nrec][3][nsteps].
 *   Step n (0-based since the last sem_set_state) advances u^n -> u^{n+1}; the source acts
 *   at t_{n+1} = (n+1) dt and the record of step n is u^{n+1}.
 *
 * Ownership: host pointers are read (or written) during the call only. Pointers named
 * *_dev are device pointers on the context's GPU, borrowed for the call (asynchronous
 * calls: until the context's stream reaches that point). The library owns all the other
 * device memory it allocates and frees it in sem_destroy.
 *
 * Errors: every int-returning call returns SEM_OK (0) or a negative code below and leaves a
 * message for sem_last_error. No call aborts the process. A sem_ctx is not thread-safe.
 */
#ifndef SEM_H
#define SEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SEM_OK 0
#define SEM_EINVAL (-1)    /* bad argument: size, index out of range, J <= 0, NaN ...     */
#define SEM_ENOMEM (-2)    /* device or host allocation failed                             */
#define SEM_ECUDA (-3)     /* a CUDA runtime call failed (message holds cudaGetErrorString) */
#define SEM_ESTATE (-4)    /* call order: mesh, then material, then dt, before stepping     */
#define SEM_ETIMEOUT (-5)  /* a bounded device wait gave up                                 */
#define SEM_EDIVERGED (-6) /* NaN or Inf found in the wavefield                             */

typedef struct sem_ctx sem_ctx;

/* Library version as 10000*major + 100*minor + patch. */
int sem_version(void);

/* GLL nodes, weights and derivative matrix for ngll points (Sec. II-B: tensor-product GLL
 * interpolation; the 1D differentiation matrix of the small products).
 * xi[ngll] ascending on [-1, 1]; w[ngll]; hprime[ngll*ngll] row-major with
 * hprime[i*ngll + l] = l_l'(xi_i). Host only, no GPU needed. Any output may be NULL. */
int sem_gll(int ngll, double* xi, double* w, double* hprime);

/* Greedy colouring of elements (Sec. IV-C): corner vertices taken from ibool give an
 * element-to-vertex incidence; elements sharing a vertex are adjacent (the sparsity of the
 * incidence times its transpose); colours are assigned greedily in element order. On
 * return color[e] in [0, *ncolors) and no two elements of one colour share any ibool
 * entry (checked; SEM_EINVAL otherwise, e.g. for a non-conforming mesh or an element that
 * repeats a node). Host only, no GPU needed. */
int sem_color_elements(int nspec, int ngll, int nglob, const int32_t* ibool,
                       int32_t* color, int* ncolors);

/* The patches sem_set_mesh builds for the force sweep (see SEM_OPT_ASSEMBLY), for a mesh
 * given by ibool alone. Lattice coordinates come from a walk across shared element faces
 * (the neighbour across an element's own +xi face sits one step along x, and so on), the
 * patches are bricks of those coordinates (shape from info[4..6]), coloured greedily so
 * that no two patches of a colour share a node (Sec. IV-C's colouring applied to groups of
 * elements). Outputs, each caller-owned and may be NULL: patch_of[nspec] the patch of every
 * element (patches numbered in sweep order, colour after colour), color_of[nspec] the colour
 * of patch P at index P (entries past the patch count are untouched), info[7] = patches,
 * colours, largest patch node count, distinct patch tables, brick x, y, z. Host only, no GPU
 * needed. SEM_EINVAL for bad sizes or an ibool entry out of range. */
int sem_patch_plan(int ngll, int nspec, int nglob, const int32_t* ibool, int32_t* patch_of, int32_t* color_of,
                   int64_t* info);

/* Geometry of trilinear hexahedra at their GLL points (Sec. II-B: the mapping of each
 * element to the reference cube and its Jacobian), exactly as sem_set_mesh computes it:
 * the GLL positions from the eight corners, dx/dxi by differentiating those positions with
 * hprime, its inverse by cofactors, all in double precision. ctrl[nspec][8][3] as in
 * sem_set_mesh (corner c at reference (2a-1, 2b-1, 2d-1), c = a + 2b + 4d). Outputs, each
 * caller-owned and may be NULL: xyz[nspec][ngll^3][3], dxi_dx[nspec][ngll^3][3][3] with
 * [r][d] = d xi_r / d x_d, jac[nspec][ngll^3] = det(dx/dxi); the point index is
 * i + ngll*(j + ngll*k). SEM_EINVAL for bad sizes or non-finite corners, and, after all
 * outputs are written, if any determinant is <= 0 (the message names the first such
 * element). Host only, no GPU needed. */
int sem_geometry(int ngll, int nspec, const double* ctrl, double* xyz, double* dxi_dx, double* jac);

/* The geometry sem_set_mesh computes from per-point positions xyz[nspec][ngll^3][3] (the
 * isoparametric map: dx/dxi by differentiating the positions with hprime along each
 * reference direction, its inverse by cofactors and its determinant, float64). Outputs as
 * in sem_geometry, each caller-owned and may be NULL. SEM_EINVAL for bad sizes, non-finite
 * positions, or (after all outputs are written) a determinant <= 0. Host only. */
int sem_geometry_points(int ngll, int nspec, const double* xyz, double* dxi_dx, double* jac);

/* Point location in trilinear hexahedra: for each of npts points xyz[npts][3], the
 * lowest-numbered element of ctrl[nspec][8][3] that holds it, elem_out[npts] (-1 for a point
 * outside every element), and its reference coordinates ref_out[npts][3] in [-1, 1] (may be
 * NULL; 0 for points outside). Elements are tried in index order when their corner bounding
 * box (widened by 1e-9 of its largest side) holds the point; the trilinear map is inverted by
 * Newton's method from the element centre; a solution within 1e-9 of the reference cube
 * counts as inside. For many points a uniform grid of buckets over the elements' boxes
 * supplies the candidates instead of a scan of every element, with the same result (4096
 * points on a 64^3-element mesh: 0.15 s). Host only, no GPU needed. SEM_EINVAL for bad
 * sizes or non-finite input. */
int sem_locate_points(int nspec, const double* ctrl, int npts, const double* xyz, int32_t* elem_out,
                      double* ref_out);

/* Nodal forces of a point source between nodes (Sec. II-B Lagrange basis psi_(i,j,k) =
 * l_i(xi) l_j(eta) l_k(zeta) of the element with corners ctrl_e[8][3]), at reference
 * coordinates ref[3] in [-1, 1]: with force[3] (N), f_out[p] = F psi_p(ref); with
 * moment[6] = (Mxx, Myy, Mzz, Mxy, Mxz, Myz) (N m), f_out[p] = M grad psi_p(ref) (the body
 * force -M . grad delta tested against psi_p), grad through the inverse of the trilinear
 * Jacobian at ref. Exactly one of force and moment is non-NULL. f_out: [ngll^3][3] in local
 * point order. Host only, no GPU needed. SEM_EINVAL for bad arguments. */
int sem_point_source_forces(int ngll, const double* ctrl_e, const double* ref, const double* force,
                            const double* moment, double* f_out);

/* Create a solver context on CUDA device `device` for polynomial degree ngll-1.
 * `cuda_stream` is a cudaStream_t to issue all work on, or NULL for a stream the context
 * creates and owns. */
int sem_create(sem_ctx** out, int ngll, int device, void* cuda_stream);

/* Free every device and host resource of the context. NULL is allowed. */
int sem_destroy(sem_ctx* ctx);

/* Tunables.
 *   SEM_OPT_SWEEP_SLABS (applied by the next sem_set_mesh): the force sweep visits the
 *   elements slab by slab (equal-count slabs along the longest axis of the element
 *   centroids) and colour by colour inside a slab, so that a slab's nodes can stay in L2
 *   across its colour launches; value = slab count, 0 or 1 = colour by colour over the
 *   whole mesh (the default). Results change only by the summation order at nodes.
 * SEM_EINVAL for an unknown option or a value out of range. */
#define SEM_OPT_SWEEP_SLABS 1
/*   SEM_OPT_CONTRACTION (takes effect at once): the force kernel's eta/zeta contraction
 *   form, 0 = the order's default (line owners from NGLL 4 up, per point below), 1 = line
 *   owners, 2 = per point; sem_autotune sets it from measurement. */
#define SEM_OPT_CONTRACTION 2
/*   SEM_OPT_ASSEMBLY (takes effect at once): how the force sweep assembles element forces
 *   on the context's own fields. Patches are bricks of neighbouring elements
 *   (1 x 4 x 2 at NGLL 5; SEM_OPT_PATCH_SHAPE sets another, sem_patch_info gives the shape in
 *   use) evaluated by one CTA each, which
 *   sums the forces meeting at each of the brick's nodes in a fixed order and writes each
 *   node once; the bricks are coloured so that no two of a colour share a node (Sec. IV-C's
 *   colouring applied to groups of elements).
 *     0 (default) = patches, one launch per patch colour (with several shots one CTA per
 *       patch and shot);
 *     1 = element by element, one launch per element colour (the form always used for
 *       caller-layout arrays);
 *     2 = patches, all colours in one persistent launch (single shot; several shots use 0):
 *       CTAs take patches in sweep order
 *       and a patch writes only after every patch of the previous colour has finished (a
 *       bounded wait; if one gives up, the next sem_sync, sem_run or sem_check_finite
 *       returns SEM_ETIMEOUT).
 *     3 = the colouring ablation (Sec. V-D-1 compares the colouring with atomics): the
 *       element kernel of 1 over every element in one launch, each point's forces added to
 *       its node with a float atomic add into f zeroed first. Not deterministic (the order
 *       of the additions varies from run to run); for timing comparisons only.
 *   0 and 2 give bitwise equal results; 1 differs from them only in the order of the
 *   float32 sums at shared nodes. 0, 1 and 2 are deterministic. */
#define SEM_OPT_ASSEMBLY 3
/*   SEM_OPT_NODE_ORDER (takes effect at once): the node order of the device arrays of
 *   sem_set_state_dev, sem_get_state_dev, sem_run_snapshots and of the snapshots
 *   sem_adjoint_accumulate / sem_adjoint_segment read: 0 (default) the caller's order, 1 the
 *   solver's internal order (sem_node_order), which saves a permutation per node and copy
 *   for arrays that only travel between these calls (checkpoints and snapshots of the
 *   adjoint). Host arrays always use the caller's order. */
#define SEM_OPT_NODE_ORDER 5
/*   SEM_OPT_SWEEP_STALL_TEST (failure-detection test, one-shot): 1 makes the next direct
 *   persistent sweep (SEM_OPT_ASSEMBLY 2, sem_apply_stiffness_strided with stride 4) wait
 *   for a count that never arrives, so that its bounded waits give up and the next sem_sync
 *   returns SEM_ETIMEOUT; the sweep after that runs normally. Sweeps replayed from a
 *   captured time step are not affected. */
#define SEM_OPT_SWEEP_STALL_TEST 4
/*   SEM_OPT_FUSED_NEWMARK (takes effect at once; used with SEM_OPT_ASSEMBLY 0): 2 (default)
 *   = 1 for a single shot, 0 for several (where the separate pass over the shot-innermost
 *   fields measures faster); 1 = time steps run the Newmark update (Sec. I) inside the force
 *   sweep: the patch that touches a node last in the sweep adds the step's point sources to
 *   the node's complete force and runs the corrector of step n fused with the predictor of
 *   step n+1 there, so a
 *   step is one receiver-sampling launch plus the sweep, with no separate pass over the
 *   nodes; sem_step / sem_run start with a predictor pass and end with a sweep that runs the
 *   corrector alone, so the state is complete between calls. 0 = separate Newmark passes
 *   (one fused corrector/predictor pass per step; the state between calls is completed on
 *   demand). Both give bitwise equal wavefields and seismograms. */
#define SEM_OPT_FUSED_NEWMARK 6
/*   SEM_OPT_SHOT_PAIRS (takes effect at once; several shots, SEM_OPT_ASSEMBLY 0): 1 (default)
 *   = each CTA of the patch sweep takes one patch for two shots, every thread carrying both
 *   shots as float32 pairs (one packed fma for both; each geometry and modulus value read
 *   once for both); 0 = one CTA per patch and shot. The same arithmetic per shot; results
 *   differ only by the rounding order of a few sums. */
#define SEM_OPT_SHOT_PAIRS 7
/*   SEM_OPT_PATCH_SHAPE (applied by the next sem_set_mesh): the brick of elements one CTA of
 *   the patch sweep takes, value = bx | by << 8 | bz << 16 in elements along the mesh's
 *   lattice x, y, z; 0 = the order's default (sem_patch_info reports the shape in use).
 *   bx*by*bz may not exceed the elements a patch CTA holds at this order (8 at NGLL 5; the
 *   default brick's count); every brick shape with that count runs the same kernel.
 *   sem_tune_patch_shape measures them and sets the fastest. */
#define SEM_OPT_PATCH_SHAPE 8
int sem_set_option(sem_ctx* ctx, int option, long long value);

/* Set the mesh (Sec. II-B: hexahedral elements mapped to the reference cube, the
 * solution interpolated at the tensor-product GLL points; Sec. IV-C: the global-to-local
 * map ibool). xyz[nspec][ngll^3][3] (float64, metres) is the position of every LOCAL point
 * in local point order, so any element geometry the GLL points can describe (curved faces,
 * topography) is allowed, and a periodic ibool stays well defined (a node may appear with
 * different coordinates in different elements). The library computes dx/dxi at every GLL
 * point by differentiating the positions with hprime along each reference direction (the
 * isoparametric map), its inverse and determinant in float64, the element colouring, the
 * force-sweep patches and the internal node order, and the device copies. Point location
 * and sources between nodes (sem_locate_points, sem_set_shot_sources_at) use the trilinear
 * map of each element's corner GLL points. Node coordinates (sem_node_xyz,
 * sem_locate_nodes, sem_set_sources, sem_set_receivers) are read from the local points
 * (the last element naming a node wins). SEM_EINVAL if nspec < 1, an ibool entry is
 * outside [0, nglob), an element repeats a node, some node in [0, nglob) is never
 * referenced, a coordinate is not finite, or J <= 0 somewhere (the message names the
 * element). Replaces the previous mesh, material, dt, sources, receivers and state. */
int sem_set_mesh(sem_ctx* ctx, int nspec, int nglob, const int32_t* ibool, const double* xyz);

/* sem_set_mesh for trilinear hexahedra given by their corners ctrl[nspec][8][3] (corner
 * c = a + 2b + 4d at reference (2a-1, 2b-1, 2d-1)): the GLL point positions come from the
 * trilinear map (sem_geometry), then everything as sem_set_mesh. */
int sem_set_mesh_corners(sem_ctx* ctx, int nspec, int nglob, const int32_t* ibool, const double* ctrl);

/* Set the isotropic material per local point, float32 [nspec][ngll^3] each
 * (Sec. II-B: density rho and stiffness C; here C from the wave speeds with
 * mu = rho vs^2, lambda = rho (vp^2 - 2 vs^2), kappa = lambda + 2/3 mu). Assembles the
 * diagonal mass M_I = sum rho J w_i w_j w_k. SEM_EINVAL for rho <= 0, vs < 0, vp <= vs,
 * or non-finite values. Requires sem_set_mesh. */
int sem_set_material(sem_ctx* ctx, const float* rho, const float* vp, const float* vs);

/* Same with the moduli given directly: kappa (bulk) and mu (shear) per local point, float32
 * [nspec][ngll^3] each; SEM_EINVAL unless rho > 0, kappa > 0, mu >= 0. */
int sem_set_moduli(sem_ctx* ctx, const float* rho, const float* kappa, const float* mu);
/* Same as sem_set_moduli from device arrays float32 [nspec][ngll^3] on the context's GPU
 * (caller-owned, read during the call); checked on the device (SEM_EINVAL names the first
 * offending local point). Synchronous. For model updates that stay in device memory. */
int sem_set_moduli_dev(sem_ctx* ctx, const float* rho_dev, const float* kappa_dev, const float* mu_dev);

/* dt = courant * min over elements of (smallest distance between neighbouring GLL points
 * along a grid line / largest vp of the element) (Sec. IV-B, V-C). Requires material. */
int sem_suggest_dt(sem_ctx* ctx, double courant, double* dt_out);

/* Time step in seconds (> 0, finite). Requires material. */
int sem_set_dt(sem_ctx* ctx, double dt);

/* Nearest global GLL node to each of npts points xyz[npts][3] (ties: lowest index).
 * With surface_z non-NULL only nodes whose z is within 1e-9 * max(1, |*surface_z|) of
 * *surface_z are candidates. Requires sem_set_mesh. Host computation. */
int sem_locate_nodes(sem_ctx* ctx, int npts, const double* xyz, const double* surface_z,
                     int32_t* node_out);

/* Physical position of global nodes: xyz_out[i][0..2] of node[i] (GLL points of the
 * trilinear elements, Sec. II-B), float64 host arrays. */
int sem_node_xyz(sem_ctx* ctx, int npts, const int32_t* node, double* xyz_out);

/* Point forces at positions xyz[nsrc][3] (metres), each snapped to the nearest global GLL
 * node (ties: lowest index), with force[nsrc][3] (N) and the Ricker time function of
 * sem_set_source_nodes. Replaces all sources; nsrc may be 0. Requires sem_set_mesh.
 * SEM_EINVAL for non-finite positions or forces. */
int sem_set_sources(sem_ctx* ctx, int nsrc, const double* xyz, const double* force, double f0, double t0);

/* Point forces (Sec. V-C): at step n, accel_raw[node[s]] += force[s][0..2] * R(t_{n+1} - t0)
 * with the Ricker wavelet R(tau) = (1 - 2 a) exp(-a), a = (pi f0 tau)^2, evaluated in
 * float64. nsrc may be 0. */
int sem_set_source_nodes(sem_ctx* ctx, int nsrc, const int32_t* node, const double* force,
                    double f0, double t0);

/* Several shots on one model (same mesh, material, dt and receivers; each shot its own
 * sources and wavefield): the shots advance together and every element's geometry and
 * moduli are read once per step for all of them. Reallocates the wavefields, zeroes the
 * state and the step counter and clears the sources (set them again). nshots >= 1; the
 * wavefields take 3 * 16 * nglob * nshots bytes. Requires sem_set_mesh. */
int sem_set_shots(sem_ctx* ctx, int nshots);

/* Point forces per shot: source s acts only in shot shot[s] (0 <= shot[s] < nshots), with
 * the Ricker time function of sem_set_sources (which instead applies each source in every
 * shot). */
int sem_set_shot_sources(sem_ctx* ctx, int nsrc, const int32_t* shot, const int32_t* node,
                         const double* force, double f0, double t0);

/* Moment-tensor point sources per shot (the equivalent body force -M . grad(delta) of a
 * source at node[s], with the Ricker time function of sem_set_sources): node I receives
 * f_I = M grad(psi_I)(x_s), the gradient taken in the lowest-numbered element that holds
 * node[s] (the Lagrange basis of Sec. II-B through its inverse Jacobian), so the forces sit
 * on the 3 NGLL - 2 nodes of the three GLL lines through the source. moment: float64
 * [nsrc][6] = (Mxx, Myy, Mzz, Mxy, Mxz, Myz) in N m. Replaces all sources. */
int sem_set_shot_moment_sources(sem_ctx* ctx, int nsrc, const int32_t* shot, const int32_t* node,
                                const double* moment, double f0, double t0);

/* Sources at arbitrary positions xyz[nsrc][3] (metres) inside the mesh, spread over the
 * nodes of the element that holds each one (sem_locate_points: lowest-numbered element) by
 * sem_point_source_forces: either point forces force[nsrc][3] or moment tensors
 * moment[nsrc][6] (exactly one non-NULL), with the Ricker time function of sem_set_sources.
 * shot[nsrc] assigns each source to a shot (0 <= shot[s] < nshots); NULL applies every source
 * in every shot. Forces that land on the same (shot, node) add. Replaces all sources.
 * SEM_EINVAL for a source outside the mesh (the message names it) or non-finite values.
 * Requires sem_set_mesh. */
int sem_set_shot_sources_at(sem_ctx* ctx, int nsrc, const int32_t* shot, const double* xyz,
                            const double* force, const double* moment, double f0, double t0);

/* Receivers at positions xyz[nrec][3] (metres), each snapped to the nearest global GLL node
 * (ties: lowest index); node_out[nrec] (may be NULL) receives those nodes. The displacement
 * there is recorded after every step of sem_run / sem_run_dev, for every shot. Replaces
 * all receivers; nrec may be 0. Requires sem_set_mesh. SEM_EINVAL for non-finite
 * positions. (Receivers confined to a surface: sem_locate_nodes with surface_z, then
 * sem_set_receiver_nodes.) */
int sem_set_receivers(sem_ctx* ctx, int nrec, const double* xyz, int32_t* node_out);

/* Receivers at global nodes node[nrec]. nrec may be 0. */
int sem_set_receiver_nodes(sem_ctx* ctx, int nrec, const int32_t* node);

/* Set (u, v, a) at t = 0 from host arrays [nglob][3] (NULL = zero) and reset the step
 * counter. SEM_EINVAL if a value is not finite (checked on the device; the state is then
 * zero). Requires sem_set_mesh. Synchronous. */
int sem_set_state(sem_ctx* ctx, const float* u, const float* v, const float* a);
/* Same from device arrays (NULL = zero). Asynchronous on the context's stream. */
int sem_set_state_dev(sem_ctx* ctx, const float* u_dev, const float* v_dev, const float* a_dev);

/* Declare the current state to be u^n, v^n, a^n of step n = step >= 0 (sem_set_state sets
 * n = 0): the next step applies the sources at t_{n+1}. Used to restart a run from a state
 * saved at step n. Host-only, no device work. */
int sem_set_step(sem_ctx* ctx, long long step);

/* Replace a by the acceleration of the current displacement, a = M^-1 (-K u) (no source
 * term), so that a state set from u and v alone (an initial condition) is consistent for
 * the first step. Asynchronous on the context's stream. Requires mesh, material and dt. */
int sem_init_acceleration(sem_ctx* ctx);

/* Copy the current state (u^n, v^n, a^n) to host arrays [nglob][3] (NULL = skip).
 * Reading v or a completes the pending half step (the trajectory is unchanged up to
 * rounding); reading u alone does not touch the state. Synchronous. */
int sem_get_state(sem_ctx* ctx, float* u, float* v, float* a);
/* Same into device arrays. Asynchronous on the context's stream. */
int sem_get_state_dev(sem_ctx* ctx, float* u_dev, float* v_dev, float* a_dev);

/* Advance nsteps >= 0 time steps without recording. Asynchronous on the stream. */
int sem_step(sem_ctx* ctx, int nsteps);

/* Advance nsteps time steps and record seismograms into host seis[nrec][3][nsteps]
 * (may be NULL). Synchronous. Ends with sem_check_finite: SEM_EDIVERGED (seismograms
 * still copied) when the run blew up. */
int sem_run(sem_ctx* ctx, int nsteps, float* seis);
/* Same, recording into a device buffer seis_dev[nrec][3][nsteps] (may be NULL).
 * Asynchronous on the context's stream. */
int sem_run_dev(sem_ctx* ctx, int nsteps, float* seis_dev);

/* Advance nsteps time steps and store the displacement after every step: u_dev receives
 * u^{n+1}, ..., u^{n+nsteps} as float32 [nsteps][shots][nglob][3] (device, caller-owned,
 * borrowed until the stream reaches the end of the call). Used to recompute a segment of
 * a checkpointed run for the adjoint. Asynchronous on the context's stream. */
int sem_run_snapshots(sem_ctx* ctx, int nsteps, float* u_dev);
/* The same, also recording seismograms into the device buffer seis_dev[nrec][3][nsteps]
 * (may be NULL) as sem_run_dev does: a forward run that keeps every displacement for the
 * adjoint (no recomputation), when [nsteps][nglob][3] floats fit in device memory. With the
 * fused sweep the snapshot of a step is taken when its receivers are sampled, before the
 * sweep; the wavefields and seismograms equal those of sem_run_dev bit for bit. */
int sem_run_record_snapshots(sem_ctx* ctx, int nsteps, float* seis_dev, float* u_dev);

/* Divergence watchdog: SEM_OK if every value of u, v and a is finite, SEM_EDIVERGED
 * otherwise (an explicit scheme run above its stability limit grows until it overflows).
 * Synchronous. */
int sem_check_finite(sem_ctx* ctx);

/* One matrix-free stiffness application on the device: f_dev = -K u_dev, both
 * [nglob][3] float32 in the caller's node order (Sec. II-B), by the element kernel, colour
 * by colour. Every node of f_dev is written. u_dev and f_dev must not overlap. Allocates
 * nothing. Asynchronous on the context's stream. Does not touch the solver state. */
int sem_apply_stiffness(sem_ctx* ctx, const float* u_dev, float* f_dev);

/* Same with node_stride floats per node, 3 or 4. Stride 3 is sem_apply_stiffness. Stride 4
 * is the solver's own field layout: [nglob][4] float32 (x, y, z and a 4th value that is
 * ignored and written as 0, arrays 16-byte aligned) in the solver's internal node order
 * (internal node i is caller node perm[i] of sem_node_order), evaluated by the kernel a
 * time step runs (SEM_OPT_ASSEMBLY), so this times the force sweep exactly as a step does. */
int sem_apply_stiffness_strided(sem_ctx* ctx, const float* u_dev, float* f_dev, int node_stride);

/* The solver's internal node order: perm[i] = caller node of internal node i, int32[nglob].
 * sem_set_mesh numbers the nodes so that every patch of the force sweep finds its nodes in
 * runs: the nodes a patch touches first (patch colour by patch colour) get consecutive
 * numbers, grouped by the set of patches that share them. Every call that takes or returns
 * node data (states, snapshots, sources, receivers, sem_apply_stiffness, sem_node_xyz)
 * uses the caller's order; only sem_apply_stiffness_strided with stride 4 uses this one.
 * SEM_ESTATE before sem_set_mesh. */
int sem_node_order(sem_ctx* ctx, int32_t* perm);

/* Discrete adjoint and material sensitivities of a seismogram loss L (one shot). From a
 * zero state the scheme is the leapfrog M(u^{n+1} - 2u^n + u^{n-1}) + dt^2 (K u^n - f^n) = 0
 * with u^0 = u^1 = 0; with G^m = dL/ds^m (s^m = u^m at the receivers, m = 1..N) the adjoint
 * runs backward, M(lam^{m-1} - 2 lam^m + lam^{m+1}) + dt^2 K lam^m = R^T G^m from
 * lam^N = lam^{N+1} = 0, and
 *   dL/dp = - sum_{n=1}^{N-1} (lam^n)^T [dM/dp (u^{n+1} - 2u^n + u^{n-1}) + dt^2 dK/dp u^n]
 * for p = rho, kappa, mu at every local point (Sec. II-B operator; the adjoint is not in the
 * paper). Usage: sem_adjoint_begin; for m = N down to 2: sem_adjoint_step(G^m) (lam becomes
 * lam^{m-1}), sem_adjoint_accumulate(u^{m-2}, u^{m-1}, u^m); then sem_adjoint_gradients.
 * Requires dt and one shot. G_dev: float32 [nrec][3] on the device, or NULL (zero);
 * u_*: displacement snapshots float32 [nglob][3] on the device. Gradients: float64 host
 * arrays [nspec][ngll^3] in the caller's element and point order (NULL = skip). */
int sem_adjoint_begin(sem_ctx* ctx);
int sem_adjoint_step(sem_ctx* ctx, const float* G_dev);
int sem_adjoint_accumulate(sem_ctx* ctx, const float* u_lo_dev, const float* u_mid_dev, const float* u_hi_dev);
int sem_adjoint_gradients(sem_ctx* ctx, double* g_rho, double* g_kappa, double* g_mu);
/* One segment of the backward sweep in a single call: with the adjoint at lam^{n0+count+1}
 * (and lam^{n0+count+2}), runs j = count down to 1: sem_adjoint_step(G_dev[j-1]) then
 * sem_adjoint_accumulate(u_dev[j-1], u_dev[j], u_dev[j+1]). G_dev: float32
 * [count][nrec][3] with G_dev[j-1] = G^{n0+j+1} (device; NULL = zero); u_dev: float32
 * [count+2][nglob][3] = u^{n0} .. u^{n0+count+1} (device). Asynchronous on the stream. */
int sem_adjoint_segment(sem_ctx* ctx, int count, const float* G_dev, const float* u_dev);

/* Autotuner of the force kernel's contraction form on this context's mesh (NGLL, element
 * shapes, shots): times `reps` stiffness sweeps (CUDA events, after one warm-up) with the
 * eta/zeta contractions done by line owners (form 1) and per point (form 2), keeps the
 * faster for every later step, and returns ms_out[0..1] (per sweep; may be NULL) and the
 * chosen form in *choice_out (may be NULL). Reads u, writes scratch only (completes a
 * pending state first). Synchronous. Requires mesh, material and dt. */
int sem_autotune(sem_ctx* ctx, int reps, double* ms_out, int* choice_out);

/* Autotuner of the element tile (the patch brick) for this order on the caller's mesh:
 * every brick shape bx x by x bz whose element count is the one a patch CTA holds at this
 * order (8 at NGLL 5: 2x2x2, 4x2x1, 8x1x1, ...; each side at most 16) is built on a scratch
 * context of the same order, device and stream from the given mesh (ibool with per-point
 * positions xyz[nspec][ngll^3][3] or trilinear corners ctrl[nspec][8][3]: exactly one
 * non-NULL) and material (rho, vp, vs per local point), and `reps` of its time steps (fused
 * sweep, dt at Courant number 0.4, from rest) are timed with sem_profile_steps after two of
 * warm-up. SEM_OPT_PATCH_SHAPE of ctx is set to the fastest, for the next sem_set_mesh on
 * ctx. shapes_out[k] (encoded as for SEM_OPT_PATCH_SHAPE) and ms_out[k] (ms of one step's
 * sweep) for the first max_shapes candidates (either may be NULL); *nshapes_out = the
 * number of candidates. Synchronous; allocates one scratch mesh at a time. */
int sem_tune_patch_shape(sem_ctx* ctx, int nspec, int nglob, const int32_t* ibool, const double* xyz,
                         const double* ctrl, const float* rho, const float* vp, const float* vs, int reps,
                         int max_shapes, int32_t* shapes_out, double* ms_out, int* nshapes_out);

/* Profile nsteps time steps (Sec. I, IV-C), launched one by one with CUDA events on the
 * context's stream around each step's force sweep: ms_out[0] = mean milliseconds of the
 * sweep (all of its colour launches; with SEM_OPT_FUSED_NEWMARK the Newmark update and the
 * sources included), ms_out[1] = mean milliseconds per step of everything else (receiver
 * sampling, separate Newmark passes, the predictor that starts a run). The state advances
 * as with sem_step (same results); no seismogram is recorded. Blocks until the steps are
 * done. SEM_EINVAL if nsteps < 1 or ms_out is NULL. */
int sem_profile_steps(sem_ctx* ctx, int nsteps, double* ms_out);

/* Groups: several contexts on one GPU (different meshes, orders, shot counts) stepped
 * together. sem_group_step advances every context nsteps steps (no seismograms): one eager
 * step per context, then CUDA graphs of the remaining steps. In the persistent mode
 * (SEM_GROUP_MODE 1; used when every context has one shot, SEM_OPT_ASSEMBLY 0 and at most
 * 64 patch colours, and the group at most 64 contexts) a step is the contexts'
 * Newmark passes, ONE persistent force-sweep launch for all contexts of the same order and
 * contraction form (CTAs take the patches of every model colour by colour from a device
 * counter; a patch of colour c writes once its own model's colour c - 1 is done, a bounded
 * wait: if one gives up, sem_group_sync returns SEM_ETIMEOUT), and the contexts' sources;
 * otherwise (mode 0, the default: measured faster on GB300 for 16 cubes of 8^3 .. 40^3 at
 * NGLL 4 .. 8, 151 ms against 172 ms for 50 steps) every context's steps form a branch of
 * their own in the graph, so that small models run side by side. Either way each context's
 * results equal those of sem_step
 * on it alone, bit for bit. The contexts stay owned by the caller, must outlive the group,
 * and may be changed between calls (the graphs are rebuilt). Asynchronous: every context's
 * later calls are ordered after the group's work. */
typedef struct sem_group sem_group;
int sem_group_create(sem_group** out, int nctx, sem_ctx* const* ctxs);
int sem_group_destroy(sem_group* group);
int sem_group_step(sem_group* group, int nsteps);
int sem_group_sync(sem_group* group);
const char* sem_group_last_error(const sem_group* group);
/* Group options: SEM_GROUP_MODE (0 graph branches, 1 persistent sweeps); SEM_GROUP_STALL_TEST
 * (failure-detection test, one-shot: 1 makes the first persistent step of the next
 * sem_group_step with more than one step wait for counts that never arrive, so that its
 * bounded waits give up and sem_group_sync returns SEM_ETIMEOUT; the steps after it run
 * normally). SEM_EINVAL for an unknown option or value. */
#define SEM_GROUP_MODE 1
#define SEM_GROUP_STALL_TEST 2
int sem_group_set_option(sem_group* group, int option, long long value);
/* out[0] = 1 if the group's steps run as persistent sweeps, out[1] = the sweep launches per
 * step (distinct orders and contraction forms). */
int sem_group_info(sem_group* group, int* out);

/* Kinetic and potential energy of the current state in float64:
 * out[0] = 1/2 sum_I M_I |v_I|^2, out[1] = 1/2 u^T K u. Synchronous. */
int sem_energy(sem_ctx* ctx, double* out);

/* Energy sums for callers that cannot allocate device memory: code that runs where
 * cudaMalloc is unavailable or forbidden, such as a host application whose device memory
 * is owned by another runtime's pool, or a caller inside a region that must not allocate.
 * The paper has no counterpart; it is a variant of the reduction behind sem_energy.
 * Inputs: u_dev, v_dev, f_dev device arrays [nglob][3] float32 on the context's GPU, with
 * f_dev = -K u_dev (for instance from sem_apply_stiffness, which allocates nothing), all in
 * the caller's node order; the context supplies the inverse mass. Output: out[0] = 1/2 sum_I M_I |v_I|^2,
 * out[1] = -1/2 u.f = 1/2 u^T K u, host memory, float64. nglob must equal the mesh's.
 * Scratch: the per-block partial sums go to a fixed 64 KiB array in the library's device
 * memory (one per GPU that loads the library, held until the process exits), never to
 * cudaMalloc; the call makes no device or host allocation. It supports at most
 * 67,108,864 nodes and returns SEM_EINVAL with a message beyond that. All calls share the
 * array, which keeps the last call's contents, so calls that overlap on the GPU (from
 * several threads or contexts at once) race; each call rewrites every slot it reads.
 * Every call looks up the array's device address on the context's device
 * (cudaGetSymbolAddress, which allocates nothing). The call synchronizes with the context's
 * stream, so it must not be made while that stream is capturing a graph: it then returns
 * SEM_ESTATE without doing anything. Synchronous on the context's stream. */
int sem_energy_noalloc(sem_ctx* ctx, int nglob, const float* u_dev, const float* v_dev, const float* f_dev,
                       double* out);

/* Wait for all work issued on the context's stream. */
int sem_sync(sem_ctx* ctx);

/* Sizes of the set-up problem: out[0] nspec, out[1] nglob, out[2] ngll, out[3] ncolors,
 * out[4] steps taken since sem_set_state, out[5] bytes of device memory held,
 * out[6] shots, out[7] slabs of the sweep order, out[8] force-kernel launches per sweep.
 * out has room for 9 values; an entry not yet defined is 0. */
int sem_info(sem_ctx* ctx, int64_t* out);

/* Element count of each colour, counts[ncolors] (see sem_info for ncolors). */
int sem_color_counts(sem_ctx* ctx, int32_t* counts);

/* The patches of the force sweep (SEM_OPT_ASSEMBLY): out[0] patches, out[1] patch colours
 * (launches per sweep), out[2] largest patch node count, out[3] distinct patch tables (one
 * for every patch of the same local structure), out[4..6] the brick in elements along the
 * mesh's lattice x, y, z, out[7] the assembly option in force. out has room for 8 values.
 * SEM_ESTATE before sem_set_mesh. */
int sem_patch_info(sem_ctx* ctx, int64_t* out);

/* Message of the last failed call on ctx, or of the last failed context-free call when
 * ctx is NULL. Owned by the library; valid until the next call on the same ctx. */
const char* sem_last_error(const sem_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* SEM_H */
