"""GPU parity of the patch assembly (SEM_OPT_ASSEMBLY = 0, the force sweep of every time
step) with the FP64 oracle, through the C ABI.

The patch kernel sums the forces meeting at a node inside a patch before adding them to the
node, so its float32 result differs from the element kernel's only in the order of those
sums: both meet the stiffness bar against the oracle (relative L2 2e-6, every entry within
1e-5 of the largest; derivation in test_gpu_parity.py) and agree with each other to 1e-6.
Caller-side node and element numberings are scrambled in one test so that every mapping
between the caller's and the solver's internal node order is exercised."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2606_12850_gb300 import build, inputs, sem  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_KU_L2 = 2e-6
TOL_KU_MAX = 1e-5


@pytest.fixture(scope="module", autouse=True)
def library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return sem.lib()


@pytest.fixture(scope="module")
def oracle():
    from oracle import sem_oracle
    return sem_oracle


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def check_forces(f, f_ref):
    assert rel_l2(f, f_ref) <= TOL_KU_L2
    assert np.max(np.abs(f - f_ref)) <= TOL_KU_MAX * np.max(np.abs(f_ref))


def material(mesh, seed):
    shape = mesh.ibool.shape
    rho = inputs.uniform(seed, shape, 2000.0, 3000.0, stream=1).astype(np.float32)
    vp = inputs.uniform(seed, shape, 3000.0, 5000.0, stream=2).astype(np.float32)
    vs = (vp / inputs.uniform(seed, shape, 1.6, 2.0, stream=3)).astype(np.float32)
    return rho, vp, vs


def make_ctx(ngll, ibool, ctrl, nglob, mat):
    ctx = sem.sem_create(ngll, 0)
    sem.sem_set_mesh_corners(ctx, ibool, ctrl, nglob)
    sem.sem_set_material(ctx, *mat)
    return ctx


def sweep_stride4(ctx, u, assembly):
    """f = -K u through the stride-4 entry point in the solver's internal order, returned in
    caller order."""
    perm = sem.sem_node_order(ctx)
    u4 = np.zeros((len(perm), 4), dtype=np.float32)
    u4[:, :3] = u[perm]
    sem.sem_set_option(ctx, sem.SEM_OPT_ASSEMBLY, assembly)
    torch.cuda.synchronize()
    ud = torch.from_numpy(u4).cuda()
    fd = torch.full_like(ud, float("nan"))
    torch.cuda.synchronize()
    sem.sem_apply_stiffness_strided(ctx, ud, fd, 4)
    sem.sem_sync(ctx)
    f = np.empty((len(perm), 4), dtype=np.float32)
    f[perm] = fd.cpu().numpy()
    assert np.all(f[:, 3] == 0.0)
    return f[:, :3]


BRICK = {2: (4, 4, 4), 3: (3, 3, 3), 4: (4, 2, 2), 5: (1, 4, 2), 6: (2, 2, 1), 7: (1, 2, 2), 8: (2, 2, 1),
         9: (3, 1, 1), 10: (2, 1, 1)}


@pytest.mark.parametrize("ngll", [2, 3, 4, 5, 6, 7, 8, 9, 10])
def test_patch_forces_match_oracle(oracle, ngll):
    """Jittered mesh with random per-point material, ragged in every direction (brick counts
    that do not divide the mesh), several patches per colour."""
    bx, by, bz = BRICK[ngll]
    n = (2 * bx + 1, 2 * by + 1, bz + 2)
    mesh = inputs.structured_hex_mesh(n, ngll, (1000.0, 900.0, 800.0), jitter=0.15, seed=ngll)
    mat = material(mesh, 20 + ngll)
    ctx = make_ctx(ngll, mesh.ibool, mesh.ctrl, mesh.nglob, mat)
    info = sem.sem_patch_info(ctx)
    assert info["patches"] > info["colors"] and (info["bx"], info["by"], info["bz"]) == BRICK[ngll]
    u = inputs.random_field(mesh.nglob, 30 + ngll)
    f_ref = oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, *mat, ngll).forces(u.astype(np.float64))
    f_patch = sweep_stride4(ctx, u, 0)
    check_forces(f_patch, f_ref)
    f_elem = sweep_stride4(ctx, u, 1)
    check_forces(f_elem, f_ref)
    assert rel_l2(f_patch, f_elem.astype(np.float64)) <= 1e-6
    # bitwise reproducible
    assert np.array_equal(f_patch, sweep_stride4(ctx, u, 0))


def test_scrambled_caller_numbering(oracle):
    """Elements and nodes numbered at random by the caller: the forces, a short run's state
    and its seismograms still match the oracle on the caller's numbering."""
    mesh = inputs.structured_hex_mesh((5, 4, 4), 5, 1000.0, jitter=0.1, seed=9)
    rng = np.random.default_rng(5)
    eperm = rng.permutation(mesh.nspec)
    nperm = rng.permutation(mesh.nglob)  # caller node -> scrambled id
    ib = nperm[mesh.ibool[eperm]].astype(np.int32)
    ctrl = mesh.ctrl[eperm]
    mat = tuple(m[eperm] for m in material(mesh, 4))
    ctx = make_ctx(5, ib, ctrl, mesh.nglob, mat)
    model = oracle.Model(ib, ctrl, mesh.nglob, *mat, 5)
    u = inputs.random_field(mesh.nglob, 6)
    f_ref = model.forces(u.astype(np.float64))
    check_forces(sweep_stride4(ctx, u, 0), f_ref)
    # time stepping with a source and receivers on scrambled node ids
    sem.sem_set_option(ctx, sem.SEM_OPT_ASSEMBLY, 0)
    dt = sem.sem_suggest_dt(ctx, 0.4)
    sem.sem_set_dt(ctx, dt)
    src = np.array([nperm[mesh.nglob // 2]], dtype=np.int32)
    rec = nperm[np.arange(0, mesh.nglob, mesh.nglob // 7)[:6]].astype(np.int32)
    force = np.array([[0.0, 0.0, 1e10]])
    sem.sem_set_source_nodes(ctx, src, force, 10.0, 0.12)
    sem.sem_set_receiver_nodes(ctx, rec)
    sem.sem_set_state(ctx)
    nsteps = 60
    seis = sem.sem_run(ctx, nsteps)
    u_gpu, _, _ = sem.sem_get_state(ctx, want=(True, False, False))
    seis_ref, u_ref, _, _ = oracle.newmark_run(model, dt, nsteps, src_nodes=src, src_force=force, f0=10.0, t0=0.12,
                                              rec_nodes=rec)
    assert rel_l2(u_gpu.reshape(-1, 3), u_ref) <= 2e-5
    assert rel_l2(seis, seis_ref) <= 1e-4


def test_patch_and_element_time_steps_agree():
    """200 steps of the homogeneous 8^3 cube with either assembly: the two runs differ only by
    the order of float32 sums at nodes."""
    w = inputs.homogeneous_cube()
    outs = []
    for asm in (0, 1):
        s = sem.setup_workload(w, device=0)
        sem.sem_set_option(s.ctx, sem.SEM_OPT_ASSEMBLY, asm)
        seis = sem.sem_run(s.ctx, 200)
        u, _, _ = sem.sem_get_state(s.ctx, want=(True, False, False))
        outs.append((seis, u))
    assert rel_l2(outs[0][1], outs[1][1].astype(np.float64)) <= 2e-6
    assert rel_l2(outs[0][0], outs[1][0].astype(np.float64)) <= 2e-6


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 3), (3, 1, 1)])
def test_patch_degenerate_meshes(oracle, shape):
    """A single element (a patch without shared nodes) and single rows of elements."""
    mesh = inputs.structured_hex_mesh(shape, 5, (300.0, 200.0, 250.0), jitter=0.0)
    mat = material(mesh, 8)
    ctx = make_ctx(5, mesh.ibool, mesh.ctrl, mesh.nglob, mat)
    u = inputs.random_field(mesh.nglob, 12)
    f_ref = oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, *mat, 5).forces(u.astype(np.float64))
    check_forces(sweep_stride4(ctx, u, 0), f_ref)


def test_persistent_sweep_equals_colour_launches():
    """All colours in one persistent launch (assembly 2) against one launch per patch colour
    (assembly 0): the same sums in the same order, so bitwise equal; repeated sweeps too
    (the launch's counters reset themselves)."""
    mesh = inputs.structured_hex_mesh((9, 7, 6), 5, 1000.0, jitter=0.1, seed=3)
    mat = material(mesh, 13)
    ctx = make_ctx(5, mesh.ibool, mesh.ctrl, mesh.nglob, mat)
    u = inputs.random_field(mesh.nglob, 14)
    f0 = sweep_stride4(ctx, u, 0)
    f2 = sweep_stride4(ctx, u, 2)
    assert np.array_equal(f0, f2)
    for _ in range(3):
        assert np.array_equal(sweep_stride4(ctx, u, 2), f0)


def test_persistent_sweep_wait_gives_up_and_recovers(oracle):
    """Failure detection without a fault: a sweep whose waits target a count that never
    arrives gives up within its bound, the host reads SEM_ETIMEOUT, and the next sweep is
    complete and correct."""
    mesh = inputs.structured_hex_mesh((6, 4, 4), 5, 800.0, jitter=0.1, seed=5)
    mat = material(mesh, 15)
    ctx = make_ctx(5, mesh.ibool, mesh.ctrl, mesh.nglob, mat)
    u = inputs.random_field(mesh.nglob, 16)
    sem.sem_set_option(ctx, sem.SEM_OPT_ASSEMBLY, 2)
    sem.sem_set_option(ctx, sem.SEM_OPT_SWEEP_STALL_TEST, 1)
    perm = sem.sem_node_order(ctx)
    u4 = np.zeros((len(perm), 4), dtype=np.float32)
    u4[:, :3] = u[perm]
    torch.cuda.synchronize()
    ud = torch.from_numpy(u4).cuda()
    fd = torch.zeros_like(ud)
    torch.cuda.synchronize()
    sem.sem_apply_stiffness_strided(ctx, ud, fd, 4)
    with pytest.raises(sem.SemError) as ei:
        sem.sem_sync(ctx)
    assert ei.value.code == -5 and "gave up" in str(ei.value)
    sem.sem_sync(ctx)  # the flag was cleared
    f_ref = oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, *mat, 5).forces(u.astype(np.float64))
    check_forces(sweep_stride4(ctx, u, 2), f_ref)


@pytest.mark.parametrize("ngll", [5, 9])
def test_atomic_ablation_agrees_within_rounding(oracle, ngll):
    """The colouring ablation (one launch, float atomics; assembly 3) computes the same
    forces up to the order of float32 sums: within the stiffness bar of the oracle and 1e-6
    of the coloured element kernel."""
    mesh = inputs.structured_hex_mesh((4, 3, 3), ngll, 900.0, jitter=0.1, seed=21)
    mat = material(mesh, 22)
    ctx = make_ctx(ngll, mesh.ibool, mesh.ctrl, mesh.nglob, mat)
    u = inputs.random_field(mesh.nglob, 23)
    f_atomic = sweep_stride4(ctx, u, 3)
    f_elem = sweep_stride4(ctx, u, 1)
    check_forces(f_atomic, oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, *mat, ngll).forces(u.astype(np.float64)))
    assert rel_l2(f_atomic, f_elem.astype(np.float64)) <= 1e-6


def test_patch_shape_tuner_and_option(oracle):
    """The element-tile autotuner times every brick shape of the order's patch CTA (8
    elements at NGLL 5) on the caller's mesh and sets the fastest for the next sem_set_mesh;
    non-default bricks (elongated 8x1x1, 1x2x4) through SEM_OPT_PATCH_SHAPE meet the
    stiffness bar, a brick larger than the CTA holds is refused, and a time step on a
    non-default brick runs the fused Newmark update bitwise like the separate passes."""
    mesh = inputs.structured_hex_mesh((6, 5, 4), 5, 1000.0, jitter=0.1, seed=31)
    mat = material(mesh, 33)
    ctx = sem.sem_create(5, 0)
    rows, best = sem.sem_tune_patch_shape(ctx, mesh.ibool, mesh.nglob, *mat, ctrl=mesh.ctrl, reps=3)
    shapes = [r[0] for r in rows]
    assert len(shapes) == 10 and (2, 2, 2) in shapes and all(bx * by * bz == 8 for bx, by, bz in shapes)
    assert all(ms > 0 for _, ms in rows)
    sem.sem_set_mesh_corners(ctx, mesh.ibool, mesh.ctrl, mesh.nglob)
    sem.sem_set_material(ctx, *mat)
    info = sem.sem_patch_info(ctx)
    assert (info["bx"], info["by"], info["bz"]) == best
    u = inputs.random_field(mesh.nglob, 34)
    f_ref = oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, *mat, 5).forces(u.astype(np.float64))
    check_forces(sweep_stride4(ctx, u, 0), f_ref)
    with pytest.raises(sem.SemError):
        sem.sem_set_option(ctx, sem.SEM_OPT_PATCH_SHAPE, sem.patch_shape_code(3, 3, 1))
    for shape in ((8, 1, 1), (1, 2, 4)):
        c2 = sem.sem_create(5, 0)
        sem.sem_set_option(c2, sem.SEM_OPT_PATCH_SHAPE, sem.patch_shape_code(*shape))
        sem.sem_set_mesh_corners(c2, mesh.ibool, mesh.ctrl, mesh.nglob)
        sem.sem_set_material(c2, *mat)
        info = sem.sem_patch_info(c2)
        assert (info["bx"], info["by"], info["bz"]) == shape
        check_forces(sweep_stride4(c2, u, 0), f_ref)
    outs = []
    for fused in (0, 1):
        c3 = sem.sem_create(5, 0)
        sem.sem_set_option(c3, sem.SEM_OPT_PATCH_SHAPE, sem.patch_shape_code(4, 2, 1))
        sem.sem_set_mesh_corners(c3, mesh.ibool, mesh.ctrl, mesh.nglob)
        sem.sem_set_material(c3, *mat)
        sem.sem_set_option(c3, sem.SEM_OPT_FUSED_NEWMARK, fused)
        sem.sem_set_dt(c3, sem.sem_suggest_dt(c3, 0.4))
        sem.sem_set_source_nodes(c3, np.array([mesh.ibool[mesh.nspec // 2, 0]], dtype=np.int32),
                                 np.array([[1e10, 2e10, -1e10]]), 10.0, 0.0)
        sem.sem_set_receiver_nodes(c3, np.arange(0, mesh.nglob, 101, dtype=np.int32))
        sem.sem_set_state(c3)
        seis = sem.sem_run(c3, 14)
        outs.append((seis,) + tuple(sem.sem_get_state(c3)))
    assert np.abs(outs[0][0]).max() > 0
    for x, y in zip(*outs):
        assert np.array_equal(x, y)
