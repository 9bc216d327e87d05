"""GPU parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances:
* one stiffness application f = -K u on random u: relative L2 <= 2e-6 and every entry
  within 1e-5 * max|f|. FP32 unit roundoff is 6e-8; an entry of f is a sum of about
  2N + 25 rounded products per quadrature point (derivative, chain rule, stress, flux,
  transposed product) and up to 8 element contributions; rounding errors that add like a
  random walk give sqrt(40) * 6e-8 ~ 4e-7 relative to the magnitude of the terms, and
  random u cancels up to a factor of ~5 between the terms and the result: 2e-6.
* wavefield after 200 steps: relative L2 <= 2e-5; seismograms: relative L2 <= 1e-4
  (the solver's stated accuracy targets for the homogeneous 8^3 cube).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2606_12850_gb300 import build, inputs, sem  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_KU_L2 = 2e-6
TOL_KU_MAX = 1e-5
TOL_WAVEFIELD = 2e-5
TOL_SEIS = 1e-4


@pytest.fixture(scope="module", autouse=True)
def library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return sem.lib()


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def random_material(mesh, seed):
    shape = mesh.ibool.shape
    rho = inputs.uniform(seed, shape, 2000.0, 3000.0, stream=1).astype(np.float32)
    vp = inputs.uniform(seed, shape, 3000.0, 5000.0, stream=2).astype(np.float32)
    vs = (vp / inputs.uniform(seed, shape, 1.6, 2.0, stream=3)).astype(np.float32)
    return rho, vp, vs


def make_ctx(mesh, rho, vp, vs):
    ctx = sem.sem_create(mesh.ngll, 0)
    sem.sem_set_mesh_corners(ctx, mesh.ibool, mesh.ctrl, mesh.nglob)
    sem.sem_set_material(ctx, rho, vp, vs)
    return ctx


def gpu_forces(ctx, u):
    torch.cuda.synchronize()
    ud = torch.from_numpy(np.ascontiguousarray(u, dtype=np.float32)).cuda()
    fd = torch.full_like(ud, float("nan"))
    torch.cuda.synchronize()
    sem.sem_apply_stiffness(ctx, ud, fd)
    sem.sem_sync(ctx)
    return fd.cpu().numpy()


def check_forces(f_gpu, f_ref):
    assert np.all(np.isfinite(f_gpu))
    err = rel_l2(f_gpu, f_ref)
    assert err <= TOL_KU_L2, err
    assert np.abs(f_gpu - f_ref).max() <= TOL_KU_MAX * np.abs(f_ref).max()
    return err


@pytest.mark.parametrize("ngll", range(2, 11))
def test_stiffness_every_order(oracle, ngll):
    """f = -K u for NGLL = 2..10 on a jittered 3x2x2 mesh with random per-point material:
    ragged colour classes (1-2 elements each), every element-per-CTA tail."""
    mesh = inputs.structured_hex_mesh((3, 2, 2), ngll, (900.0, 600.0, 600.0), jitter=0.2, seed=ngll)
    mat = random_material(mesh, 40 + ngll)
    ctx = make_ctx(mesh, *mat)
    u = inputs.random_field(mesh.nglob, 100 + ngll)
    f_ref = oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, *mat, ngll).forces(u.astype(np.float64))
    check_forces(gpu_forces(ctx, u), f_ref)


@pytest.mark.parametrize("ngll,n", [(3, (9, 8, 7)), (5, (7, 6, 5)), (7, (5, 4, 4)), (9, (4, 3, 3))])
def test_stiffness_several_tiles(oracle, ngll, n):
    """Meshes spanning many CTAs per colour with a ragged last CTA."""
    mesh = inputs.structured_hex_mesh(n, ngll, 1000.0, jitter=0.1, seed=3)
    mat = random_material(mesh, 7)
    ctx = make_ctx(mesh, *mat)
    u = inputs.random_field(mesh.nglob, 11)
    f_ref = oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, *mat, ngll).forces(u.astype(np.float64))
    check_forces(gpu_forces(ctx, u), f_ref)


def test_stiffness_strided_matches(oracle):
    """The stride-4 entry point (the solver's own field layout, internal node order) gives
    the same forces."""
    mesh = inputs.structured_hex_mesh((4, 3, 3), 5, 600.0, jitter=0.2, seed=2)
    mat = random_material(mesh, 3)
    ctx = make_ctx(mesh, *mat)
    perm = sem.sem_node_order(ctx)
    assert np.array_equal(np.sort(perm), np.arange(mesh.nglob))
    u = inputs.random_field(mesh.nglob, 4)
    u4 = np.zeros((mesh.nglob, 4), dtype=np.float32)
    u4[:, :3] = u[perm]
    torch.cuda.synchronize()
    ud = torch.from_numpy(u4).cuda()
    fd = torch.full_like(ud, float("nan"))
    torch.cuda.synchronize()
    sem.sem_apply_stiffness_strided(ctx, ud, fd, 4)
    sem.sem_sync(ctx)
    f4 = np.empty((mesh.nglob, 4), dtype=np.float32)
    f4[perm] = fd.cpu().numpy()
    f_ref = oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, *mat, 5).forces(u.astype(np.float64))
    check_forces(f4[:, :3], f_ref)
    assert np.all(f4[:, 3] == 0.0)
    f3 = gpu_forces(ctx, u)  # same arithmetic; the compiler may contract differently
    assert rel_l2(f4[:, :3], f3.astype(np.float64)) <= 1e-6
    assert sem.lib().sem_apply_stiffness_strided(ctx.handle, sem._P(ud.data_ptr()), sem._P(fd.data_ptr()), 5) == -1


def test_stiffness_periodic(oracle):
    """Periodic numbering (wrapped ibool, 8 colours for an even lattice, 27 for an odd one)."""
    for n in (2, 3, 4):
        mesh = inputs.structured_hex_mesh(n, 4, 300.0, periodic=True)
        mat = random_material(mesh, n)
        ctx = make_ctx(mesh, *mat)
        u = inputs.random_field(mesh.nglob, n)
        f_ref = oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, *mat, 4).forces(u.astype(np.float64))
        check_forces(gpu_forces(ctx, u), f_ref)


def test_single_element(oracle):
    mesh = inputs.structured_hex_mesh(1, 5, 100.0)
    mat = random_material(mesh, 1)
    ctx = make_ctx(mesh, *mat)
    assert sem.sem_info(ctx)["ncolors"] == 1
    u = inputs.random_field(mesh.nglob, 2)
    f_ref = oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, *mat, 5).forces(u.astype(np.float64))
    check_forces(gpu_forces(ctx, u), f_ref)


@pytest.fixture(scope="module")
def cube_reference(oracle):
    w = inputs.homogeneous_cube()
    return w, oracle.run_workload(w)


def test_homogeneous_cube_200_steps(cube_reference):
    """The 8^3 homogeneous cube at NGLL=5 for 200 Newmark steps: the library's own CFL step
    and node location agree with the oracle's, the FP32 wavefield matches the FP64
    oracle to 2e-5 and the seismograms to 1e-4 (relative L2)."""
    w, ref = cube_reference
    s = sem.setup_workload(w)
    assert abs(s.dt / ref["dt"] - 1.0) < 1e-12
    assert list(s.src_nodes) == list(ref["src"])
    assert list(s.rec_nodes) == list(ref["rec"])
    seis = sem.sem_run(s.ctx, w.nsteps)
    u, v, a = sem.sem_get_state(s.ctx)
    e_u = rel_l2(u, ref["u"])
    e_v = rel_l2(v, ref["v"])
    e_s = rel_l2(seis, ref["seis"])
    assert e_u <= TOL_WAVEFIELD, e_u
    assert e_v <= TOL_WAVEFIELD, e_v
    assert e_s <= TOL_SEIS, e_s
    worst = max(rel_l2(seis[r], ref["seis"][r]) for r in range(seis.shape[0]))
    assert worst <= 2 * TOL_SEIS, worst


def test_step_paths_bitwise_equal(cube_reference):
    """Graph-captured steps (10 per graph), eager steps and separate calls give bitwise
    identical states, and two runs agree bitwise (coloured assembly is deterministic)."""
    w, _ = cube_reference
    states = []
    for chunks in ((25,), (1,) * 25, (7, 3, 15), (25,)):
        s = sem.setup_workload(w)
        for c in chunks:
            sem.sem_step(s.ctx, c)
        states.append(sem.sem_get_state(s.ctx))
    for st in states[1:]:
        for x, y in zip(states[0], st):
            assert np.array_equal(x, y)


def test_run_resumes_after_get_state(cube_reference):
    """Reading the state mid-run (which completes the pending corrector) does not change
    the trajectory beyond rounding of the completed velocity."""
    w, ref = cube_reference
    s = sem.setup_workload(w)
    a = sem.sem_run(s.ctx, 60)
    sem.sem_get_state(s.ctx)
    b = sem.sem_run(s.ctx, 140)
    seis = np.concatenate([a, b], axis=2)
    assert rel_l2(seis, ref["seis"]) <= TOL_SEIS


def test_energy_matches_oracle(oracle):
    """Kinetic and potential energy from sem_energy track the oracle's FP64 energies along
    a source-free run from a smooth initial displacement."""
    mesh = inputs.structured_hex_mesh(4, 5, 800.0, jitter=0.15, seed=9)
    mat = random_material(mesh, 5)
    m = oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, *mat, 5)
    X = m.node_xyz
    u0 = (np.sin(X / 300.0) * 1e-3).astype(np.float32)
    dt = m.cfl_dt(0.4)
    ctx = make_ctx(mesh, *mat)
    sem.sem_set_dt(ctx, dt)
    sem.sem_set_state(ctx, u=u0)
    u = u0.astype(np.float64)
    v = np.zeros_like(u)
    a = np.zeros_like(u)
    for chunk in (0, 50, 150):
        if chunk:
            sem.sem_step(ctx, chunk)
            _, u, v, a = oracle.newmark_run(m, dt, chunk, u0=u, v0=v, a0=a)
        kin, pot = sem.sem_energy(ctx)
        kin_ref = 0.5 * np.sum(m.mass[:, None] * v * v)
        pot_ref = -0.5 * np.sum(u * m.forces(u))
        assert abs(pot - pot_ref) <= 1e-5 * (kin_ref + pot_ref)
        assert abs(kin - kin_ref) <= 1e-5 * (kin_ref + pot_ref)


def test_zero_steps_and_empty_sources(cube_reference):
    w, _ = cube_reference
    s = sem.setup_workload(w)
    sem.sem_set_source_nodes(s.ctx, [], np.zeros((0, 3)), w.f0, w.t0)
    sem.sem_set_receiver_nodes(s.ctx, [])
    assert sem.sem_run(s.ctx, 0) is None
    assert sem.sem_run(s.ctx, 15) is None
    u, v, a = sem.sem_get_state(s.ctx)
    assert not np.any(u) and not np.any(v) and not np.any(a)
    assert sem.sem_info(s.ctx)["steps"] == 15


def test_duplicate_sources_merge(oracle):
    """Two sources on one node act as their sum."""
    w = inputs.homogeneous_cube(n=4, side=500.0, nsteps=30)
    s1 = sem.setup_workload(w)
    node = s1.src_nodes[0]
    seis1 = sem.sem_run(s1.ctx, 30)
    s2 = sem.setup_workload(w)
    f = w.source_force[0]
    sem.sem_set_source_nodes(s2.ctx, [node, node], [0.25 * f, 0.75 * f], w.f0, w.t0)
    seis2 = sem.sem_run(s2.ctx, 30)
    assert rel_l2(seis2, seis1.astype(np.float64)) < 1e-6


def test_argument_errors():
    mesh = inputs.structured_hex_mesh(2, 3, 100.0)
    ctx = sem.sem_create(3, 0)
    rho, vp, vs = random_material(mesh, 1)
    ptr = lambda a: a.ctypes.data_as(sem._P)
    assert sem.lib().sem_set_material(ctx.handle, ptr(rho), ptr(vp), ptr(vs)) == -4  # before the mesh
    assert "sem_set_mesh" in sem.sem_last_error(ctx)
    bad = mesh.ibool.copy()
    bad[0, 0] = -1
    with pytest.raises(sem.SemError) as ei:
        sem.sem_set_mesh_corners(ctx, bad, mesh.ctrl, mesh.nglob)
    assert ei.value.code == -1
    with pytest.raises(sem.SemError):
        sem.sem_set_mesh_corners(ctx, mesh.ibool, mesh.ctrl, mesh.nglob + 1)  # unreferenced node
    inverted = mesh.ctrl.copy()
    inverted[0, [0, 1]] = inverted[0, [1, 0]]
    with pytest.raises(sem.SemError) as ei:
        sem.sem_set_mesh_corners(ctx, mesh.ibool, inverted, mesh.nglob)
    assert "Jacobian" in str(ei.value)
    sem.sem_set_mesh_corners(ctx, mesh.ibool, mesh.ctrl, mesh.nglob)
    with pytest.raises(sem.SemError) as ei:
        sem.sem_step(ctx, 1)
    assert ei.value.code == -4
    rho, vp, vs = random_material(mesh, 2)
    with pytest.raises(sem.SemError):
        sem.sem_set_material(ctx, rho, vs, vp)  # vp < vs
    sem.sem_set_material(ctx, rho, vp, vs)
    with pytest.raises(sem.SemError):
        sem.sem_set_dt(ctx, -1.0)
    with pytest.raises(sem.SemError):
        sem.sem_set_source_nodes(ctx, [mesh.nglob], [[0, 0, 1.0]], 10.0, 0.1)
    v = np.ones((mesh.nglob, 3), dtype=np.float32)
    v[3, 1] = np.nan
    with pytest.raises(sem.SemError) as ei:
        sem.sem_set_state(ctx, None, v, None)
    assert ei.value.code == -1 and "non-finite" in str(ei.value)
    _, v_now, _ = sem.sem_get_state(ctx)
    assert not np.any(v_now)  # the rejected state was reset to zero


def test_plane_wave_periodic(oracle):
    """Travelling plane wave in a periodic box: GPU seismograms match the oracle's."""
    L = 1000.0
    mesh = inputs.structured_hex_mesh((2, 2, 3), 5, (2 * L / 3, 2 * L / 3, L), periodic=True)
    one = np.ones(mesh.nspec)
    mat = (inputs.per_point(mesh, 2500 * one), inputs.per_point(mesh, 3000 * one), inputs.per_point(mesh, 1730 * one))
    m = oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, *mat, 5)
    k = 2 * np.pi / L
    w = 3000.0 * k
    z = m.node_xyz[:, 2]
    u0 = np.zeros((m.nglob, 3))
    u0[:, 2] = np.sin(k * z)
    v0 = np.zeros((m.nglob, 3))
    v0[:, 2] = -w * np.cos(k * z)
    a0 = m.forces(u0) / m.mass[:, None]
    dt = m.cfl_dt(0.4)
    n = 150
    rec = np.arange(0, m.nglob, 97)
    seis_ref, u_ref, *_ = oracle.newmark_run(m, dt, n, u0=u0, v0=v0, a0=a0, rec_nodes=rec)
    ctx = make_ctx(mesh, *mat)
    sem.sem_set_dt(ctx, dt)
    sem.sem_set_receiver_nodes(ctx, rec)
    sem.sem_set_state(ctx, u0.astype(np.float32), v0.astype(np.float32), a0.astype(np.float32))
    seis = sem.sem_run(ctx, n)
    assert rel_l2(seis, seis_ref) <= TOL_SEIS
    u, _, _ = sem.sem_get_state(ctx)
    assert rel_l2(u, u_ref) <= TOL_WAVEFIELD


def test_divergence_watchdog():
    """Failure detection without a GPU fault: a time step 3x above the CFL limit makes the
    explicit scheme blow up to Inf; sem_run reports SEM_EDIVERGED and the context stays
    usable (a fresh state with a stable dt runs again)."""
    w = inputs.homogeneous_cube(n=4, side=500.0, nsteps=400)
    s = sem.setup_workload(w)
    dt_cfl = sem.sem_suggest_dt(s.ctx, 1.0)
    sem.sem_set_dt(s.ctx, 3.0 * dt_cfl)
    sem.sem_set_state(s.ctx, inputs.random_field(s.ctx.nglob, 3, scale=1e-6))
    with pytest.raises(sem.SemError) as ei:
        sem.sem_run(s.ctx, 400)
    assert ei.value.code == -6 and "non-finite" in str(ei.value)
    sem.sem_set_dt(s.ctx, s.dt)
    sem.sem_set_state(s.ctx)
    sem.sem_run(s.ctx, 20)
    sem.sem_check_finite(s.ctx)


def test_sweep_slabs_option(oracle):
    """A slab-major sweep order (SEM_OPT_SWEEP_SLABS) gives the same stiffness action up to
    the summation order at nodes, and sem_info reports the slabs and launches."""
    mesh = inputs.structured_hex_mesh((6, 4, 4), 4, (1200.0, 800.0, 800.0), jitter=0.1, seed=3)
    mat = random_material(mesh, 71)
    u = inputs.random_field(mesh.nglob, 72)
    out = []
    for K in (1, 3):
        ctx = sem.sem_create(mesh.ngll, 0)
        sem.sem_set_option(ctx, sem.SEM_OPT_SWEEP_SLABS, K)
        sem.sem_set_mesh_corners(ctx, mesh.ibool, mesh.ctrl, mesh.nglob)
        sem.sem_set_material(ctx, *mat)
        info = sem.sem_info(ctx)
        assert info["slabs"] == K
        assert K * 2 <= info["launches"] <= K * info["ncolors"]
        out.append(gpu_forces(ctx, u))
    assert rel_l2(out[1], out[0].astype(np.float64)) <= 1e-6
    m = oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, *mat, mesh.ngll)
    check_forces(out[1], m.forces(u.astype(np.float64)))
    with pytest.raises(sem.SemError):
        sem.sem_set_option(ctx, 99, 1)
