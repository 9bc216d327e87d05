"""GPU parity of meshes given by per-point positions (sem_set_mesh), of sources and receivers
given by position (sem_set_sources, sem_set_receivers), through the C ABI, against the FP64
oracle's isoparametric route. Tolerances as in test_gpu_parity.py (stiffness: relative L2
2e-6, every entry 1e-5 of the largest; wavefield 2e-5; seismograms 1e-4)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2606_12850_gb300 import build, inputs, sem  # noqa: E402

pytestmark = pytest.mark.gpu

AMP = (0.15, 0.10, 0.12)


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


def material(mesh, seed):
    shape = mesh.ibool.shape
    rho = inputs.uniform(seed, shape, 2000.0, 3000.0, stream=1).astype(np.float32)
    vp = inputs.uniform(seed, shape, 3000.0, 5000.0, stream=2).astype(np.float32)
    vs = (vp / inputs.uniform(seed, shape, 1.6, 2.0, stream=3)).astype(np.float32)
    return rho, vp, vs


def both_sides(oracle, mesh, mat):
    """Library context on library-built bent points, oracle model on oracle-built ones."""
    lib_xyz, _, _ = sem.sem_geometry(mesh.ctrl, mesh.ngll)
    ctx = sem.sem_create(mesh.ngll, 0)
    sem.sem_set_mesh(ctx, mesh.ibool, inputs.bent_map(lib_xyz, mesh.lengths, AMP), mesh.nglob)
    sem.sem_set_material(ctx, *mat)
    xyz_o, _, _ = oracle.element_geometry(mesh.ctrl, oracle.Basis(mesh.ngll))
    pts_o = inputs.bent_map(np.moveaxis(xyz_o, 1, 4).reshape(mesh.nspec, -1, 3), mesh.lengths, AMP)
    model = oracle.Model(mesh.ibool, None, mesh.nglob, *mat, mesh.ngll, points=pts_o)
    return ctx, model


def gpu_forces(ctx, u):
    torch.cuda.synchronize()
    ud = torch.from_numpy(np.ascontiguousarray(u, dtype=np.float32)).cuda()
    fd = torch.full_like(ud, float("nan"))
    torch.cuda.synchronize()
    sem.sem_apply_stiffness(ctx, ud, fd)
    sem.sem_sync(ctx)
    return fd.cpu().numpy()


@pytest.mark.parametrize("ngll", [3, 5, 7])
def test_bent_mesh_forces(oracle, ngll):
    mesh = inputs.structured_hex_mesh((4, 3, 3), ngll, (1000.0, 800.0, 700.0), jitter=0.1, seed=ngll)
    mat = material(mesh, 40 + ngll)
    ctx, model = both_sides(oracle, mesh, mat)
    u = inputs.random_field(mesh.nglob, 50 + ngll)
    f = gpu_forces(ctx, u)
    f_ref = model.forces(u.astype(np.float64))
    assert rel_l2(f, f_ref) <= 2e-6
    assert np.max(np.abs(f - f_ref)) <= 1e-5 * np.max(np.abs(f_ref))


def test_per_point_mesh_equals_corner_mesh():
    """Trilinear positions through sem_set_mesh give the corner form's forces bit for bit."""
    mesh = inputs.structured_hex_mesh((3, 3, 2), 5, 900.0, jitter=0.2, seed=4)
    mat = material(mesh, 5)
    a = sem.sem_create(5, 0)
    sem.sem_set_mesh_corners(a, mesh.ibool, mesh.ctrl, mesh.nglob)
    sem.sem_set_material(a, *mat)
    b = sem.sem_create(5, 0)
    xyz, _, _ = sem.sem_geometry(mesh.ctrl, 5)
    sem.sem_set_mesh(b, mesh.ibool, xyz, mesh.nglob)
    sem.sem_set_material(b, *mat)
    u = inputs.random_field(mesh.nglob, 6)
    assert np.array_equal(gpu_forces(a, u), gpu_forces(b, u))


def test_bent_mesh_run_with_sources_and_receivers_by_position(oracle):
    """100 steps on a bent mesh with a point force and receivers given by position: the
    snapped nodes equal the oracle's nearest nodes, the wavefield and the seismograms match."""
    mesh = inputs.structured_hex_mesh((5, 4, 4), 5, (1000.0, 800.0, 800.0), jitter=0.1, seed=8)
    mat = material(mesh, 9)
    ctx, model = both_sides(oracle, mesh, mat)
    dt = sem.sem_suggest_dt(ctx, 0.4)
    assert abs(dt - model.cfl_dt(0.4)) <= 1e-12 * dt
    sem.sem_set_dt(ctx, dt)
    src_xyz = inputs.bent_map(np.array([[500.0, 400.0, 400.0]]), mesh.lengths, AMP)
    rec_xyz = inputs.bent_map(np.array([[100.0 + 150.0 * r, 300.0, 800.0] for r in range(6)]), mesh.lengths, AMP)
    force = np.array([[0.0, 0.0, 1.0e10]])
    sem.sem_set_sources(ctx, src_xyz, force, 10.0, 0.12)
    rec_nodes = sem.sem_set_receivers(ctx, rec_xyz)
    assert np.array_equal(rec_nodes, model.nearest_nodes(rec_xyz))
    sem.sem_set_state(ctx)
    nsteps = 100
    seis = sem.sem_run(ctx, nsteps)
    u, _, _ = sem.sem_get_state(ctx, want=(True, False, False))
    seis_ref, u_ref, _, _ = oracle.newmark_run(model, dt, nsteps, src_nodes=model.nearest_nodes(src_xyz),
                                              src_force=force, f0=10.0, t0=0.12, rec_nodes=rec_nodes)
    assert rel_l2(u.reshape(-1, 3), u_ref) <= 2e-5
    assert rel_l2(seis.reshape(seis_ref.shape), seis_ref) <= 1e-4


def test_positions_rejected():
    mesh = inputs.structured_hex_mesh((2, 2, 2), 4, 100.0)
    xyz, _, _ = sem.sem_geometry(mesh.ctrl, 4)
    ctx = sem.sem_create(4, 0)
    bad = xyz.copy()
    bad[1, 3, 2] = np.nan
    with pytest.raises(sem.SemError):
        sem.sem_set_mesh(ctx, mesh.ibool, bad, mesh.nglob)
    folded = xyz.copy()
    folded[0] = folded[0][::-1]
    with pytest.raises(sem.SemError) as ei:
        sem.sem_set_mesh(ctx, mesh.ibool, folded, mesh.nglob)
    assert "Jacobian" in str(ei.value)
    sem.sem_set_mesh(ctx, mesh.ibool, xyz, mesh.nglob)
    with pytest.raises(sem.SemError):
        sem.sem_set_sources(ctx, np.array([[np.inf, 0.0, 0.0]]), np.array([[1.0, 0, 0]]), 10.0, 0.1)
