"""Full-size parity: the three-layer jittered cube at the sizes and launch configuration the
benchmark times (256 GLL intervals per side: 128^3 elements at NGLL=3, 64^3 at 5, 43^3 at
7, 32^3 at 9), checked on sampled nodes that the FP64 oracle evaluates one by one (it
visits only the elements touching them), plus properties that hold at any size.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2606_12850_gb300 import build, inputs, sem  # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL_L2 = 2e-5
TOL_MAX = 1e-4


@pytest.fixture(scope="module", autouse=True)
def library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return sem.lib()


def sample_nodes(mesh, nsample, seed, extra=()):
    pick = (inputs.uniform(seed, nsample, 0, mesh.nglob, stream=5)).astype(np.int64)
    fixed = [0, mesh.nglob - 1, mesh.nglob // 2]
    return np.unique(np.concatenate([pick, fixed, np.asarray(extra, dtype=np.int64)]))


@pytest.mark.parametrize("ngll", [3, 5, 7, 9])
def test_layered_cube_full_size(oracle, ngll):
    w = inputs.layered_cube(ngll)
    mesh = w.mesh
    s = sem.setup_workload(w)
    info = sem.sem_info(s.ctx)
    assert info["nspec"] == mesh.nspec and info["nglob"] == mesh.nglob
    counts = sem.sem_color_counts(s.ctx)
    assert counts.sum() == mesh.nspec and len(counts) == 8

    nodes = sample_nodes(mesh, 48, ngll, extra=s.src_nodes)
    elems = oracle.elements_touching(mesh.ibool, nodes)
    sub = oracle.build_model(w, elems)
    # (1) one stiffness application on a random field
    u = inputs.random_field(mesh.nglob, 2000 + ngll, scale=1e-3)
    torch.cuda.synchronize()
    ud = torch.from_numpy(u).cuda()
    fd = torch.empty_like(ud)
    torch.cuda.synchronize()
    sem.sem_apply_stiffness(s.ctx, ud, fd)
    sem.sem_sync(s.ctx)
    f = fd.cpu().numpy()
    assert np.all(np.isfinite(f))
    f_ref = sub.forces(u.astype(np.float64))[nodes]
    err = np.linalg.norm(f[nodes] - f_ref) / np.linalg.norm(f_ref)
    assert err <= TOL_L2, err
    assert np.abs(f[nodes] - f_ref).max() <= TOL_MAX * np.abs(f_ref).max()
    # any size: K annihilates a rigid translation (exactly up to FP32 rounding of -K 1)
    ud.fill_(1.0)
    torch.cuda.synchronize()
    sem.sem_apply_stiffness(s.ctx, ud, fd)
    sem.sem_sync(s.ctx)
    stiffness_scale = np.abs(f_ref).max() / 1e-3  # |f| per unit displacement
    assert fd.abs().max().item() <= 1e-5 * stiffness_scale

    # (2) one full time step from a random state, with the source active
    u0 = inputs.random_field(mesh.nglob, 1, scale=1e-4)
    v0 = inputs.random_field(mesh.nglob, 2, scale=1e-3)
    a0 = inputs.random_field(mesh.nglob, 3, scale=1e-1)
    sem.sem_set_state(s.ctx, u0, v0, a0)
    sem.sem_step(s.ctx, 1)
    u1, v1, a1 = sem.sem_get_state(s.ctx)
    dt = s.dt
    u1_ref = u0.astype(np.float64) + dt * v0 + 0.5 * dt * dt * a0.astype(np.float64)
    assert np.abs(u1 - u1_ref).max() <= 1e-6 * np.abs(u1_ref).max()
    f1 = sub.forces(u1_ref)
    src = np.zeros_like(f1)
    src[s.src_nodes[0]] = w.source_force[0] * oracle.ricker(dt, w.f0, w.t0)
    a1_ref = (f1 + src)[nodes] / sub.mass[nodes, None]
    e_a = np.linalg.norm(a1[nodes] - a1_ref) / np.linalg.norm(a1_ref)
    assert e_a <= TOL_L2, e_a
    v1_ref = v0[nodes] + 0.5 * dt * (a0[nodes].astype(np.float64) + a1_ref)
    e_v = np.linalg.norm(v1[nodes] - v1_ref) / np.linalg.norm(v1_ref)
    assert e_v <= TOL_L2, e_v


def test_layered_cube_locate_and_dt(oracle):
    """Node location and the CFL step on the full NGLL=5 mesh agree with the oracle (the
    source sits at a jittered interior vertex; receivers snap to top-surface nodes)."""
    w = inputs.layered_cube(5)
    s = sem.setup_workload(w)
    m = oracle.build_model(w)
    src, rec = oracle.locate_workload(m, w)
    assert list(s.src_nodes) == list(src)
    assert list(s.rec_nodes) == list(rec)
    assert abs(s.dt / m.cfl_dt(w.courant) - 1.0) < 1e-12
