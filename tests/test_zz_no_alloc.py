"""The allocation-free energy entry point (sem_energy_noalloc) against sem_energy.

Some callers cannot call cudaMalloc (their device memory belongs to another runtime's
pool, or they run where allocation is not allowed); sem_energy_noalloc serves them with a
fixed scratch array inside the library. This file is collected last so that, if it fails,
a run stopping at the first failure has already run every other test; it also passes on
its own in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2606_12850_gb300 import build, inputs, sem  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_ENERGY = 1e-5  # the energy tolerance of the GPU parity tests


@pytest.fixture(scope="module", autouse=True)
def library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return sem.lib()


def _context(n, seed):
    mesh = inputs.structured_hex_mesh(n, 5, 100.0 * n, jitter=0.15, seed=seed)
    shape = mesh.ibool.shape
    rho = inputs.uniform(seed, shape, 2000.0, 3000.0, stream=1).astype(np.float32)
    vp = inputs.uniform(seed, shape, 3000.0, 5000.0, stream=2).astype(np.float32)
    vs = (vp / 1.8).astype(np.float32)
    ctx = sem.sem_create(5, 0)
    sem.sem_set_mesh_corners(ctx, mesh.ibool, mesh.ctrl, mesh.nglob)
    sem.sem_set_material(ctx, rho, vp, vs)
    sem.sem_set_dt(ctx, sem.sem_suggest_dt(ctx, 0.4))
    u0 = inputs.random_field(mesh.nglob, seed, scale=1e-3)
    v0 = inputs.random_field(mesh.nglob, seed + 1, scale=1e-2)
    sem.sem_set_state(ctx, u0, v0)
    sem.sem_step(ctx, 7)
    return ctx


def _state_on_device(ctx):
    n3 = 3 * ctx.nglob
    u = torch.empty(n3, device="cuda")
    v = torch.empty(n3, device="cuda")
    f = torch.empty(n3, device="cuda")
    torch.cuda.synchronize()
    sem.sem_get_state_dev(ctx, u, v, None)
    sem.sem_apply_stiffness(ctx, u, f)
    sem.sem_sync(ctx)
    return u, v, f


def _close(a, b):
    scale = abs(b[0]) + abs(b[1])
    return abs(a[0] - b[0]) <= TOL_ENERGY * scale and abs(a[1] - b[1]) <= TOL_ENERGY * scale


def test_noalloc_energy_matches_sem_energy_twice():
    """Two calls in a row on one context, then a smaller mesh (the shared scratch array
    holds the previous call's sums): each result matches sem_energy."""
    big = _context(6, 3)
    u, v, f = _state_on_device(big)
    ref = sem.sem_energy(big)
    first = sem.sem_energy_noalloc(big, u, v, f)
    second = sem.sem_energy_noalloc(big, u, v, f)
    assert ref[0] > 0 and ref[1] > 0
    assert _close(first, ref) and _close(second, ref)
    assert first == second
    small = _context(2, 5)
    us, vs_, fs = _state_on_device(small)
    ref_s = sem.sem_energy(small)
    assert _close(sem.sem_energy_noalloc(small, us, vs_, fs), ref_s)
    assert _close(sem.sem_energy_noalloc(big, u, v, f), ref)


def test_noalloc_energy_rejects_oversize():
    ctx = _context(2, 7)
    u, v, f = _state_on_device(ctx)
    with pytest.raises(sem.SemError) as ei:
        sem.sem_energy_noalloc(ctx, u, v, f, nglob=67108864 + 1)
    assert ei.value.code == -1 and "maximum" in str(ei.value)
