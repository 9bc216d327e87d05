"""The Newmark update run inside the force sweep (SEM_OPT_FUSED_NEWMARK 1, the default)
against separate Newmark passes (0).

Both perform the same float32 operations in the same order: the forces meeting at a node
summed in sweep order, the step's point sources added to the complete force, then the
corrector a = M^-1 f, v = v_half + dt/2 a and the predictor u + dt v + dt^2/2 a,
v + dt/2 a (Sec. I). So wavefields and seismograms are bitwise equal: through graph
replays, eager remainders, runs split across calls (which end with the corrector alone and
start with the predictor), several shots, and element orders whose last toucher is not the
first patch. Accuracy against the oracle is covered by the parity tests, which run the
default (fused) path."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2606_12850_gb300 import build, inputs, sem  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return sem.lib()


def run(w, fused, splits, seed=1, shots=None):
    """Steps of workload w from a seeded random state; splits = steps per sem_run call.
    shots = (node per shot, force) runs that many shots of one model instead."""
    s = sem.setup_workload(w, device=0)
    ctx = s.ctx
    sem.sem_set_option(ctx, sem.SEM_OPT_FUSED_NEWMARK, fused)
    nglob = w.mesh.nglob
    if shots is not None:
        nodes, force = shots
        sem.sem_set_shots(ctx, len(nodes))
        sem.sem_set_shot_sources(ctx, np.arange(len(nodes)), nodes, force, w.f0, w.t0)
        shape = (len(nodes), nglob, 3)
        state = [inputs.uniform(seed + k, shape, -sc, sc, stream=k).astype(np.float32)
                 for k, sc in enumerate((1e-4, 1e-3, 1e-1))]
    else:
        state = [inputs.random_field(nglob, seed + k, scale=sc) for k, sc in enumerate((1e-4, 1e-3, 1e-1))]
    sem.sem_set_state(ctx, *state)
    seis = np.concatenate([sem.sem_run(ctx, k) for k in splits], axis=-1)
    u, v, a = sem.sem_get_state(ctx)
    return seis, u, v, a


def assert_same(x, y):
    for p, q in zip(x, y):
        assert p.shape == q.shape
        assert np.array_equal(p, q), float(np.max(np.abs(p.astype(np.float64) - q)))


@pytest.mark.parametrize("ngll,n", [(3, 7), (5, 5), (7, 3)])
def test_fused_sweep_equals_separate_passes(ngll, n):
    """Layered jittered cube with the source active from step 1: 23 steps as two graph
    replays plus three eager steps, and the same steps split 7 + 16 across two calls."""
    w = dataclasses.replace(inputs.layered_cube(ngll, n=n, side=1200.0, nrec_side=3), t0=0.02)
    ref = run(w, 0, [23])
    assert np.abs(ref[0]).max() > 0
    assert_same(run(w, 1, [23]), ref)
    assert_same(run(w, 1, [7, 16]), ref)
    assert_same(run(w, 1, [1, 1, 21]), ref)


def test_fused_sweep_with_shots():
    """Four shots of one model, each with its own source node (one shared by two shots):
    fused and separate passes agree bitwise."""
    w = inputs.layered_cube(5, n=5, side=1200.0, nrec_side=2)
    probe = sem.setup_workload(w, device=0)
    nodes = sem.sem_locate_nodes(probe.ctx, np.array([[300.0, 400.0, 500.0], [900.0, 600.0, 700.0],
                                                      [300.0, 400.0, 500.0], [600.0, 600.0, 1100.0]]))
    force = np.array([[0.0, 0.0, 1e10], [1e10, 0.0, 0.0], [0.0, 5e9, 0.0], [0.0, 0.0, -1e10]])
    ref = run(w, 0, [13], shots=(nodes, force))
    assert_same(run(w, 1, [13], shots=(nodes, force)), ref)
    assert_same(run(w, 1, [4, 9], shots=(nodes, force)), ref)


def test_fused_sweep_scrambled_elements():
    """Elements and nodes numbered at random by the caller: the patches, their sweep order
    and each node's last toucher do not depend on the numbering, and fused and separate
    passes still agree bitwise with a source on a node shared by several patches."""
    mesh = inputs.structured_hex_mesh((6, 5, 4), 5, 1000.0, jitter=0.1, seed=21)
    rng = np.random.default_rng(8)
    eperm = rng.permutation(mesh.nspec)
    nperm = rng.permutation(mesh.nglob)
    ib = nperm[mesh.ibool[eperm]].astype(np.int32)
    ctrl = mesh.ctrl[eperm]
    shape = mesh.ibool.shape
    rho = inputs.uniform(3, shape, 2000.0, 3000.0, stream=1).astype(np.float32)[eperm]
    vp = inputs.uniform(3, shape, 3000.0, 5000.0, stream=2).astype(np.float32)[eperm]
    vs = (vp / 1.8).astype(np.float32)
    outs = []
    for fused in (0, 1):
        ctx = sem.sem_create(5, 0)
        sem.sem_set_mesh_corners(ctx, ib, ctrl, mesh.nglob)
        sem.sem_set_material(ctx, rho, vp, vs)
        sem.sem_set_option(ctx, sem.SEM_OPT_FUSED_NEWMARK, fused)
        sem.sem_set_dt(ctx, sem.sem_suggest_dt(ctx, 0.4))
        # a lattice vertex in the interior: met by 8 elements, so by several patches
        src = np.array([nperm[mesh.ibool[mesh.nspec // 2, 0]]], dtype=np.int32)
        sem.sem_set_source_nodes(ctx, src, np.array([[1e10, -2e10, 3e10]]), 10.0, 0.0)
        sem.sem_set_receiver_nodes(ctx, nperm[np.arange(0, mesh.nglob, 97)].astype(np.int32))
        sem.sem_set_state(ctx)
        seis = np.concatenate([sem.sem_run(ctx, k) for k in (11, 5)], axis=-1)
        outs.append((seis,) + tuple(sem.sem_get_state(ctx)))
    assert np.abs(outs[0][0]).max() > 0
    assert_same(outs[1], outs[0])


@pytest.mark.parametrize("fused", [0, 1])
def test_profile_steps_advance_like_step(fused):
    """sem_profile_steps (eager steps with events around each sweep) advances the state
    exactly as sem_step does, and reports positive times."""
    w = inputs.layered_cube(5, n=4, side=1200.0, nrec_side=2)
    outs = []
    for profile in (False, True):
        s = sem.setup_workload(w, device=0)
        sem.sem_set_option(s.ctx, sem.SEM_OPT_FUSED_NEWMARK, fused)
        sem.sem_set_state(s.ctx, *[inputs.random_field(w.mesh.nglob, 40 + k, scale=sc)
                                   for k, sc in enumerate((1e-4, 1e-3, 1e-1))])
        if profile:
            sweep_ms, rest_ms = sem.sem_profile_steps(s.ctx, 12)
            assert sweep_ms > 0 and rest_ms > 0
        else:
            sem.sem_step(s.ctx, 12)
        outs.append(sem.sem_get_state(s.ctx))
    assert_same(outs[1], outs[0])


@pytest.mark.parametrize("ngll,n", [(5, 5), (3, 6), (7, 3)])
def test_shot_pairs_match_one_cta_per_shot(ngll, n):
    """Five shots (two pairs and a lone shot): the pair kernel (SEM_OPT_SHOT_PAIRS 1) against
    one CTA per (patch, shot) (0), the same arithmetic up to the rounding order of a few sums."""
    w = inputs.layered_cube(ngll, n=n, side=1200.0, nrec_side=2)
    probe = sem.setup_workload(w, device=0)
    pos = np.array([[300.0, 400.0, 500.0], [900.0, 600.0, 700.0], [500.0, 500.0, 600.0],
                    [600.0, 600.0, 1100.0], [200.0, 900.0, 300.0]])
    nodes = sem.sem_locate_nodes(probe.ctx, pos)
    force = np.array([[0.0, 0.0, 1e10], [1e10, 0.0, 0.0], [0.0, 5e9, 0.0], [0.0, 0.0, -1e10], [3e9, 3e9, 3e9]])
    outs = []
    for pairs in (0, 1):
        s = sem.setup_workload(w, device=0)
        sem.sem_set_shots(s.ctx, len(nodes))
        sem.sem_set_option(s.ctx, sem.SEM_OPT_SHOT_PAIRS, pairs)
        sem.sem_set_shot_sources(s.ctx, np.arange(len(nodes)), nodes, force, w.f0, w.t0)
        sem.sem_set_state(s.ctx)
        seis = sem.sem_run(s.ctx, 40)
        outs.append((seis,) + tuple(sem.sem_get_state(s.ctx)))
    for x, y in zip(outs[1], outs[0]):
        y = y.astype(np.float64)
        assert np.linalg.norm(x - y) <= 1e-6 * np.linalg.norm(y)


@pytest.mark.parametrize("ngll", [2, 4, 6, 8, 9, 10])
def test_fused_sweep_every_order(ngll):
    """The remaining orders (the parametrized test above covers 3, 5 and 7): a jittered
    layered cube of a few bricks, 12 steps split 5 + 7, fused against separate passes."""
    w = dataclasses.replace(inputs.layered_cube(ngll, n=4, side=800.0, nrec_side=2), t0=0.02)
    ref = run(w, 0, [12])
    assert np.abs(ref[0]).max() > 0
    assert_same(run(w, 1, [5, 7]), ref)
