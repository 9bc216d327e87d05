"""Batched shots (several sources on one model, shot index innermost): the batched run of S
shots matches S plain single-shot runs, and one shot matches the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2606_12850_gb300 import build, inputs, sem  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_BATCH = 2e-5   # batched vs plain (the accuracy at which batched throughput is quoted)
TOL_WAVEFIELD = 2e-5
TOL_SEIS = 1e-4


@pytest.fixture(scope="module", autouse=True)
def library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return sem.lib()


def rel_l2(a, b):
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _batched_and_plain(ngll, n, nshots, nsteps):
    w, pos = inputs.batched_layered_cube(n=n, ngll=ngll, nshots=nshots, nsteps=nsteps)
    ref = sem.setup_workload(w)
    nodes = sem.sem_locate_nodes(ref.ctx, pos)
    force = np.tile([0.0, 0.0, 1.0e10], (nshots, 1))
    b = sem.setup_workload(w, rec_nodes=ref.rec_nodes)
    sem.sem_set_shots(b.ctx, nshots)
    sem.sem_set_shot_sources(b.ctx, np.arange(nshots), nodes, force, w.f0, w.t0)
    sem.sem_set_state(b.ctx)
    seis_b = sem.sem_run(b.ctx, nsteps)
    u_b, v_b, _ = sem.sem_get_state(b.ctx)
    plain = []
    for s in range(nshots):
        p = sem.setup_workload(w, src_nodes=nodes[s:s + 1], rec_nodes=ref.rec_nodes)
        seis = sem.sem_run(p.ctx, nsteps)
        u, v, _ = sem.sem_get_state(p.ctx)
        plain.append((seis, u, v))
    return w, nodes, seis_b, u_b, v_b, plain, ref


@pytest.mark.parametrize("ngll,n,nshots", [(5, 6, 5), (5, 5, 9), (3, 8, 3), (7, 4, 6)])
def test_batched_matches_plain(ngll, n, nshots):
    """S shots advanced together equal S separate single-shot runs (rel L2 <= 2e-5); shot
    counts that are not multiples of the shots-per-CTA exercise the tail."""
    _, _, seis_b, u_b, v_b, plain, _ = _batched_and_plain(ngll, n, nshots, 60)
    assert seis_b.shape[0] == nshots and u_b.shape == (nshots,) + plain[0][1].shape
    for s, (seis, u, v) in enumerate(plain):
        assert rel_l2(seis_b[s], seis) <= TOL_BATCH
        assert rel_l2(u_b[s], u) <= TOL_BATCH
        assert rel_l2(v_b[s], v) <= TOL_BATCH


def test_batched_shot_matches_oracle(oracle):
    w, nodes, seis_b, u_b, _, _, ref = _batched_and_plain(5, 5, 4, 80)
    model = oracle.build_model(w)
    dt = model.cfl_dt(w.courant)
    seis_ref, u_ref, _, _ = oracle.newmark_run(model, dt, 80, src_nodes=nodes[2:3],
                                               src_force=[[0.0, 0.0, 1.0e10]], f0=w.f0, t0=w.t0,
                                               rec_nodes=ref.rec_nodes)
    assert rel_l2(u_b[2], u_ref) <= TOL_WAVEFIELD
    assert rel_l2(seis_b[2], seis_ref) <= TOL_SEIS


def test_shot_sources_validation():
    w = inputs.homogeneous_cube(n=3, side=300.0, nsteps=10)
    s = sem.setup_workload(w)
    sem.sem_set_shots(s.ctx, 3)
    with pytest.raises(sem.SemError):
        sem.sem_set_shot_sources(s.ctx, [3], s.src_nodes, [[0, 0, 1.0]], w.f0, w.t0)
    assert sem.sem_info(s.ctx)["shots"] == 3


def test_batched_energy_is_sum_over_shots():
    w = inputs.homogeneous_cube(n=3, side=300.0, nsteps=10)
    s = sem.setup_workload(w)
    n = s.ctx.nglob
    fields = [inputs.random_field(n, 10 + k, scale=1e-3) for k in range(3)]
    sem.sem_set_shots(s.ctx, 3)
    sem.sem_set_state(s.ctx, np.stack(fields))
    kin, pot = sem.sem_energy(s.ctx)
    total = 0.0
    for f in fields:
        p = sem.setup_workload(w)
        sem.sem_set_state(p.ctx, f)
        total += sum(sem.sem_energy(p.ctx))
    assert abs(kin + pot - total) <= 1e-6 * total
