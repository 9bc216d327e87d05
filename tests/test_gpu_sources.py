"""GPU parity of moment-tensor sources (batched shots) with the FP64 oracle: each shot's
wavefield after 100 steps within relative L2 2e-5 and its seismograms within 1e-4 (the
solver's accuracy targets), on a jittered layered 4^3 mesh at NGLL 5."""
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


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_moment_sources_match_oracle(oracle):
    w = inputs.layered_cube(5, n=4, side=1000.0, nsteps=100, nrec_side=3)
    w.f0, w.t0 = 15.0, 0.08
    m = oracle.Model(w.mesh.ibool, w.mesh.ctrl, w.mesh.nglob, w.rho, w.vp, w.vs, 5)
    dt = m.cfl_dt(0.4)
    pos = inputs.shot_positions(3, 1000.0, seed=8)
    nodes = m.nearest_nodes(pos)
    moments = inputs.uniform(8, (3, 6), -1.0, 1.0, stream=12) * 1e13
    rec = m.nearest_nodes(w.receiver_xyz, surface_z=1000.0)
    s = sem.setup_workload(w, dt=dt, src_nodes=nodes[:1], rec_nodes=rec)
    sem.sem_set_shots(s.ctx, 3)
    sem.sem_set_shot_moment_sources(s.ctx, np.arange(3), nodes, moments, w.f0, w.t0)
    sem.sem_set_receiver_nodes(s.ctx, rec)
    sem.sem_set_state(s.ctx)
    seis = sem.sem_run(s.ctx, 100)
    u, _, _ = sem.sem_get_state(s.ctx, want=(True, False, False))
    for sh in range(3):
        fn, ff = oracle.moment_tensor_forces(m, int(nodes[sh]), moments[sh])
        ref_seis, ref_u, _, _ = oracle.newmark_run(m, dt, 100, src_nodes=fn, src_force=ff, f0=w.f0, t0=w.t0,
                                                   rec_nodes=rec)
        assert rel_l2(u[sh], ref_u) <= 2e-5
        assert rel_l2(seis[sh], ref_seis) <= 1e-4
