"""Contexts stepped together (sem_group_step) give every context the same state as
stepping it alone, bit for bit, across graph rebuilds; the autotuner times both
contraction forms and either form meets the parity bar against the FP64 oracle."""
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


def workloads():
    return [inputs.homogeneous_cube(3, 4, nsteps=40), inputs.homogeneous_cube(4, 5, nsteps=40),
            inputs.layered_cube(6, n=2, side=500.0, nsteps=40, nrec_side=2)]


def fresh(w):
    return sem.setup_workload(w)


@pytest.mark.parametrize("mode", [1, 0])
def test_group_equals_separate_runs(mode):
    """Persistent sweeps (one launch per order for all contexts; mode 1) and graph branches
    (mode 0) both give every context the state of stepping it alone, bit for bit."""
    ws = workloads()
    alone = []
    for w in ws:
        s = fresh(w)
        sem.sem_step(s.ctx, 27)
        alone.append(sem.sem_get_state(s.ctx, want=(True, False, False))[0])
    setups = [fresh(w) for w in ws]
    group = sem.Group([s.ctx for s in setups])
    group.set_option(sem.SEM_GROUP_MODE, mode)
    info = group.info()
    assert info["persistent"] == (mode == 1)
    if mode == 1:
        assert info["sweep_launches"] == 3  # NGLL 4, 5 and 6
    group.step(27)
    group.sync()
    for s, ref in zip(setups, alone):
        u = sem.sem_get_state(s.ctx, want=(True, False, False))[0]
        assert np.array_equal(u, ref)
        assert sem.sem_info(s.ctx)["steps"] == 27
    # change one context (dt), the group rebuilds its graphs and still matches
    sem.sem_set_dt(setups[1].ctx, 0.9 * setups[1].dt)
    ref = fresh(ws[1])
    sem.sem_step(ref.ctx, 27)
    sem.sem_set_dt(ref.ctx, 0.9 * ref.dt)
    sem.sem_step(ref.ctx, 13)
    group.step(13)
    group.sync()
    assert np.array_equal(sem.sem_get_state(setups[1].ctx, want=(True, False, False))[0],
                          sem.sem_get_state(ref.ctx, want=(True, False, False))[0])


def test_autotune_forms_meet_parity(oracle):
    w = inputs.homogeneous_cube(4, 5, nsteps=60)
    m = oracle.Model(w.mesh.ibool, w.mesh.ctrl, w.mesh.nglob, w.rho, w.vp, w.vs, 5)
    s = fresh(w)
    ms, choice = sem.sem_autotune(s.ctx, reps=3)
    assert choice in (1, 2) and np.all(ms > 0)
    assert ms[choice - 1] == ms.min()
    u0 = inputs.random_field(w.mesh.nglob, 5)
    ref = m.forces(u0.astype(np.float64))
    ud = torch.from_numpy(u0).cuda()
    for form in (1, 2):
        sem.sem_set_option(s.ctx, sem.SEM_OPT_CONTRACTION, form)
        f = torch.empty_like(ud)
        torch.cuda.synchronize()
        sem.sem_apply_stiffness(s.ctx, ud, f)
        sem.sem_sync(s.ctx)
        f = f.cpu().numpy()
        assert np.linalg.norm(f - ref) / np.linalg.norm(ref) <= 2e-6, form


def test_group_of_one_order_is_one_sweep_launch():
    """Several models of one order (different sizes, one with a scrambled element order and
    a point source) in one persistent sweep launch per step, equal to separate runs."""
    ws = [inputs.layered_cube(5, n=n, side=600.0, nsteps=30, nrec_side=2) for n in (2, 3, 5)]
    alone = []
    for w in ws:
        s = fresh(w)
        sem.sem_step(s.ctx, 23)
        alone.append(sem.sem_get_state(s.ctx))
    setups = [fresh(w) for w in ws]
    group = sem.Group([s.ctx for s in setups])
    assert group.info() == {"persistent": False, "sweep_launches": 0}  # graph branches by default
    group.set_option(sem.SEM_GROUP_MODE, 1)
    assert group.info() == {"persistent": True, "sweep_launches": 1}
    group.step(23)
    group.sync()
    for s, ref in zip(setups, alone):
        for x, y in zip(sem.sem_get_state(s.ctx), ref):
            assert np.array_equal(x, y)


def test_group_sweep_wait_gives_up_and_recovers():
    """Failure detection without a fault: a persistent group step whose waits target counts
    that never arrive gives up within its bound, sem_group_sync reports SEM_ETIMEOUT, and the
    group's next steps run."""
    setups = [fresh(w) for w in workloads()[:2]]
    group = sem.Group([s.ctx for s in setups])
    group.set_option(sem.SEM_GROUP_MODE, 1)
    group.set_option(sem.SEM_GROUP_STALL_TEST, 1)
    group.step(3)
    with pytest.raises(sem.SemError) as ei:
        group.sync()
    assert ei.value.code == -5 and "gave up" in str(ei.value)
    group.step(4)
    group.sync()
