"""The object form of the binding (``sem.Solver``) issues the same calls as the function
form: the homogeneous cube run through both gives bitwise equal seismograms and state, and
host and device wavefields are accepted alike."""
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


def test_solver_equals_function_calls():
    w = inputs.homogeneous_cube(4, 5, nsteps=60)
    s = sem.Solver.from_workload(w)
    seis = s.run(60)
    u, v, a = s.state()
    ref = sem.setup_workload(w)
    assert s.dt == ref.dt
    seis_ref = sem.sem_run(ref.ctx, 60)
    u_ref, v_ref, a_ref = sem.sem_get_state(ref.ctx)
    assert np.array_equal(seis, seis_ref)
    assert np.array_equal(u, u_ref) and np.array_equal(v, v_ref) and np.array_equal(a, a_ref)
    # device wavefields: restart both from the same state and compare again
    ud, vd, ad = (torch.from_numpy(x).cuda() for x in (u, v, a))
    s.set_state(ud, vd, ad)
    s.sync()  # the device arrays are borrowed until the context's stream has read them
    sem.sem_set_state(ref.ctx, u, v, a)
    out = torch.empty((ref.rec_nodes.size, 3, 20), device="cuda")
    s.run(20, out)
    s.sync()
    assert np.array_equal(out.cpu().numpy(), sem.sem_run(ref.ctx, 20))
