"""Energy of the float32 GPU run over 1000 source-free steps. The explicit Newmark scheme
(beta = 0, gamma = 1/2) conserves, at integer steps,
    E_n = 1/2 v^T M v + 1/2 u^T K u - dt^2/8 a^T M a
exactly in exact arithmetic (the staggered leapfrog energy rewritten with v^{n+1/2} =
v^n + dt/2 a^n and K u^n = -M a^n); the GPU's float32 rounding may move it by at most 1e-5
relative over 1000 steps."""
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


def test_discrete_energy_drift_fp32(oracle):
    mesh = inputs.structured_hex_mesh(4, 5, 800.0, jitter=0.15, seed=9)
    shape = mesh.ibool.shape
    rho = inputs.uniform(1, shape, 2000, 3000, stream=1).astype(np.float32)
    vp = inputs.uniform(1, shape, 3000, 5000, stream=2).astype(np.float32)
    vs = (vp / 1.8).astype(np.float32)
    m = oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, rho, vp, vs, 5)  # FP64 mass for the a^T M a term
    ctx = sem.sem_create(5, 0)
    sem.sem_set_mesh_corners(ctx, mesh.ibool, mesh.ctrl, mesh.nglob)
    sem.sem_set_material(ctx, rho, vp, vs)
    dt = sem.sem_suggest_dt(ctx, 0.4)
    sem.sem_set_dt(ctx, dt)
    u0 = (np.sin(m.node_xyz / 300.0 + np.array([0.0, 1.0, 2.0])) * 1e-3).astype(np.float32)
    sem.sem_set_state(ctx, u=u0)
    sem.sem_init_acceleration(ctx)

    def energy():
        kin, pot = sem.sem_energy(ctx)
        _, _, a = sem.sem_get_state(ctx, want=(False, False, True))
        return kin + pot - dt * dt / 8.0 * float(np.sum(m.mass[:, None] * a.astype(np.float64) ** 2))

    E = [energy()]
    for _ in range(4):
        sem.sem_step(ctx, 250)
        E.append(energy())
    E = np.array(E)
    drift = float(np.abs(E / E[0] - 1.0).max())
    assert drift <= 1e-5, (drift, E)
