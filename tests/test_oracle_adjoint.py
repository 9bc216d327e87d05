"""Pins of the oracle's discrete adjoint: its gradients equal central finite differences of
the loss (FP64, relative 1e-6), and the history-keeping forward run equals newmark_run."""
import numpy as np
import pytest

from paper_2606_12850_gb300 import inputs


@pytest.fixture(scope="module")
def problem(oracle):
    mesh = inputs.structured_hex_mesh(3, 4, 600.0, jitter=0.15, seed=4)
    shape = mesh.ibool.shape
    rho = inputs.uniform(2, shape, 2200, 2800, stream=1)
    vp = inputs.uniform(2, shape, 3000, 4000, stream=2)
    vs = vp / 1.8
    m = oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, rho, vp, vs, 4)
    dt = m.cfl_dt(0.4)
    X = m.node_xyz
    src = m.nearest_nodes([[300.0, 300.0, 300.0]])
    rec = m.nearest_nodes([[100.0, 500.0, 600.0], [500.0, 100.0, 600.0], [300.0, 300.0, 0.0]])
    nsteps = 60
    kw = dict(src_nodes=src, src_force=[[1e6, -2e6, 3e6]], f0=20.0, t0=0.04, rec_nodes=rec)
    u_hist, seis = oracle.forward_history(m, dt, nsteps, **kw)
    d_obs = 0.9 * seis + 1e-9 * np.sin(np.arange(seis.size)).reshape(seis.shape)
    return dict(m=m, dt=dt, kw=kw, nsteps=nsteps, u_hist=u_hist, seis=seis, d_obs=d_obs)


def _loss(oracle, model, p):
    _, seis = oracle.forward_history(model, p["dt"], p["nsteps"], **p["kw"])
    return 0.5 * p["dt"] * np.sum((seis - p["d_obs"]) ** 2)


def test_history_matches_newmark(oracle, problem):
    p = problem
    seis, u, _, _ = oracle.newmark_run(p["m"], p["dt"], p["nsteps"], **p["kw"])
    np.testing.assert_allclose(p["seis"], seis, rtol=0, atol=1e-15 * np.abs(seis).max())
    np.testing.assert_allclose(p["u_hist"][-1], u, rtol=0, atol=1e-15 * np.abs(u).max())
    assert not np.any(p["u_hist"][1])  # u^1 = 0 from rest (the source acts from t_1)


@pytest.mark.parametrize("which", ["kappa", "mu", "rho"])
def test_adjoint_gradient_matches_finite_differences(oracle, problem, which):
    p = problem
    m = p["m"]
    G = p["dt"] * (p["seis"] - p["d_obs"])
    g_rho, g_kappa, g_mu = oracle.adjoint_gradient(m, p["dt"], p["u_hist"], p["kw"]["rec_nodes"], G)
    grad = {"rho": g_rho, "kappa": g_kappa, "mu": g_mu}[which]
    base = {"rho": m.rho, "kappa": m.kappa, "mu": m.mu}[which]
    idx = np.unravel_index(np.argsort(np.abs(grad).ravel())[-3:], grad.shape)
    for q in zip(*idx):
        h = 1e-4 * base[q]
        vals = []
        for s in (+1, -1):
            pert = base.copy()
            pert[q] += s * h
            vals.append(_loss(oracle, oracle.set_moduli(m, **{which: pert}), p))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - grad[q]) <= 1e-6 * abs(fd), (which, q, fd, grad[q])


def test_adjoint_directional_derivative_on_anomaly_copy(oracle):
    """On the 8^3 copy of the sensitivity workload (layered, jittered, 5 % anomaly as the true
    model), the adjoint gradient's directional derivative along a seeded per-element
    direction in (rho, kappa, mu) at once equals the central finite difference of the misfit
    to relative 1e-6 (step 1e-4 of each parameter, FP64)."""
    from tests import adjoint_cases
    case = adjoint_cases.anomaly_copy(oracle)
    m = case["m"]
    g_rho, g_kappa, g_mu = oracle.adjoint_gradient(m, case["dt"], case["u_hist"], case["kw"]["rec_nodes"], case["G"])
    shape = m.rho.shape
    r = [np.broadcast_to(inputs.uniform(9, (m.nspec, 1, 1, 1), -1, 1, stream=s), shape) for s in (1, 2, 3)]
    d_rho, d_kappa, d_mu = m.rho * r[0], m.kappa * r[1], m.mu * r[2]
    predicted = np.sum(g_rho * d_rho) + np.sum(g_kappa * d_kappa) + np.sum(g_mu * d_mu)
    h = 1e-4
    L = [adjoint_cases.misfit(oracle, oracle.set_moduli(m, rho=m.rho + s * h * d_rho, kappa=m.kappa + s * h * d_kappa,
                                                        mu=m.mu + s * h * d_mu), case) for s in (+1, -1)]
    fd = (L[0] - L[1]) / (2 * h)
    assert abs(predicted) > 0
    assert abs(fd - predicted) <= 1e-6 * abs(fd), (fd, predicted)


ADJOINT_MUTATIONS = [
    ("g_mu -= dt * dt * wJ * 2.0 * (ee - tr_l * tr_u / 3.0)", "g_mu -= dt * dt * wJ * 2.0 * ee"),
    ("u_e = gather(u_hist[k], model.ibool, n)", "u_e = gather(u_hist[k + 1], model.ibool, n)"),
    ("np.add.at(inj, rec_nodes, G[:, :, m - 1])", "np.add.at(inj, rec_nodes, G[:, :, m - 2])"),
    ("(dt * dt * model.forces(lam) + inj)", "(dt * dt * model.forces(lam) - inj)"),
    ("g_rho -= wJ * np.einsum", "g_rho += wJ * np.einsum"),
    ("lam_prev = 2.0 * lam - lam_next", "lam_prev = 2.0 * lam + lam_next"),
]


@pytest.fixture(scope="module")
def fd_points(oracle, problem):
    """Central differences of the loss at the three largest-gradient points of each field."""
    p = problem
    m = p["m"]
    G = p["dt"] * (p["seis"] - p["d_obs"])
    grads = dict(zip(("rho", "kappa", "mu"), oracle.adjoint_gradient(m, p["dt"], p["u_hist"], p["kw"]["rec_nodes"], G)))
    out = []
    for which, grad in grads.items():
        base = getattr(m, which)
        idx = np.unravel_index(np.argsort(np.abs(grad).ravel())[-3:], grad.shape)
        for q in zip(*idx):
            h = 1e-4 * base[q]
            vals = []
            for s in (+1, -1):
                pert = base.copy()
                pert[q] += s * h
                vals.append(_loss(oracle, oracle.set_moduli(m, **{which: pert}), p))
            out.append((which, q, (vals[0] - vals[1]) / (2 * h)))
    return G, out


@pytest.mark.parametrize("old,new", ADJOINT_MUTATIONS)
def test_planted_adjoint_mistake_is_caught(oracle, problem, fd_points, old, new):
    """A slip planted in a copy of the oracle's adjoint (a dropped deviatoric shift, a time
    index off by one, a sign flip of the injection, of the mass term or of the leapfrog
    recursion) breaks the finite-difference pin at one of the checked points at least."""
    import inspect
    src = inspect.getsource(oracle.adjoint_gradient)
    assert old in src, old
    ns = dict(oracle.__dict__)
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    p = problem
    G, points = fd_points
    grads = dict(zip(("rho", "kappa", "mu"), ns["adjoint_gradient"](p["m"], p["dt"], p["u_hist"], p["kw"]["rec_nodes"], G)))
    assert any(abs(fd - grads[which][q]) > 1e-6 * abs(fd) for which, q, fd in points)
