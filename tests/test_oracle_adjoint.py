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
