"""The 8^3 copy of the sensitivity workload, shared by the oracle's finite-difference pin and
the GPU adjoint parity test: the three-layer jittered cube (side 4 km, NGLL 5) with the 5 %
Gaussian velocity anomaly as the true model and the unperturbed layers as the model whose
gradient is taken, rho/kappa/mu rounded to float32 so that both sides see the same numbers.
The receivers are the eight corners of a 600 m cube around the source (the surface is
beyond the reach of a 40-step run at this element size)."""
import numpy as np

from paper_2606_12850_gb300 import inputs


def anomaly_copy(oracle, nsteps: int = 40):
    w = inputs.perturbed_layered_cube(n=8, ngll=5, nsteps=nsteps)
    mesh = w.mesh
    rho_b, vp_b, vs_b = w.extra["background"]
    true = oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, w.rho, w.vp, w.vs, mesh.ngll)
    bg = oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, rho_b, vp_b, vs_b, mesh.ngll)
    f32 = lambda x: x.astype(np.float32).astype(np.float64)  # noqa: E731
    bg = oracle.set_moduli(bg, rho=f32(bg.rho), kappa=f32(bg.kappa), mu=f32(bg.mu))
    dt = true.cfl_dt(0.4)  # the faster model sets the stable step for both
    src = bg.nearest_nodes(w.source_xyz)
    corners = np.array([[a, b, c] for c in (-1, 1) for b in (-1, 1) for a in (-1, 1)], dtype=np.float64)
    rec = bg.nearest_nodes(w.source_xyz[0] + 300.0 * corners)
    kw = dict(src_nodes=src, src_force=w.source_force, f0=w.f0, t0=w.t0, rec_nodes=rec)
    _, d_obs = oracle.forward_history(true, dt, nsteps, **kw)
    u_hist, seis = oracle.forward_history(bg, dt, nsteps, **kw)
    G = dt * (seis - d_obs)
    return dict(workload=w, mesh=mesh, m=bg, dt=dt, kw=kw, nsteps=nsteps, u_hist=u_hist, seis=seis,
                d_obs=d_obs, G=G)


def misfit(oracle, model, case) -> float:
    """L = dt/2 * sum over receivers, components and steps of (s - d_obs)^2."""
    _, seis = oracle.forward_history(model, case["dt"], case["nsteps"], **case["kw"])
    return 0.5 * case["dt"] * float(np.sum((seis - case["d_obs"]) ** 2))
