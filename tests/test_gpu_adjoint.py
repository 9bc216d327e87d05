"""GPU parity of the discrete adjoint and the material gradients with the FP64 oracle.

The problem is the one the oracle's finite-difference pins use (jittered 3^3 mesh, NGLL 4,
random per-point rho/kappa/mu, one point force, three receivers, 60 steps), with the
material rounded to float32 on both sides. The same G^m = dL/ds^m (float64 on the oracle
side, float32 on the device) drives both adjoints.

Tolerances (relative L2 over all local points):
* seismograms: 1e-4, the solver's stated seismogram accuracy;
* g_kappa, g_mu: 1e-4. Each term is a product of an adjoint strain and a forward strain in
  float32; relative errors of a product add, the forward field and the adjoint field (run
  by the same kernels) each carry up to the solver's stated 2e-5, and the sum over time
  and points cancels terms of opposite sign, which we allow for with a factor of 2.5;
* g_rho: the mass term reads the second difference u^{n+1} - 2u^n + u^{n-1} of float32
  snapshots, which cancels most of their digits. The tolerance is 1e-4 plus twice the
  change that rounding the oracle's own snapshots to float32 causes in its g_rho.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2606_12850_gb300 import build, inputs, sem  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_SEIS = 1e-4
TOL_MODULI = 1e-4


@pytest.fixture(scope="module", autouse=True)
def library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return sem.lib()


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def problem(oracle):
    mesh = inputs.structured_hex_mesh(3, 4, 600.0, jitter=0.15, seed=4)
    shape = mesh.ibool.shape
    rho = inputs.uniform(2, shape, 2200, 2800, stream=1)
    vp = inputs.uniform(2, shape, 3000, 4000, stream=2)
    vs = vp / 1.8
    m = oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, rho, vp, vs, 4)
    f32 = lambda x: x.astype(np.float32).astype(np.float64)  # noqa: E731
    m = oracle.set_moduli(m, rho=f32(m.rho), kappa=f32(m.kappa), mu=f32(m.mu))
    dt = m.cfl_dt(0.4)
    src = m.nearest_nodes([[300.0, 300.0, 300.0]])
    rec = m.nearest_nodes([[100.0, 500.0, 600.0], [500.0, 100.0, 600.0], [300.0, 300.0, 0.0]])
    nsteps = 60
    kw = dict(src_nodes=src, src_force=[[1e6, -2e6, 3e6]], f0=20.0, t0=0.04, rec_nodes=rec)
    u_hist, seis = oracle.forward_history(m, dt, nsteps, **kw)
    d_obs = 0.9 * seis + 1e-9 * np.sin(np.arange(seis.size)).reshape(seis.shape)
    G = dt * (seis - d_obs)
    grads = oracle.adjoint_gradient(m, dt, u_hist, rec, G)
    return dict(mesh=mesh, m=m, dt=dt, kw=kw, nsteps=nsteps, u_hist=u_hist, seis=seis, d_obs=d_obs, G=G,
                grads=grads)


def make_sim(p, every, keep_all=False):
    from paper_2606_12850_gb300 import adjoint
    mesh = p["mesh"]
    ctx = sem.sem_create(mesh.ngll, 0)
    sem.sem_set_mesh_corners(ctx, mesh.ibool, mesh.ctrl, mesh.nglob)
    kw = p["kw"]
    sem.sem_set_source_nodes(ctx, kw["src_nodes"], kw["src_force"], kw["f0"], kw["t0"])
    sem.sem_set_receiver_nodes(ctx, kw["rec_nodes"])
    return ctx, adjoint.Simulation(ctx, p["dt"], p["nsteps"], checkpoint_every=every, keep_all=keep_all)


def material(p):
    m = p["m"]
    n3 = m.ngll ** 3
    return [torch.from_numpy(x.reshape(-1, n3).astype(np.float32)).cuda() for x in (m.rho, m.kappa, m.mu)]


def rho_tolerance(oracle, p):
    """1e-4 plus twice the change of g_rho that float32 rounding of the displacement
    snapshots causes by itself, measured with the oracle."""
    m = p["m"]
    u32 = p["u_hist"].astype(np.float32).astype(np.float64)
    g32 = oracle.adjoint_gradient(m, p["dt"], u32, p["kw"]["rec_nodes"], p["G"])[0]
    g64 = p["grads"][0] if "grads" in p else oracle.adjoint_gradient(m, p["dt"], p["u_hist"], p["kw"]["rec_nodes"],
                                                                     p["G"])[0]
    return TOL_MODULI + 2 * rel_l2(g32, g64)


def test_adjoint_matches_oracle(oracle, problem):
    p = problem
    ctx, sim = make_sim(p, every=50)
    rho, kappa, mu = material(p)
    seis = sim.forward(rho, kappa, mu).cpu().numpy()
    assert rel_l2(seis, p["seis"]) <= TOL_SEIS
    G = torch.from_numpy(p["G"].astype(np.float32)).cuda()
    g_rho, g_kappa, g_mu = sim.gradient(G)
    r_rho, r_kappa, r_mu = (x.reshape(g_rho.shape) for x in p["grads"])
    e_kappa, e_mu, e_rho = rel_l2(g_kappa, r_kappa), rel_l2(g_mu, r_mu), rel_l2(g_rho, r_rho)
    tol_rho = rho_tolerance(oracle, p)
    print(f"adjoint rel L2: kappa {e_kappa:.2e} mu {e_mu:.2e} rho {e_rho:.2e} (rho tol {tol_rho:.2e})")
    assert e_kappa <= TOL_MODULI
    assert e_mu <= TOL_MODULI
    assert e_rho <= tol_rho


def test_checkpoint_interval_does_not_change_gradient(problem):
    """Checkpoints every 7 steps (ragged last segment) against one segment of 60 steps."""
    p = problem
    G = torch.from_numpy(p["G"].astype(np.float32)).cuda()
    out = []
    for every in (7, 60):
        ctx, sim = make_sim(p, every)
        sim.forward(*material(p))
        out.append(sim.gradient(G))
    for a, b in zip(*out):
        assert rel_l2(a, b) <= 1e-5


@pytest.mark.parametrize("fused", [0, 1])
def test_kept_snapshots_match_checkpoints(oracle, problem, fused):
    """Every displacement kept from the forward run (sem_run_record_snapshots, one adjoint
    segment, no recomputation) against checkpoints every 7 steps: the same seismograms bit
    for bit, gradients within 1e-5 (the float32 partial sums are flushed on another
    schedule), and the oracle bar; with the fused sweep and with separate Newmark passes."""
    p = problem
    G = torch.from_numpy(p["G"].astype(np.float32)).cuda()
    seis, grads = [], []
    for keep in (False, True):
        ctx, sim = make_sim(p, 7, keep_all=keep)
        sem.sem_set_option(ctx, sem.SEM_OPT_FUSED_NEWMARK, fused)
        seis.append(sim.forward(*material(p)).cpu().numpy())
        assert (sim.snapshots is not None) == keep
        grads.append(sim.gradient(G))
    assert np.array_equal(seis[0], seis[1])
    for a, b in zip(*grads):
        assert rel_l2(b, a) <= 1e-5
    r_rho, r_kappa, r_mu = (x.reshape(grads[1][0].shape) for x in p["grads"])
    assert rel_l2(grads[1][1], r_kappa) <= TOL_MODULI and rel_l2(grads[1][2], r_mu) <= TOL_MODULI
    assert rel_l2(grads[1][0], r_rho) <= rho_tolerance(oracle, p)


def test_fused_adjoint_sweep_equals_separate_passes(problem):
    """The adjoint step with the residual injection and the leapfrog at each node's last
    touch in the sweep of lam (SEM_OPT_FUSED_NEWMARK 1) against the sweep followed by the
    injection and leapfrog passes (0): the same float operations, bitwise equal gradients."""
    p = problem
    G = torch.from_numpy(p["G"].astype(np.float32)).cuda()
    out = []
    for fused in (0, 1):
        ctx, sim = make_sim(p, 7, keep_all=True)
        sem.sem_set_option(ctx, sem.SEM_OPT_FUSED_NEWMARK, fused)
        sim.forward(*material(p))
        out.append(sim.gradient(G))
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_segment_equals_single_steps(problem):
    """sem_adjoint_segment (the mass term formed per node by the leapfrog pass) against
    sem_adjoint_step + sem_adjoint_accumulate one step at a time (formed at every local
    point): bitwise equal gradients."""
    p = problem
    ctx, sim = make_sim(p, 7, keep_all=True)
    sim.forward(*material(p))
    U = sim.snapshots
    N = p["nsteps"]
    Gt = torch.from_numpy(p["G"].astype(np.float32)).cuda().permute(2, 0, 1).contiguous()
    torch.cuda.synchronize()
    sem.sem_adjoint_begin(ctx)
    sem.sem_adjoint_segment(ctx, N - 1, Gt[1:N], U)
    seg = sem.sem_adjoint_gradients(ctx)
    sem.sem_adjoint_begin(ctx)
    for j in range(N - 1, 0, -1):
        sem.sem_adjoint_step(ctx, Gt[j])
        sem.sem_adjoint_accumulate(ctx, U[j - 1], U[j], U[j + 1])
    one = sem.sem_adjoint_gradients(ctx)
    for a, b in zip(seg, one):
        assert np.array_equal(a, b)


def test_restart_from_saved_state(problem):
    """A run restarted at step 30 from the saved state (sem_set_step) continues the source
    time function: its last 30 seismogram samples equal those of the straight run."""
    p = problem
    ctx, sim = make_sim(p, 50)
    mat = material(p)
    sim.set_material(*mat)
    sem.sem_set_state(ctx)
    straight = sem.sem_run(ctx, 60)
    sem.sem_set_state(ctx)
    sem.sem_run(ctx, 30)
    u, v, a = sem.sem_get_state(ctx)
    sem.sem_set_state(ctx, u, v, a)
    sem.sem_set_step(ctx, 30)
    rest = sem.sem_run(ctx, 30)
    assert rel_l2(rest, straight[:, :, 30:]) <= 1e-5
    # without sem_set_step the source would restart at t_1
    sem.sem_set_state(ctx, u, v, a)
    wrong = sem.sem_run(ctx, 30)
    assert rel_l2(wrong, straight[:, :, 30:]) > 1e-3


def test_autograd_function(problem):
    """loss.backward() through Seismograms gives the gradients of Simulation.gradient for
    G = dL/ds of the same loss."""
    from paper_2606_12850_gb300 import adjoint
    p = problem
    ctx, sim = make_sim(p, 20)
    rho, kappa, mu = (x.clone().requires_grad_(True) for x in material(p))
    seis = adjoint.Seismograms.apply(rho, kappa, mu, sim)
    d_obs = torch.from_numpy(p["d_obs"].astype(np.float32)).cuda()
    loss = 0.5 * p["dt"] * ((seis - d_obs) ** 2).sum()
    loss.backward()
    G = (p["dt"] * (seis - d_obs)).detach()
    ctx2, sim2 = make_sim(p, 20)
    sim2.forward(*material(p))
    ref = sim2.gradient(G)
    for t, r in zip((rho, kappa, mu), ref):
        assert rel_l2(t.grad.cpu().numpy(), r) <= 1e-6


def test_adjoint_on_anomaly_copy(oracle):
    """The 8^3 copy of the sensitivity workload (layered, jittered, 5 % Gaussian anomaly as the
    true model, NGLL 5, 40 steps): device gradients against the oracle's FP64 adjoint, whose
    directional derivative the CPU suite pins to finite differences."""
    from tests import adjoint_cases
    p = adjoint_cases.anomaly_copy(oracle)
    ctx, sim = make_sim(p, every=16)
    seis = sim.forward(*material(p)).cpu().numpy()
    assert rel_l2(seis, p["seis"]) <= TOL_SEIS
    grads = sim.gradient(torch.from_numpy(p["G"].astype(np.float32)).cuda())
    ref = oracle.adjoint_gradient(p["m"], p["dt"], p["u_hist"], p["kw"]["rec_nodes"], p["G"])
    errs = [rel_l2(g, r.reshape(g.shape)) for g, r in zip(grads, ref)]
    print("anomaly copy adjoint rel L2 (rho, kappa, mu):", " ".join(f"{e:.2e}" for e in errs))
    assert errs[0] <= rho_tolerance(oracle, p)
    assert max(errs[1:]) <= TOL_MODULI


@pytest.mark.parametrize("order", [0, 1])
def test_run_snapshots_match_the_graph_run(problem, order):
    """sem_run_snapshots stores u^{n+1} after every step, bit for bit the displacement of
    the same steps taken by sem_run (CUDA graph of ten steps plus single steps), in the
    caller's node order (SEM_OPT_NODE_ORDER 0) or the solver's (1, mapped by sem_node_order)."""
    p = problem
    ctx, sim = make_sim(p, 50)
    sim.set_material(*material(p))
    sem.sem_set_option(ctx, sem.SEM_OPT_NODE_ORDER, order)
    perm = sem.sem_node_order(ctx)
    sem.sem_set_state(ctx)
    snaps = torch.empty((23, 3 * p["mesh"].nglob), device="cuda")
    sem.sem_run_snapshots(ctx, 23, snaps)
    sem.sem_sync(ctx)
    for k in (0, 9, 22):
        sem.sem_set_state(ctx)
        sem.sem_run(ctx, k + 1)
        u, _, _ = sem.sem_get_state(ctx, want=(True, False, False))
        snap = snaps[k].cpu().numpy().reshape(-1, 3)
        if order == 1:
            snap_caller = np.empty_like(snap)
            snap_caller[perm] = snap
            snap = snap_caller
        assert np.array_equal(snap.reshape(u.shape), u)


def test_device_moduli_match_host_moduli(problem):
    """sem_set_moduli_dev gives the same operator, mass and CFL step as sem_set_moduli, and
    rejects a bad value naming its local point."""
    p = problem
    mats = material(p)
    ctx_h, _ = make_sim(p, 50)
    ctx_d, _ = make_sim(p, 50)
    sem.sem_set_moduli(ctx_h, *(x.cpu().numpy() for x in mats))
    sem.sem_set_moduli_dev(ctx_d, *mats)
    assert sem.sem_suggest_dt(ctx_h, 0.4) == sem.sem_suggest_dt(ctx_d, 0.4)
    u = torch.from_numpy(inputs.random_field(p["mesh"].nglob, 3)).cuda()
    out = []
    for ctx in (ctx_h, ctx_d):
        sem.sem_set_dt(ctx, p["dt"])
        f = torch.empty_like(u)
        torch.cuda.synchronize()
        sem.sem_apply_stiffness(ctx, u, f)
        sem.sem_sync(ctx)
        sem.sem_set_state(ctx, None, u.cpu().numpy(), None)
        out.append((f.cpu().numpy(), sem.sem_energy(ctx)))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]  # kinetic energy reads the mass
    bad = mats[0].clone()
    bad[1, 7] = -1.0
    with pytest.raises(sem.SemError, match="local point 71"):
        sem.sem_set_moduli_dev(ctx_d, bad, mats[1], mats[2])
