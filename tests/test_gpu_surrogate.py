"""GPU parity of the surrogate network's kernels with the FP64 oracle network, through the
C ABI: forward outputs, the loss, every parameter gradient and an Adam step. The oracle
takes the bfloat16-rounded weights the kernels read (biases stay float32).

The kernels run their products on the tensor cores (tcgen05 with TMEM accumulators by
default, warp-level mma.sync as the alternative; both are tested) with bfloat16 operands
(activations and gradients rounded to nearest even, weights stored so) and float32
accumulation; the oracle
rounds the same operands (bf16_operands=True) in float64. Tolerances: relative L2 <= 2e-3
for outputs and gradients, 1e-3 for the loss: an operand whose float32 and float64 values
straddle a bfloat16 rounding boundary rounds differently on the two sides (2^-8 relative
for that operand), which a handful of operands per output do; a transposed fragment or a
wrong index gives errors of order one.

Against the unrounded oracle (float64 activations, the same bfloat16 weights) the bound is
derived from the rounding itself: an activation rounded to bfloat16 carries a relative error
uniform in [-u, u], u = 2^-9, of RMS u / sqrt(3) = 1.1e-3. The forward output passes seven
such roundings (three dense layers, four convolutions), which add in quadrature to 3.0e-3;
a gradient passes those and about seven more in the backward products, 4.2e-3. Cancellation
inside the products (a sum smaller than the sum of its terms' magnitudes) amplifies the
relative error; the bound allows a factor of 3: 1e-2 for outputs, 1.5e-2 for gradients and
5e-3 for the loss (measured on GB300: 5.7e-3, 4.0e-3 and 9.6e-4)."""
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


@pytest.fixture(scope="module")
def so():
    from oracle import surrogate_oracle
    return surrogate_oracle


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def oracle_net(so, spec, flat, bf16_operands=True):
    params = {}
    for name, arr in spec.split(flat.astype(np.float64)).items():
        params[name] = so.bf16_round(arr) if name[0] in "WC" else arr
    return so.Surrogate(params, spec.c0, spec.l0, list(zip((spec.c0,) + tuple(spec.stage_cout[:-1]),
                                                           spec.stage_cout, spec.stage_up)), spec.contract,
                        bf16_operands=bf16_operands)


def tiny_spec():
    from paper_2606_12850_gb300 import surrogate
    return surrogate.Spec(in_dim=9, hidden=24, c0=6, l0=7, stage_cout=(10, 8, 5), stage_up=(2, 2, 1), contract=0)


def tiny_contract_spec():
    from paper_2606_12850_gb300 import surrogate
    return surrogate.Spec(in_dim=9, hidden=24, c0=6, l0=7, stage_cout=(10, 8, 12), stage_up=(2, 2, 1), contract=6)


@pytest.mark.parametrize("product", [1, 0])
@pytest.mark.parametrize("contract", [False, True])
def test_loss_and_gradients_match_oracle(so, contract, product):
    from paper_2606_12850_gb300 import surrogate
    spec = tiny_contract_spec() if contract else tiny_spec()
    m = surrogate.Model(spec, max_batch=70)
    m.product = product
    assert m.product == product
    flat = spec.init_params(5)
    flat += inputs.uniform(6, flat.shape, -0.05, 0.05).astype(np.float32)  # nonzero biases
    m.set_params(flat)
    B = 67  # not a multiple of the 64-wide tiles
    x = inputs.uniform(7, (B, 9), -1, 1).astype(np.float32)
    t = inputs.uniform(8, (B, spec.out_c, spec.out_l), -1, 1).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    loss = m.loss_grad(xd, td)
    g = spec.split(m.get_grads())
    net = oracle_net(so, spec, flat)
    ref_loss, ref_g = net.backward(x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - ref_loss) <= 1e-3 * ref_loss
    for name in ref_g:
        assert rel_l2(g[name], ref_g[name]) <= 2e-3, name
    y = torch.empty((B, spec.out_c, spec.out_l), device="cuda")
    m.forward(xd, y)
    m.sync()
    ref_y, _ = net.forward(x.astype(np.float64))
    assert rel_l2(y.cpu().numpy(), ref_y) <= 2e-3
    exact = oracle_net(so, spec, flat, bf16_operands=False)
    exact_y, _ = exact.forward(x.astype(np.float64))
    assert rel_l2(y.cpu().numpy(), exact_y) <= 1e-2
    exact_loss, exact_g = exact.backward(x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - exact_loss) <= 5e-3 * exact_loss
    for name in exact_g:
        assert rel_l2(g[name], exact_g[name]) <= 1.5e-2, name


@pytest.mark.parametrize("product", [1, 0])
def test_full_size_forward_matches_oracle(so, product):
    """The default network (9 -> 512 -> 512 -> [64][125] -> 1000 samples of 6 x 192 channels
    combined with the moment entries) on three inputs, run in chunks smaller than the batch."""
    from paper_2606_12850_gb300 import surrogate
    spec = surrogate.Spec()
    m = surrogate.Model(spec, max_batch=2)
    m.product = product
    flat = spec.init_params(9)
    m.set_params(flat)
    x = inputs.uniform(10, (3, 9), -1, 1).astype(np.float32)
    y = torch.empty((3, spec.out_c, spec.out_l), device="cuda")
    m.forward(torch.from_numpy(x).cuda(), y)
    m.sync()
    ref, _ = oracle_net(so, spec, flat).forward(x.astype(np.float64))
    assert y.shape == ref.shape
    assert rel_l2(y.cpu().numpy(), ref) <= 2e-3
    exact, _ = oracle_net(so, spec, flat, bf16_operands=False).forward(x.astype(np.float64))
    assert rel_l2(y.cpu().numpy(), exact) <= 1e-2


def test_adam_step_matches_oracle(so):
    from paper_2606_12850_gb300 import surrogate
    spec = tiny_spec()
    m = surrogate.Model(spec, max_batch=8)
    flat = spec.init_params(11)
    m.set_params(flat)
    x = torch.from_numpy(inputs.uniform(12, (8, 9), -1, 1).astype(np.float32)).cuda()
    t = torch.from_numpy(inputs.uniform(13, (8, spec.out_c, spec.out_l), -1, 1).astype(np.float32)).cuda()
    p = flat.astype(np.float64)
    mm, vv = np.zeros_like(p), np.zeros_like(p)
    for step in (1, 2):
        m.loss_grad(x, t)
        g = m.get_grads().astype(np.float64)
        m.adam_step(1e-3)
        so.adam_step(p, g, mm, vv, step, 1e-3)
        np.testing.assert_allclose(m.get_params(), p, rtol=1e-6, atol=1e-9)  # same gradients in, float32 update


def test_training_fits_a_smooth_map():
    """300 Adam steps on a smooth synthetic map (traces whose amplitudes depend on the
    inputs) cut the loss by more than ten times."""
    from paper_2606_12850_gb300 import surrogate
    spec = tiny_spec()
    m = surrogate.Model(spec, max_batch=64)
    m.set_params(spec.init_params(21))
    n = 256
    x = inputs.uniform(22, (n, 9), -1, 1).astype(np.float32)
    tt = np.linspace(0, 1, spec.out_l)
    ch = np.arange(spec.out_c)[:, None]
    y = (x[:, :1, None] * np.sin(2 * np.pi * (2 * tt[None, None, :] + 0.1 * ch[None]))
         + 0.5 * x[:, 1:2, None] * np.cos(2 * np.pi * 3 * tt[None, None, :]))
    xd = torch.from_numpy(x).cuda()
    yd = torch.from_numpy(y.astype(np.float32)).cuda()
    losses = surrogate.train(m, xd, yd, epochs=75, batch=64, lr=3e-3, seed=1)
    assert losses[-1] < losses[0] / 10, losses[::10]


def test_predict_or_solve_falls_back_to_the_solver():
    """An untrained network fails the spot check and the solver's traces come back."""
    from paper_2606_12850_gb300 import surrogate
    w = inputs.surrogate_cube(n=4, nsteps=40, nrec_side=2)
    solver = surrogate.Solver(w, shots=4)
    spec = surrogate.Spec(in_dim=9, hidden=16, c0=4, l0=10, stage_cout=(6, 6 * 3 * solver.nrec), stage_up=(2, 2))
    m = surrogate.Model(spec, max_batch=8)
    m.set_params(spec.init_params(3))
    amp = solver.amplitude_model()
    amp.coef = np.zeros(5)  # unit amplitude
    sur = surrogate.Surrogate(m, target_scale=1.0, side=w.mesh.lengths[0], amplitude=amp, solver=solver)
    pos, mom = inputs.surrogate_sources(5, w.mesh.lengths[0], seed=4)
    _, xyz = solver.snapped(pos)
    out, used_solver, errs = sur.predict_or_solve(xyz, mom, tol=0.05, check=2)
    assert used_solver and np.all(errs > 0.05)
    ref, _ = solver.run(xyz, mom)
    assert torch.equal(out, ref)


def test_trained_surrogate_beats_the_nearest_run_and_the_solver_time():
    """On a small medium (8^3 elements, 4 km, 16 surface receivers, 500 steps, Ricker
    0.5 Hz), a network trained on 1024 solver runs predicts 64 held-out runs with a lower
    median error than the traces of the nearest training run (the answer without learning),
    and faster than the solver."""
    import time
    from paper_2606_12850_gb300 import surrogate
    w = inputs.surrogate_cube(n=8, nsteps=500, nrec_side=4)
    solver = surrogate.Solver(w, shots=32)
    tr = surrogate.generate_runs(solver, 1024, seed=1)
    te = surrogate.generate_runs(solver, 64, seed=2)
    spec = surrogate.Spec(in_dim=9, hidden=256, c0=16, l0=125, stage_cout=(32, 32, 6 * 3 * solver.nrec),
                          stage_up=(2, 2, 1))
    m = surrogate.Model(spec, max_batch=64)
    m.set_params(spec.init_params(7))
    amp = solver.amplitude_model().fit(tr.xyz, surrogate.run_rms(tr.y))
    yn = surrogate.training_targets(tr.y, amp(tr.xyz), 1.0)
    scale = 1.0 / float(yn.pow(2).mean().sqrt())
    surrogate.train(m, torch.from_numpy(tr.x).cuda(), yn * scale, epochs=60, batch=64, lr=2e-3, seed=5)
    sur = surrogate.Surrogate(m, scale, w.mesh.lengths[0], amp, solver)
    t = time.perf_counter()
    pred = sur.predict(te.xyz, te.moments)
    t_net = time.perf_counter() - t
    err = np.median(surrogate.rel_l2_per_run(pred, te.y))
    err_nn = np.median(surrogate.rel_l2_per_run(surrogate.nearest_run_baseline(tr, te), te.y))
    print(f"held-out median rel L2: network {err:.3f}, nearest run {err_nn:.3f}; "
          f"network {t_net * 1e3:.1f} ms vs solver {te.seconds * 1e3:.1f} ms")
    assert err < err_nn
    assert t_net < te.seconds


def test_product_kernels_agree_at_full_size():
    """tcgen05 (TMEM accumulators, 128 x 128 tiles) against mma.sync (128/256 x 64 tiles) on
    the default network: loss, every gradient and the output of a ragged batch of 75 runs
    (several 128-wide tiles and a tail in every product, split-K in the weight gradients). The
    two round the same operands to bfloat16 and differ only in the order of float32 sums, which
    can move an activation across a bfloat16 rounding boundary: 2e-3 relative L2 as against
    the oracle."""
    from paper_2606_12850_gb300 import surrogate
    spec = surrogate.Spec()
    flat = spec.init_params(31)
    flat += inputs.uniform(32, flat.shape, -0.02, 0.02).astype(np.float32)
    B = 75
    x = torch.from_numpy(inputs.uniform(33, (B, 9), -1, 1).astype(np.float32)).cuda()
    t = torch.from_numpy(inputs.uniform(34, (B, spec.out_c, spec.out_l), -1, 1).astype(np.float32)).cuda()
    outs = []
    for product in (0, 1):
        m = surrogate.Model(spec, max_batch=B)
        m.product = product
        m.set_params(flat)
        loss = m.loss_grad(x, t)
        y = torch.empty((B, spec.out_c, spec.out_l), device="cuda")
        m.forward(x, y)
        m.sync()
        outs.append((loss, spec.split(m.get_grads()), y.cpu().numpy()))
    (l0, g0, y0), (l1, g1, y1) = outs
    assert abs(l1 - l0) <= 1e-4 * l0
    for name in g0:
        assert rel_l2(g1[name], g0[name].astype(np.float64)) <= 2e-3, name
    assert rel_l2(y1, y0.astype(np.float64)) <= 2e-3


def test_product_wait_limit_reports_timeout():
    """A tcgen05 product that waits for an mbarrier phase nothing completes (the stall test)
    gives up after its limit: the call reports SEM_ETIMEOUT, and with the test switched off
    the same model computes the same loss and gradients as a fresh one."""
    from paper_2606_12850_gb300 import surrogate
    spec = tiny_spec()
    flat = spec.init_params(41)
    x = torch.from_numpy(inputs.uniform(42, (16, 9), -1, 1).astype(np.float32)).cuda()
    t = torch.from_numpy(inputs.uniform(43, (16, spec.out_c, spec.out_l), -1, 1).astype(np.float32)).cuda()
    m = surrogate.Model(spec, max_batch=16)
    m.set_params(flat)
    m.set_option(surrogate.SG_OPT_STALL_TEST, 1)
    with pytest.raises(sem.SemError) as info:
        m.loss_grad(x, t)
    assert info.value.code == -5 and "timed out" in str(info.value)
    m.set_option(surrogate.SG_OPT_STALL_TEST, 0)
    loss = m.loss_grad(x, t)
    fresh = surrogate.Model(spec, max_batch=16)
    fresh.set_params(flat)
    assert loss == fresh.loss_grad(x, t)
    assert np.array_equal(m.get_grads(), fresh.get_grads())
