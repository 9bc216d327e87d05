"""Host-side helpers (no GPU): the algorithmic byte counts behind the benchmark's roofline,
the profile-hash guard on the committed DRAM traffic, the surrogate's input features and
its fitted amplitude model, and the seeded generator of the inputs."""
import os

import numpy as np
import pytest

from paper_2606_12850_gb300 import inputs


def test_algorithmic_bytes():
    import bench
    a = bench.algorithmic_bytes(8, 5, 33 ** 3)
    nloc = 8 * 125
    assert a["nloc"] == nloc
    assert a["forces"] == 52 * nloc + 24 * 33 ** 3
    assert a["step"] == 52 * nloc + 76 * 33 ** 3


def test_profiled_traffic_follows_the_kernel_sources(tmp_path, monkeypatch):
    import bench
    got = bench.profiled_traffic(5)
    text = open(os.path.join(bench.ROOT, "profiles", "patch_forces_kernel_ngll5_layered.md")).read()
    if bench.kernel_source_hash() in text:
        assert got is not None and got > 2.0e9  # the committed capture is of these sources
    else:
        assert got is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0000000000000000")
    assert bench.profiled_traffic(5) is None  # a changed kernel voids the counters


def test_surrogate_features_and_amplitude_model():
    from paper_2606_12850_gb300 import surrogate
    side = 4000.0
    pos, mom = inputs.surrogate_sources(500, side, seed=6)
    x = surrogate.features(pos, mom, side)
    assert x.shape == (500, 9) and x.dtype == np.float32
    assert np.all(np.abs(x[:, :3]) <= 1.0)
    rec = np.array([[1000.0, 1000.0, side], [3000.0, 3000.0, side]])
    amp = surrogate.AmplitudeModel(side, rec)
    coef = np.array([1.5, 0.7, -0.2, 0.1, -1.1])
    rms = np.exp(amp.design(pos) @ coef)
    amp.fit(pos, rms)
    np.testing.assert_allclose(amp.coef, coef, rtol=0, atol=1e-9)
    np.testing.assert_allclose(amp(pos), rms, rtol=1e-9)


def test_spec_split_roundtrip():
    from paper_2606_12850_gb300 import surrogate
    spec = surrogate.Spec(in_dim=9, hidden=8, c0=3, l0=5, stage_cout=(4, 12), stage_up=(2, 1), contract=6)
    flat = spec.init_params(2)
    parts = spec.split(flat)
    assert list(parts) == [n for n, _ in spec.shapes()]
    assert np.array_equal(np.concatenate([parts[n].ravel() for n in parts]), flat)
    assert (spec.out_c, spec.out_l) == (2, 10)


def test_splitmix64_known_answers():
    """The seeded generator both sides draw their inputs from is splitmix64 as published:
    from state 0 its first outputs are 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
    0x06C45D188009454F. Uniforms lie in [low, high); Box-Muller normals have mean 0 and
    variance 1 (within 4 standard errors over 2^17 samples)."""
    from paper_2606_12850_gb300 import inputs
    assert [int(v) for v in inputs.splitmix64(0, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    u = inputs.uniform(7, (1 << 17,), -2.0, 3.0)
    assert u.min() >= -2.0 and u.max() < 3.0
    z = inputs.normal(7, (1 << 17,))
    se = 1.0 / np.sqrt(z.size)
    assert abs(z.mean()) < 4 * se and abs(z.var() - 1.0) < 4 * np.sqrt(2.0) * se
    assert np.array_equal(inputs.uniform(7, (5,), stream=3), inputs.uniform(7, (5,), stream=3))
    assert not np.array_equal(inputs.uniform(7, (5,), stream=3), inputs.uniform(7, (5,), stream=4))


class _FakeDevice:
    def __init__(self, index):
        self.index = index


class _FakeCudaTensor:
    """Stands in for a CUDA tensor: only the attributes the binding inspects."""

    is_cuda = True

    def __init__(self, dtype, device, n=12, contiguous=True):
        self.dtype = dtype
        self.device = _FakeDevice(device)
        self._n = n
        self._contiguous = contiguous

    def is_contiguous(self):
        return self._contiguous

    def numel(self):
        return self._n

    def data_ptr(self):  # never reached by the rejected cases
        raise AssertionError("the address of a rejected tensor was taken")


def test_device_arrays_checked_before_any_library_call():
    """A float16/bfloat16 tensor (half the byte size the kernels assume), a tensor on
    another GPU, a non-contiguous or too-small tensor are refused by the binding itself."""
    import pytest
    torch = pytest.importorskip("torch")
    from paper_2606_12850_gb300 import sem
    ctx = sem.Ctx(0, 5)
    ctx.handle = None  # no library context: a call that got through would fail differently
    ctx.device, ctx.nglob = 0, 4
    for dt in (torch.float16, torch.bfloat16, torch.float64, torch.int32):
        with pytest.raises(TypeError):
            sem._dev(_FakeCudaTensor(dt, 0), 12, ctx)
    with pytest.raises(ValueError, match="cuda:1"):
        sem._dev(_FakeCudaTensor(torch.float32, 1), 12, ctx)
    with pytest.raises(ValueError, match="contiguous"):
        sem._dev(_FakeCudaTensor(torch.float32, 0, contiguous=False), 12, ctx)
    with pytest.raises(ValueError, match="needs 12"):
        sem._dev(_FakeCudaTensor(torch.float32, 0, n=11), 12, ctx)
    with pytest.raises(TypeError):
        sem.sem_apply_stiffness(ctx, _FakeCudaTensor(torch.float16, 0), _FakeCudaTensor(torch.float32, 0))


def test_predict_or_solve_requires_a_solver():
    from paper_2606_12850_gb300 import surrogate
    amp = surrogate.AmplitudeModel(4000.0, np.array([[1000.0, 1000.0, 4000.0]]))
    sur = surrogate.Surrogate(None, 1.0, 4000.0, amp, solver=None)
    with pytest.raises(ValueError, match="solver"):
        sur.predict_or_solve(np.zeros((2, 3)), np.zeros((2, 6)), tol=0.5)


def test_product_flops_of_the_default_network():
    """The FLOP count behind the surrogate's reported TFLOP/s: 2 per multiply-add of the three
    dense layers (9x512, 512x512, 512x8000) and the four width-3 convolutions (64->96 at 250
    samples, 96->96 at 500 and 1000, 96->1152 at 1000)."""
    import bench
    from paper_2606_12850_gb300 import surrogate
    dense = 9 * 512 + 512 * 512 + 512 * 64 * 125
    conv = 96 * 64 * 3 * 250 + 96 * 96 * 3 * 500 + 96 * 96 * 3 * 1000 + 1152 * 96 * 3 * 1000
    assert bench.product_flops(surrogate.Spec()) == 2 * (dense + conv) == 764437504


def test_reciprocal_division_is_exact_below_2_pow_24():
    """The products' index maps divide k (a sample-time index, k < 2^24 as sg_create enforces)
    by a layer length d with q = trunc(float(k) * float(1/d)) in float32 and one correction
    step q += (r >= d) - (r < 0), r = k - q d. Checked for every k < 2^24 against integer
    division, for the lengths of the default and test networks and a spread of others."""
    ks = np.arange(1 << 24, dtype=np.int64)
    kf = ks.astype(np.float32)  # exact: every k < 2^24 is a float32
    for d in (1, 3, 7, 14, 28, 125, 250, 500, 1000, 997, 1024, 4093, 65537):
        inv = np.float32(1.0) / np.float32(d)
        q = np.trunc(kf * inv).astype(np.int64)  # float32 product rounded to nearest
        r = ks - q * d
        q += (r >= d).astype(np.int64) - (r < 0).astype(np.int64)
        assert np.array_equal(q, ks // d), d
