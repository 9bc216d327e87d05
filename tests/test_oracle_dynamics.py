"""Pins of the oracle's time stepping (explicit second-order Newmark, Sec. I and V-C) and of
the whole solver against closed forms: exact discrete energy conservation, a travelling
plane wave in a periodic box, second-order accuracy in time, spectral accuracy in the
polynomial order at fixed points per wavelength (the trend behind the iso-accuracy study
of Sec. V-C), the CFL step of the homogeneous cube, and mirror symmetry of its surface
seismograms.
"""
import numpy as np
import pytest

from paper_2606_12850_gb300 import inputs


def test_discrete_energy_conserved(oracle):
    """Without a source the explicit Newmark scheme conserves
    E^{n+1/2} = 1/2 v_h^T M v_h + 1/2 (u^{n+1})^T K u^n exactly for symmetric K."""
    mesh = inputs.structured_hex_mesh(3, 4, 600.0, jitter=0.2, seed=31)
    shape = mesh.ibool.shape
    rho = inputs.uniform(1, shape, 2000, 3000, stream=1).astype(np.float32)
    vp = inputs.uniform(1, shape, 3000, 5000, stream=2).astype(np.float32)
    vs = (vp / 1.8).astype(np.float32)
    m = oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, rho, vp, vs, mesh.ngll)
    u0 = inputs.random_field(m.nglob, 3).astype(np.float64) * 1e-3
    dt = m.cfl_dt(0.4)
    *_, E = oracle.newmark_run(m, dt, 200, u0=u0, energy=True)
    assert E[0] > 0
    assert np.max(np.abs(E / E[0] - 1.0)) < 1e-11


def test_integer_step_energy_conserved(oracle):
    """The same conserved energy at integer steps, E_n = 1/2 v^T M v + 1/2 u^T K u -
    dt^2/8 a^T M a (the staggered form with v^{n+1/2} = v^n + dt/2 a^n and K u^n = -M a^n),
    holds to rounding across restarts of the run, while kinetic plus potential energy alone
    moves at the 1e-3 level; the GPU energy-drift test measures this quantity."""
    mesh = inputs.structured_hex_mesh(4, 5, 800.0, jitter=0.15, seed=9)
    shape = mesh.ibool.shape
    rho = inputs.uniform(1, shape, 2000, 3000, stream=1).astype(np.float32)
    vp = inputs.uniform(1, shape, 3000, 5000, stream=2).astype(np.float32)
    vs = (vp / 1.8).astype(np.float32)
    m = oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, rho, vp, vs, 5)
    dt = m.cfl_dt(0.4)
    u = np.sin(m.node_xyz / 300.0 + np.array([0.0, 1.0, 2.0])) * 1e-3
    v = np.zeros_like(u)
    a = m.forces(u) / m.mass[:, None]

    def energies(u, v, a):
        plain = 0.5 * np.sum(m.mass[:, None] * v * v) - 0.5 * np.sum(u * m.forces(u))
        return plain - dt * dt / 8.0 * np.sum(m.mass[:, None] * a * a), plain

    E = [energies(u, v, a)]
    for _ in range(3):
        _, u, v, a = oracle.newmark_run(m, dt, 40, u0=u, v0=v, a0=a)
        E.append(energies(u, v, a))
    E = np.array(E)
    assert np.abs(E[:, 0] / E[0, 0] - 1.0).max() < 1e-12
    assert np.abs(E[:, 1] / E[0, 1] - 1.0).max() > 1e-4


def _plane_wave(oracle, ngll, nz, courant, periods=2.0, comp=2):
    """Travelling plane wave u_comp = sin(k z - w t) along z in a periodic box of height
    1 km; returns the Sec. V-C-1 error of the recorded waveforms on a line of stations."""
    L = 1000.0
    mesh = inputs.structured_hex_mesh((2, 2, nz), ngll, (2 * L / nz, 2 * L / nz, L), periodic=True)
    one = np.ones(mesh.nspec)
    vp, vs = 3000.0, 1730.0
    m = oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, inputs.per_point(mesh, 2500 * one),
                     inputs.per_point(mesh, vp * one), inputs.per_point(mesh, vs * one), ngll)
    k = 2 * np.pi / L
    w = (vp if comp == 2 else vs) * k
    X = m.node_xyz
    z = X[:, 2]
    u0 = np.zeros((m.nglob, 3))
    u0[:, comp] = np.sin(k * z)
    v0 = np.zeros((m.nglob, 3))
    v0[:, comp] = -w * np.cos(k * z)
    a0 = m.forces(u0) / m.mass[:, None]
    dt = m.cfl_dt(courant)
    T = periods * 2 * np.pi / w
    n = int(round(T / dt))
    dt = T / n
    line = np.isclose(np.mod(X[:, 0], mesh.lengths[0]), 0) & np.isclose(np.mod(X[:, 1], mesh.lengths[1]), 0)
    rec = np.nonzero(line)[0]
    seis, *_ = oracle.newmark_run(m, dt, n, u0=u0, v0=v0, a0=a0, rec_nodes=rec)
    t = dt * np.arange(1, n + 1)
    theory = np.sin(k * z[rec][:, None] - w * t[None, :])
    return oracle.dispersion_error(seis[:, comp, :].ravel(), theory.ravel())


def test_plane_wave_fixed_points_per_wavelength(oracle):
    """At 12 GLL intervals per wavelength the waveform error falls monotonically as the
    order rises (p = 2, 3, 4, 6 on 6, 4, 3, 2 elements per wavelength): the effect that
    drives the (h, p) iso-accuracy frontier of Sec. IV-B / V-C. The time step is small
    (Courant 0.1) so that spatial dispersion dominates."""
    errs = [_plane_wave(oracle, ngll, nz, 0.1) for ngll, nz in ((3, 6), (4, 4), (5, 3), (7, 2))]
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert errs[0] < 1e-4 and errs[-1] < 1e-7


def test_shear_plane_wave_travels_at_vs(oracle):
    """A transverse plane wave u_x (or u_y) = sin(k z - w t) with w = vs k is a solution of
    the isotropic elastic equation: the recorded waveform error is small and falls with the
    order at fixed points per wavelength, and the two polarisations agree (symmetry of the
    box). A shear modulus with a wrong weight would move the wave at another speed."""
    errs = [_plane_wave(oracle, ngll, nz, 0.1, comp=0) for ngll, nz in ((3, 6), (5, 3), (7, 2))]
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert errs[0] < 1e-4 and errs[-1] < 1e-7
    assert abs(_plane_wave(oracle, 5, 3, 0.1, comp=1) / errs[1] - 1.0) < 1e-9


def test_newmark_second_order_in_time(oracle):
    """Halving dt at high order divides the squared-norm error ratio by about 2^4
    (amplitude error O(dt^2))."""
    e1 = _plane_wave(oracle, 7, 2, 0.4)
    e2 = _plane_wave(oracle, 7, 2, 0.2)
    assert 10.0 < e1 / e2 < 22.0


def test_cfl_step_homogeneous_cube(oracle):
    """Homogeneous 8^3 cube of side 1 km at NGLL=5: dx_min = 62.5 m (1 - sqrt(3/7)) and
    dt = 0.4 dx_min / 3000 m/s."""
    w = inputs.homogeneous_cube()
    m = oracle.build_model(w)
    expect = 0.4 * 62.5 * (1 - np.sqrt(3.0 / 7.0)) / 3000.0
    assert abs(m.cfl_dt(w.courant) / expect - 1.0) < 1e-13


def test_locate_homogeneous_cube(oracle):
    """Source at the cube centre is lattice node (16,16,16) of the 33^3 GLL lattice; the
    receivers are top-face lattice nodes (4 x, 4 y) multiples."""
    w = inputs.homogeneous_cube()
    m = oracle.build_model(w)
    src, rec = oracle.locate_workload(m, w)
    G = 33
    assert src[0] == 16 + G * (16 + G * 16)
    expect = [gx + G * (gy + G * 32) for gy in (12, 20) for gx in (4, 12, 20, 28)]
    assert list(rec) == expect


@pytest.mark.slow
def test_homogeneous_cube_mirror_symmetry(oracle):
    """Homogeneous cube, +z force at the centre: the problem is symmetric under x -> L-x,
    y -> L-y and x <-> y, so mirrored receivers record u_z equal and the mirrored
    horizontal component with opposite sign (to FP64 rounding)."""
    w = inputs.homogeneous_cube(nsteps=120)
    r = oracle.run_workload(w)
    s = r["seis"]  # receivers: x in (125,375,625,875) for y=375, then for y=625
    scale = np.abs(s).max()
    assert scale > 0
    tol = 1e-12 * scale
    for a, b in ((0, 3), (1, 2), (4, 7), (5, 6)):  # x mirror
        np.testing.assert_allclose(s[a, 2], s[b, 2], atol=tol)
        np.testing.assert_allclose(s[a, 0], -s[b, 0], atol=tol)
        np.testing.assert_allclose(s[a, 1], s[b, 1], atol=tol)
    for a, b in ((0, 4), (1, 5), (2, 6), (3, 7)):  # y mirror
        np.testing.assert_allclose(s[a, 2], s[b, 2], atol=tol)
        np.testing.assert_allclose(s[a, 1], -s[b, 1], atol=tol)
    np.testing.assert_allclose(s[1, 0], s[1, 1], atol=tol)  # (375, 375) on the diagonal
