"""Pins of the oracle's geometry, mass and matrix-free stiffness action (Sec. II-B).

The stiffness action is fixed by facts that do not come from the oracle's own formulas:
closed-form geometry of a regular lattice, the exact volume of a box with fixed
boundary, the rigid-body null space, the finite-element patch test (a linear displacement
leaves interior nodes in equilibrium, exactly under GLL quadrature for N >= 2 on trilinear
hexahedra), symmetry and positivity of K, and a dense stiffness matrix assembled from
Kronecker products of 1D matrices with an explicit fourth-order isotropic tensor.
"""
import numpy as np
import pytest

from paper_2606_12850_gb300 import inputs


def _random_material(mesh, seed):
    shape = mesh.ibool.shape
    rho = inputs.uniform(seed, shape, 2000.0, 3000.0, stream=1).astype(np.float32)
    vp = inputs.uniform(seed, shape, 3000.0, 5000.0, stream=2).astype(np.float32)
    vs = (vp / inputs.uniform(seed, shape, 1.6, 2.0, stream=3)).astype(np.float32)
    return rho, vp, vs


def _model(oracle, mesh, rho, vp, vs):
    return oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, rho, vp, vs, mesh.ngll)


@pytest.mark.parametrize("ngll", [2, 3, 5, 8])
def test_regular_geometry_closed_form(oracle, ngll):
    """Regular lattice with spacing h: dxi/dx = 2/h on the diagonal, 0 off it,
    J = (h/2)^3, and GLL positions x = x_e + (1 + xi) h / 2."""
    h = 125.0
    mesh = inputs.structured_hex_mesh(2, ngll, 2 * h)
    basis = oracle.Basis(ngll)
    xyz, dxi_dx, jac = oracle.element_geometry(mesh.ctrl, basis)
    np.testing.assert_allclose(jac, (h / 2) ** 3, rtol=1e-14)
    eye = np.eye(3)[None, :, :, None, None, None] * (2.0 / h)
    np.testing.assert_allclose(dxi_dx, np.broadcast_to(eye, dxi_dx.shape), atol=1e-17)
    e = 5  # element (1, 0, 1)
    ex, ey, ez = mesh.elem_ijk[e]
    xi = basis.xi
    np.testing.assert_allclose(xyz[e, 0, 0, 0, :], ex * h + (1 + xi) * h / 2, rtol=1e-14)
    np.testing.assert_allclose(xyz[e, 1, 0, :, 0], ey * h + (1 + xi) * h / 2, rtol=1e-14)
    np.testing.assert_allclose(xyz[e, 2, :, 0, 0], ez * h + (1 + xi) * h / 2, rtol=1e-14)


@pytest.mark.parametrize("ngll", [3, 5])
def test_mass_sums_to_box_mass(oracle, ngll):
    """Diagonal mass (Sec. II-B): with fixed box faces, jitter moves only interior
    vertices, so sum_I M_I = rho * L^3 exactly (det J of a trilinear hexahedron has degree
    <= 2 per variable, integrated exactly by GLL for N >= 2); every M_I > 0."""
    L = 1000.0
    mesh = inputs.structured_hex_mesh(3, ngll, L, jitter=0.2, seed=11)
    rho = inputs.per_point(mesh, np.full(mesh.nspec, 2500.0))
    m = _model(oracle, mesh, rho, rho, rho * 0 + 1.0)
    assert abs(m.mass.sum() / (2500.0 * L ** 3) - 1.0) < 1e-13
    assert np.all(m.mass > 0)


@pytest.mark.parametrize("ngll", [2, 3, 5])
def test_rigid_body_null_space(oracle, ngll):
    """K annihilates rigid translations (exactly) and infinitesimal rotations
    u = omega x (x - c) (to rounding), on a jittered mesh with random material."""
    mesh = inputs.structured_hex_mesh(3, ngll, 900.0, jitter=0.2, seed=5)
    m = _model(oracle, mesh, *_random_material(mesh, 3))
    X = m.node_xyz
    u_rand = inputs.random_field(m.nglob, 9).astype(np.float64)
    scale = np.linalg.norm(m.forces(u_rand)) / np.linalg.norm(u_rand)
    t = np.tile([0.3, -1.2, 0.7], (m.nglob, 1))
    assert np.max(np.abs(m.forces(t))) <= 1e-12 * scale * np.linalg.norm(t)
    omega = np.array([0.4, -0.25, 0.9])
    u = np.cross(omega, X - X.mean(axis=0))
    assert np.linalg.norm(m.forces(u)) <= 1e-12 * scale * np.linalg.norm(u)


@pytest.mark.parametrize("ngll", [3, 5])
def test_patch_test_linear_field(oracle, ngll):
    """Patch test: a linear displacement u = A x + b gives a constant stress, so every
    interior node is in equilibrium. Under GLL quadrature this holds exactly for N >= 2 on
    trilinear hexahedra (the integrand has degree <= N+1 <= 2N-1 per variable)."""
    L = 1000.0
    mesh = inputs.structured_hex_mesh(3, ngll, L, jitter=0.2, seed=21)
    const = np.ones(mesh.nspec)
    m = _model(oracle, mesh, inputs.per_point(mesh, 2600 * const),
               inputs.per_point(mesh, 4000 * const), inputs.per_point(mesh, 2300 * const))
    A = np.array([[1.0, 0.3, -0.2], [0.1, -0.5, 0.4], [0.25, 0.6, 0.8]]) * 1e-3
    u = m.node_xyz @ A.T + np.array([0.1, 0.2, 0.3])
    f = m.forces(u)
    X = m.node_xyz
    tol = 1e-9 * L
    interior = np.all((X > tol) & (X < L - tol), axis=1)
    assert interior.sum() > 0
    boundary_scale = np.abs(f[~interior]).max()
    assert boundary_scale > 0
    assert np.abs(f[interior]).max() <= 1e-12 * boundary_scale


def test_symmetric_positive(oracle):
    """K is symmetric (v.Ku = u.Kv) and positive semi-definite (u.Ku >= 0)."""
    mesh = inputs.structured_hex_mesh(3, 4, 800.0, jitter=0.2, seed=8)
    m = _model(oracle, mesh, *_random_material(mesh, 4))
    u = inputs.random_field(m.nglob, 1).astype(np.float64)
    v = inputs.random_field(m.nglob, 2).astype(np.float64)
    vKu = -np.sum(v * m.forces(u))
    uKv = -np.sum(u * m.forces(v))
    uKu = -np.sum(u * m.forces(u))
    assert abs(vKu - uKv) <= 1e-12 * abs(uKu)
    assert uKu > 0


def _dense_element_stiffness(oracle, ctrl, rho, vp, vs, ngll):
    """Dense K_e of one element from Kronecker products of the 1D derivative matrix and
    the GLL weights, with the isotropic stiffness tensor
    C_cdab = lambda d_cd d_ab + mu (d_ca d_db + d_cb d_da) written out per quadrature point."""
    basis = oracle.Basis(ngll)
    n = ngll
    _, dxi_dx, jac = oracle.element_geometry(ctrl[None], basis)
    I = np.eye(n)
    D = basis.hprime
    Dr = [np.kron(I, np.kron(I, D)), np.kron(I, np.kron(D, I)), np.kron(D, np.kron(I, I))]
    W = np.kron(basis.w, np.kron(basis.w, basis.w))
    G = dxi_dx[0].reshape(3, 3, -1)  # [r, d, q]
    J = jac[0].reshape(-1)
    B = [sum(G[r, d][:, None] * Dr[r] for r in range(3)) for d in range(3)]
    rho, vp, vs = (np.asarray(a, dtype=np.float64).reshape(-1) for a in (rho, vp, vs))
    mu = rho * vs ** 2
    lam = rho * (vp ** 2 - 2 * vs ** 2)
    d = np.eye(3)
    npt = n ** 3
    K = np.zeros((3 * npt, 3 * npt))
    for c in range(3):
        for dd in range(3):
            for a in range(3):
                for b in range(3):
                    Cq = lam * d[c, dd] * d[a, b] + mu * (d[c, a] * d[dd, b] + d[c, b] * d[dd, a])
                    if not np.any(Cq):
                        continue
                    K[c * npt:(c + 1) * npt, a * npt:(a + 1) * npt] += \
                        B[dd].T @ ((J * W * Cq)[:, None] * B[b])
    return K


@pytest.mark.parametrize("ngll", [2, 3, 4])
def test_brute_force_dense_stiffness(oracle, ngll):
    """The matrix-free element force (Sec. II-B) equals -K_e u for a dense K_e built
    independently from Kronecker products, on a distorted trilinear element with random
    per-point material."""
    n = ngll
    mesh = inputs.structured_hex_mesh(3, ngll, 300.0, jitter=0.25, seed=17)
    e = 13  # the centre element: all eight corners jittered
    ctrl = mesh.ctrl[e]
    rho, vp, vs = (a[e] for a in _random_material(mesh, 12))
    K = _dense_element_stiffness(oracle, ctrl, rho, vp, vs, ngll)
    np.testing.assert_allclose(K, K.T, rtol=0, atol=1e-12 * np.abs(K).max())
    basis = oracle.Basis(ngll)
    _, dxi_dx, jac = oracle.element_geometry(ctrl[None], basis)
    kappa, mu = oracle.moduli(rho.reshape(1, n, n, n), vp.reshape(1, n, n, n), vs.reshape(1, n, n, n))
    u = inputs.uniform(5, (3, n ** 3), -1, 1)
    F = oracle.element_forces(u.reshape(1, 3, n, n, n), dxi_dx, jac, kappa, mu, basis)
    np.testing.assert_allclose(F.reshape(-1), -(K @ u.reshape(-1)), rtol=0,
                               atol=1e-12 * np.abs(K @ u.reshape(-1)).max())


def test_gather_assemble_are_adjoint(oracle):
    """Assembly is the transpose of the gather: <assemble(F), u> = <F, gather(u)>."""
    mesh = inputs.structured_hex_mesh(2, 3, 1.0, periodic=True)
    n = mesh.ngll
    u = inputs.random_field(mesh.nglob, 4).astype(np.float64)
    F = inputs.uniform(6, (mesh.nspec, 3, n, n, n), -1, 1)
    lhs = np.sum(oracle.assemble(F, mesh.ibool, mesh.nglob) * u)
    rhs = np.sum(F * oracle.gather(u, mesh.ibool, n))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
