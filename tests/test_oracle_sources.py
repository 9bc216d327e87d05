"""Pins of the oracle's source forces, at nodes and between nodes: against the closed form
of the work they do on linear fields (the GLL basis reproduces linear fields exactly on
trilinear elements), their net force, point location against the affine closed form of a
regular lattice and against the forward trilinear map, and planted slips."""
import numpy as np
import pytest

from paper_2606_12850_gb300 import inputs


@pytest.fixture(scope="module")
def model(oracle):
    mesh = inputs.structured_hex_mesh(3, 5, 900.0, jitter=0.2, seed=11)
    shape = mesh.ibool.shape
    ones = np.ones(shape)
    return oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, 2500 * ones, 4000 * ones, 2300 * ones, mesh.ngll)


@pytest.mark.parametrize("node_kind", ["interior", "face", "corner"])
def test_moment_force_work_on_linear_fields(oracle, model, node_kind):
    """sum_I f_I . u(x_I) = M : A for u(x) = A x + c: the discrete gradient of a linear
    field is exact, so the equivalent forces do the work M : grad u(x_s). Also sum_I f_I = 0."""
    n = model.ngll
    ib = model.ibool.reshape(model.nspec, -1)
    e = 13  # the centre element of the 3^3 lattice
    local = {"interior": 2 + n * (2 + n * 2), "face": 0 + n * (2 + n * 2), "corner": 0}[node_kind]
    node = int(ib[e, local])
    m6 = inputs.uniform(5, (6,), -1.0, 1.0, stream=4) * 1e15
    nodes, forces = oracle.moment_tensor_forces(model, node, m6)
    M = np.array([[m6[0], m6[3], m6[4]], [m6[3], m6[1], m6[5]], [m6[4], m6[5], m6[2]]])
    X = model.node_xyz
    for seed in range(3):
        A = inputs.uniform(20 + seed, (3, 3), -1.0, 1.0)
        c = inputs.uniform(30 + seed, (3,), -5.0, 5.0)
        u = X[nodes] @ A.T + c
        work = np.sum(forces * u)
        assert abs(work - np.sum(M * A)) <= 1e-10 * np.abs(M).max() * np.abs(A).max() * 9
    assert np.abs(forces.sum(axis=0)).max() <= 1e-10 * np.abs(forces).max()
    assert len(nodes) == 3 * n - 2


def test_moment_force_is_linear_in_the_tensor(oracle, model):
    """The forces are linear in the six tensor entries and sit on the same nodes."""
    ib = model.ibool.reshape(model.nspec, -1)
    n = model.ngll
    node = int(ib[13, 2 + n * (2 + n * 2)])
    a = inputs.uniform(1, (6,), -1, 1)
    b = inputs.uniform(2, (6,), -1, 1)
    na, fa = oracle.moment_tensor_forces(model, node, a)
    nb, fb = oracle.moment_tensor_forces(model, node, b)
    nab, fab = oracle.moment_tensor_forces(model, node, 2 * a - 3 * b)
    assert np.array_equal(na, nb) and np.array_equal(na, nab)
    np.testing.assert_allclose(fab, 2 * fa - 3 * fb, rtol=0, atol=1e-12 * np.abs(fab).max())


@pytest.mark.parametrize("old,new", [
    ("grad = dpsi @ D", "grad = D @ dpsi"),
    ("H[i0, i] * (j == j0) * (k == k0)", "H[i, i0] * (j == j0) * (k == k0)"),
    ("forces.append(M @ grad)", "forces.append(M @ grad * (1 if i != i0 else 0.5))"),
])
def test_planted_source_mistake_is_caught(oracle, model, old, new):
    """A transposed inverse Jacobian, a transposed derivative matrix or a halved self term
    in a copy of moment_tensor_forces breaks the linear-field work pin."""
    import inspect
    src = inspect.getsource(oracle.moment_tensor_forces)
    assert old in src
    ns = dict(oracle.__dict__)
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    ib = model.ibool.reshape(model.nspec, -1)
    n = model.ngll
    node = int(ib[13, 2 + n * (2 + n * 2)])
    m6 = inputs.uniform(5, (6,), -1.0, 1.0, stream=4)
    nodes, forces = ns["moment_tensor_forces"](model, node, m6)
    M = np.array([[m6[0], m6[3], m6[4]], [m6[3], m6[1], m6[5]], [m6[4], m6[5], m6[2]]])
    A = inputs.uniform(20, (3, 3), -1.0, 1.0)
    work = np.sum(forces * (model.node_xyz[nodes] @ A.T))
    assert abs(work - np.sum(M * A)) > 1e-6 * np.abs(M).max()


# ---- sources between nodes: point location and Lagrange interpolation ----------------------


def _trilinear_point(X, ref):
    """x(xi) of a trilinear hexahedron, written out corner by corner (corner c = a + 2b + 4d
    at reference (2a-1, 2b-1, 2d-1)), to generate points of known reference coordinates."""
    x = np.zeros(3)
    for c in range(8):
        sa, sb, sd = (1 if c & 1 else -1), (1 if c & 2 else -1), (1 if c & 4 else -1)
        x += (1 + sa * ref[0]) * (1 + sb * ref[1]) * (1 + sd * ref[2]) / 8.0 * X[c]
    return x


def _linear_work(forces, X, A, c):
    return float(np.sum(forces * (X @ A.T + c)))


@pytest.mark.parametrize("n", [2, 4, 5, 7, 10])
def test_lagrange_derivative_at_any_point(oracle, n):
    """l_i' away from the nodes: exact on polynomials of degree <= N (sum_i p(xi_i) l_i'(x)
    = p'(x)) and equal to central differences of the basis values."""
    xi = oracle.Basis(n).xi
    x = inputs.uniform(n, (17,), -1.0, 1.0)
    dL = oracle.lagrange_basis_derivative(xi, x)
    np.testing.assert_allclose(dL.sum(axis=1), 0.0, atol=1e-11 * n * n)
    for deg in range(1, n):
        np.testing.assert_allclose(dL @ xi ** deg, deg * x ** (deg - 1), rtol=0, atol=1e-11 * n * n)
    h = 1e-6
    fd = (oracle.lagrange_basis(xi, x + h) - oracle.lagrange_basis(xi, x - h)) / (2 * h)
    np.testing.assert_allclose(dL, fd, rtol=0, atol=1e-6 * n * n)


def test_locate_point_regular_lattice_closed_form(oracle):
    """On a regular lattice of spacing h the reference coordinates are affine in x:
    xi = 2 (x - x_lo) / h - 1 in the element whose box holds x."""
    mesh = inputs.structured_hex_mesh(3, 4, 900.0)
    ones = np.ones(mesh.ibool.shape)
    m = oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, ones, 2 * ones, ones, 4)
    for x in inputs.uniform(3, (20, 3), 1.0, 899.0):
        e, ref = oracle.locate_point(m, x)
        lo = m.ctrl[e].min(axis=0)
        assert np.all(lo <= x) and np.all(x <= lo + 300.0)
        np.testing.assert_allclose(ref, 2.0 * (x - lo) / 300.0 - 1.0, rtol=0, atol=1e-12)


def test_locate_point_inverts_the_jittered_map(oracle, model):
    """Points of known reference coordinates in distorted elements are found in their
    element with those coordinates; a point on the face shared by elements 12 and 13 goes to
    12 (the lowest index); a point outside the mesh is refused."""
    for e in (0, 13, 26):
        for seed in range(4):
            ref = inputs.uniform(40 + seed, (3,), -0.97, 0.97, stream=e)
            e2, r2 = oracle.locate_point(model, _trilinear_point(model.ctrl[e], ref))
            assert e2 == e
            np.testing.assert_allclose(r2, ref, rtol=0, atol=1e-12)
    ref = np.array([-1.0, 0.3, -0.2])
    e2, r2 = oracle.locate_point(model, _trilinear_point(model.ctrl[13], ref))
    assert e2 == 12 and abs(r2[0] - 1.0) < 1e-12
    with pytest.raises(ValueError):
        oracle.locate_point(model, np.array([-10.0, 450.0, 450.0]))


def test_point_force_between_nodes(oracle, model):
    """f_I = F psi_I(x_s): the forces sum to F (partition of unity) and do the work
    F . u(x_s) on every linear field (the basis reproduces linear fields); at a node the
    whole force sits on that node."""
    F = np.array([0.3, -1.2, 2.0]) * 1e10
    X = model.node_xyz
    for seed in range(3):
        ref = inputs.uniform(60 + seed, (3,), -0.9, 0.9)
        x_s = _trilinear_point(model.ctrl[13], ref)
        e, _, nodes, f = oracle.point_source_forces(model, x_s, force=F)
        assert e == 13 and len(nodes) == model.ngll ** 3
        np.testing.assert_allclose(f.sum(axis=0), F, rtol=1e-12)
        for s2 in range(2):
            A = inputs.uniform(70 + s2, (3, 3), -1.0, 1.0)
            c = inputs.uniform(80 + s2, (3,), -5.0, 5.0)
            exact = float(F @ (A @ x_s + c))
            assert abs(_linear_work(f, X[nodes], A, c) - exact) <= 1e-12 * np.abs(F).max() * 1e4
    n = model.ngll
    node = int(model.ibool.reshape(model.nspec, -1)[13, 2 + n * (1 + n * 3)])
    _, _, nodes, f = oracle.point_source_forces(model, X[node], force=F)
    k = list(nodes).index(node)
    np.testing.assert_allclose(f[k], F, rtol=1e-12)
    assert np.abs(np.delete(f, k, axis=0)).max() <= 1e-12 * np.abs(F).max()


def test_moment_source_between_nodes(oracle, model):
    """f_I = M grad psi_I(x_s): zero net force, work M : A on every linear field u = A x + c,
    and at a node it equals the node form (moment_tensor_forces, built from the nodal
    derivative matrix instead of the derivative at an arbitrary point)."""
    m6 = inputs.uniform(5, (6,), -1.0, 1.0, stream=9) * 1e15
    M = np.array([[m6[0], m6[3], m6[4]], [m6[3], m6[1], m6[5]], [m6[4], m6[5], m6[2]]])
    X = model.node_xyz
    for seed in range(3):
        x_s = _trilinear_point(model.ctrl[13], inputs.uniform(90 + seed, (3,), -0.9, 0.9))
        _, _, nodes, f = oracle.point_source_forces(model, x_s, moment=m6)
        assert np.abs(f.sum(axis=0)).max() <= 1e-10 * np.abs(f).max()
        A = inputs.uniform(100 + seed, (3, 3), -1.0, 1.0)
        c = inputs.uniform(110 + seed, (3,), -5.0, 5.0)
        assert abs(_linear_work(f, X[nodes], A, c) - np.sum(M * A)) <= 1e-10 * np.abs(M).max() * 9
    n = model.ngll
    node = int(model.ibool.reshape(model.nspec, -1)[13, 2 + n * (2 + n * 2)])
    _, _, nodes, f = oracle.point_source_forces(model, X[node], moment=m6)
    nref, fref = oracle.moment_tensor_forces(model, node, m6)
    dense = np.zeros((model.nglob, 3))
    dense[nodes] = f
    expect = np.zeros((model.nglob, 3))
    expect[nref] = fref
    np.testing.assert_allclose(dense, expect, rtol=0, atol=1e-9 * np.abs(fref).max())


@pytest.mark.parametrize("old,new", [
    ("f = M @ (dpsi @ D)", "f = M @ (D @ dpsi)"),
    ("L[0][i] * dL[1][j] * L[2][k]", "L[0][i] * dL[1][j] * dL[2][k]"),
    ("(L[0][i] * L[1][j] * L[2][k])", "(L[0][i] * L[1][i] * L[2][k])"),
    ("D = np.linalg.inv(model.ctrl[e].T @ dN)", "D = np.linalg.inv(dN.T @ model.ctrl[e])"),
])
def test_planted_interpolation_mistake_is_caught(oracle, model, old, new):
    """A transposed inverse Jacobian, a wrong factor in the gradient of psi, a wrong index in
    psi or a transposed Jacobian in a copy of point_source_forces breaks a linear-field work
    pin."""
    import inspect
    src = inspect.getsource(oracle.point_source_forces)
    assert old in src
    ns = dict(oracle.__dict__)
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    x_s = _trilinear_point(model.ctrl[13], np.array([0.31, -0.52, 0.17]))
    A = inputs.uniform(120, (3, 3), -1.0, 1.0)
    c = inputs.uniform(121, (3,), -5.0, 5.0)
    X = model.node_xyz
    m6 = inputs.uniform(5, (6,), -1.0, 1.0, stream=9)
    M = np.array([[m6[0], m6[3], m6[4]], [m6[3], m6[1], m6[5]], [m6[4], m6[5], m6[2]]])
    F = np.array([0.3, -1.2, 2.0])
    _, _, nodes, f = ns["point_source_forces"](model, x_s, moment=m6)
    bad_moment = abs(_linear_work(f, X[nodes], A, c) - np.sum(M * A)) > 1e-6 * np.abs(M).max()
    _, _, nodes, f = ns["point_source_forces"](model, x_s, force=F)
    bad_force = abs(_linear_work(f, X[nodes], A, c) - F @ (A @ x_s + c)) > 1e-6 * np.abs(F).max()
    assert bad_moment or bad_force


@pytest.mark.parametrize("old,new", [
    ("step = np.linalg.solve(A, N @ X - x)", "step = np.linalg.solve(A, x - N @ X)"),
    ("if np.all(np.abs(ref) <= 1.0 + tol):", "if np.any(np.abs(ref) <= 1.0 + tol):"),
])
def test_planted_location_mistake_is_caught(oracle, model, old, new):
    """A flipped Newton residual or an inside test on one coordinate only (a copy of
    locate_point) misplaces at least one of a few points near the faces of a distorted
    element. (A transposed Jacobian or another starting point is not a mistake of this
    kind: Newton still converges to the same point, only more slowly.)"""
    import inspect
    src = inspect.getsource(oracle.locate_point)
    assert old in src
    ns = dict(oracle.__dict__)
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    wrong = 0
    for ref in ([-0.9, 0.3, 0.2], [0.6, -0.7, 0.45], [0.1, 0.95, -0.9]):
        ref = np.array(ref)
        try:
            e2, r2 = ns["locate_point"](model, _trilinear_point(model.ctrl[13], ref))
            wrong += e2 != 13 or np.abs(r2 - ref).max() > 1e-6
        except (ValueError, np.linalg.LinAlgError):
            wrong += 1
    assert wrong > 0
