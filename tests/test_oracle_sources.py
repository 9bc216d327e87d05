"""Pins of the oracle's moment-tensor source forces: against the closed form of the work
they do on linear fields (the GLL basis reproduces linear fields exactly on trilinear
elements), and their vanishing net force."""
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
