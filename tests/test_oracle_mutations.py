"""The oracle's pins are sensitive: each plausible slip planted in a copy of the oracle's
stiffness action (on the CPU, never in the CUDA path) makes at least one pin fail.

A mutant is the oracle's ``element_forces`` with one token changed: a transposed
derivative matrix, a dropped symmetrisation, a wrong weight index, a lost factor of two
on mu, a dropped lambda shift, a sign flip of one direction.
"""
import inspect

import numpy as np
import pytest

from paper_2606_12850_gb300 import inputs

MUTATIONS = [
    ('np.einsum("il,eckjl->eckji", H, u_e)', 'np.einsum("li,eckjl->eckji", H, u_e)'),
    ('eps = 0.5 * (grad + grad.transpose(0, 2, 1, 3, 4, 5))', 'eps = grad'),
    ('np.einsum("k,i,l,lj,eckli->eckji", w, w, w, H, t[:, 1])',
     'np.einsum("k,j,l,lj,eckli->eckji", w, w, w, H, t[:, 1])'),
    ('sigma = 2.0 * mu[:, None, None] * eps', 'sigma = 1.0 * mu[:, None, None] * eps'),
    ('lam = kappa - 2.0 * mu / 3.0', 'lam = kappa'),
    ('+ np.einsum("j,i,l,lk,eclji->eckji", w, w, w, H, t[:, 2]))',
     '- np.einsum("j,i,l,lk,eclji->eckji", w, w, w, H, t[:, 2]))'),
    ('np.einsum("ecdkji,erdkji->erckji", sigma, dxi_dx)', 'np.einsum("ecdkji,edrkji->erckji", sigma, dxi_dx)'),
]


def _mutant(oracle, old, new):
    src = inspect.getsource(oracle.element_forces)
    assert old in src, old
    ns = dict(oracle.__dict__)
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    return ns["element_forces"]


def _pins(oracle):
    """Cheap pins from test_oracle_operator, returned as a list of booleans."""
    from tests.test_oracle_operator import _dense_element_stiffness
    ok = []
    mesh = inputs.structured_hex_mesh(3, 3, 900.0, jitter=0.2, seed=5)
    shape = mesh.ibool.shape
    rho = inputs.uniform(3, shape, 2000.0, 3000.0, stream=1).astype(np.float32)
    vp = inputs.uniform(3, shape, 3000.0, 5000.0, stream=2).astype(np.float32)
    vs = (vp / 1.8).astype(np.float32)
    m = oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, rho, vp, vs, mesh.ngll)
    X = m.node_xyz
    u = np.cross([0.4, -0.25, 0.9], X - X.mean(axis=0))
    r = inputs.random_field(m.nglob, 9).astype(np.float64)
    v = inputs.random_field(m.nglob, 8).astype(np.float64)
    Kr = -m.forces(r)
    scale = np.linalg.norm(Kr) / np.linalg.norm(r)
    ok.append(np.linalg.norm(m.forces(u)) <= 1e-12 * scale * np.linalg.norm(u))
    ok.append(abs(np.sum(v * Kr) + np.sum(r * m.forces(v))) <= 1e-12 * abs(np.sum(r * Kr)))
    e = 13
    n = mesh.ngll
    K = _dense_element_stiffness(oracle, mesh.ctrl[e], rho[e], vp[e], vs[e], n)
    ue = inputs.uniform(5, (3, n ** 3), -1, 1)
    Fe = oracle.element_forces(ue.reshape(1, 3, n, n, n), m.dxi_dx[e:e + 1], m.jac[e:e + 1],
                               m.kappa[e:e + 1], m.mu[e:e + 1], m.basis)
    ok.append(np.allclose(Fe.reshape(-1), -(K @ ue.reshape(-1)), rtol=0,
                          atol=1e-12 * np.abs(K @ ue.reshape(-1)).max()))
    return ok


def test_pins_pass_on_the_oracle(oracle):
    assert all(_pins(oracle))


@pytest.mark.parametrize("old,new", MUTATIONS)
def test_planted_mistake_is_caught(oracle, monkeypatch, old, new):
    monkeypatch.setattr(oracle, "element_forces", _mutant(oracle, old, new))
    assert not all(_pins(oracle))
