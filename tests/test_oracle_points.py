"""Pins of the oracle's geometry from per-point positions (isoparametric_geometry; the route
sem_set_mesh takes), against the analytic trilinear route, an exact volume and the rigid
body null space. CPU only."""
import numpy as np
import pytest

from oracle import sem_oracle as so
from paper_2606_12850_gb300 import inputs


def local_points(xyz):
    """[nspec,3,k,j,i] -> [nspec][ngll^3][3] in local point order p = i + n j + n^2 k."""
    e = xyz.shape[0]
    return np.moveaxis(xyz, 1, 4).reshape(e, -1, 3)


def bent_points(mesh, amplitude):
    """GLL point positions of the lattice elements (trilinear map, oracle basis), bent."""
    xyz, _, _ = so.element_geometry(mesh.ctrl, so.Basis(mesh.ngll))
    return inputs.bent_map(local_points(xyz), mesh.lengths, amplitude)


def model(mesh, points, rho=2500.0):
    one = np.ones(mesh.ibool.shape)
    return so.Model(mesh.ibool, None, mesh.nglob, rho * one, 3000.0 * one, 1700.0 * one, mesh.ngll, points=points)


@pytest.mark.parametrize("ngll", [2, 3, 4, 5, 6])
def test_isoparametric_equals_trilinear(ngll):
    """On trilinear elements (positions from the corners' map) the two routes agree."""
    mesh = inputs.structured_hex_mesh((3, 2, 2), ngll, (3.0, 2.0, 2.5), jitter=0.2, seed=7)
    one = np.ones(mesh.ibool.shape)
    ref = so.Model(mesh.ibool, mesh.ctrl, mesh.nglob, one, 2 * one, one, ngll)
    pts = so.Model(mesh.ibool, None, mesh.nglob, one, 2 * one, one, ngll, points=local_points(ref.xyz))
    assert np.max(np.abs(pts.jac - ref.jac)) <= 1e-12 * np.max(np.abs(ref.jac))
    assert np.max(np.abs(pts.dxi_dx - ref.dxi_dx)) <= 1e-12 * np.max(np.abs(ref.dxi_dx))
    assert np.allclose(pts.ctrl, mesh.ctrl, rtol=0, atol=1e-14 * 3)


@pytest.mark.parametrize("ngll", [3, 4, 5, 6])
def test_bent_volume_and_mass_exact(ngll):
    """The bent box has volume (1 + abc) Lx Ly Lz; its map is quadratic per coordinate, so the
    GLL interpolant is exact for N >= 2 and the quadrature of J (degree 1 per reference
    variable per element after the lattice map) is exact: the mass sums to rho times it."""
    L = (2.0, 1.5, 1.0)
    amp = (0.15, 0.10, 0.12)
    mesh = inputs.structured_hex_mesh((3, 2, 2), ngll, L)
    m = model(mesh, bent_points(mesh, amp), rho=2500.0)
    vol = (1 + amp[0] * amp[1] * amp[2]) * np.prod(L)
    w3 = so.quadrature_weights_3d(m.basis)
    assert abs(np.sum(m.jac * w3[None]) - vol) <= 1e-13 * vol
    assert abs(np.sum(m.mass) - 2500.0 * vol) <= 1e-12 * 2500.0 * vol
    assert np.all(m.jac > 0)


def test_bent_rigid_body_null_space():
    """On curved elements translations and infinitesimal rotations still give zero force:
    the discrete derivative of a field linear in the interpolated positions is exact."""
    mesh = inputs.structured_hex_mesh((2, 3, 2), 5, (1.0, 1.2, 0.8))
    m = model(mesh, bent_points(mesh, (0.2, 0.15, 0.1)))
    x = m.node_xyz
    scale = np.linalg.norm(m.forces(inputs.random_field(mesh.nglob, 3)))
    for u in (np.tile([1.0, -2.0, 0.5], (mesh.nglob, 1)), np.cross([0.3, -0.2, 0.7], x)):
        assert np.linalg.norm(m.forces(u)) <= 1e-12 * scale * np.linalg.norm(u) / np.sqrt(mesh.nglob)


def test_transposed_jacobian_slip_is_caught():
    """Planting a transposed inverse Jacobian breaks the rotation pin on curved elements."""
    mesh = inputs.structured_hex_mesh((2, 2, 2), 4, (1.0, 1.0, 1.0))
    m = model(mesh, bent_points(mesh, (0.2, 0.15, 0.1)))
    rot = np.cross([0.3, -0.2, 0.7], m.node_xyz)
    u_e = so.gather(rot, m.ibool, m.ngll)
    bad = np.swapaxes(m.dxi_dx, 1, 2)
    f_bad = so.assemble(so.element_forces(u_e, bad, m.jac, m.kappa, m.mu, m.basis), m.ibool, m.nglob)
    scale = np.linalg.norm(m.forces(inputs.random_field(mesh.nglob, 3)))
    assert np.linalg.norm(f_bad) > 1e-6 * scale
