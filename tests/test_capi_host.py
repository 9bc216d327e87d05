"""CPU-side checks of the C ABI library: it builds and loads without a GPU, exports every
symbol ``include/sem.h`` declares, and its host-only set-up (GLL basis, colouring,
argument validation) agrees with the oracle and with the colouring invariant of Sec. IV-C.
No call here launches GPU work."""
import os
import re

import numpy as np
import pytest

from paper_2606_12850_gb300 import build, inputs, sem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def library():
    build.build()
    return sem.lib()


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "sem.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sem_[a-z_]+)\s*\(", text)))


def test_header_symbols_exported_and_bound():
    declared = _declared_symbols()
    assert len(declared) >= 20
    lib = sem.lib()
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(sem.SIGNATURES) == declared


def test_surrogate_header_symbols_exported_and_bound():
    from paper_2606_12850_gb300 import surrogate
    text = open(os.path.join(ROOT, "include", "surrogate.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    declared = sorted(set(re.findall(r"\b(sg_[a-z_]+)\s*\(", text)))
    assert len(declared) >= 10
    lib = surrogate.lib()
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(surrogate.SIGNATURES) == declared


def test_surrogate_spec_sizes():
    """The default network: 9 -> 512 -> 512 -> [64][125], decoder to 6 x 192 x 1000,
    combined with the six moment entries into 192 x 1000."""
    from paper_2606_12850_gb300 import surrogate
    spec = surrogate.Spec()
    assert (spec.out_c, spec.out_l) == (192, 1000)
    n = sum(int(np.prod(s)) for _, s in spec.shapes())
    assert n == 9 * 512 + 512 + 512 * 512 + 512 + 512 * 8000 + 8000 + (96 * 64 * 3 + 96) + 2 * (96 * 96 * 3 + 96) \
        + (1152 * 96 * 3 + 1152)
    flat = spec.init_params(1)
    parts = spec.split(flat)
    assert np.all(parts["b1"] == 0) and np.abs(parts["W1"]).max() <= np.sqrt(6 / 9)


def test_surrogate_sources_are_unit_moments():
    pos, m = inputs.surrogate_sources(2000, 4000.0, seed=3)
    assert pos.min() >= 200.0 and pos.max() <= 3800.0
    np.testing.assert_allclose(np.linalg.norm(m, axis=1), 1.0, rtol=0, atol=1e-12)
    z = inputs.normal(5, (200000,))
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_version():
    assert sem.sem_version() >= 100


@pytest.mark.parametrize("ngll", range(2, 11))
def test_gll_matches_oracle(oracle, ngll):
    """Library GLL basis (Newton on (1-x^2) P_N', closed-form derivative matrix) equals the
    oracle's (Newton on P_N', product-formula derivative matrix)."""
    xi, w, h = sem.sem_gll(ngll)
    b = oracle.Basis(ngll)
    np.testing.assert_allclose(xi, b.xi, atol=2e-16)
    np.testing.assert_allclose(w, b.w, rtol=1e-14)
    np.testing.assert_allclose(h, b.hprime, atol=1e-12 * ngll ** 2)


def test_gll_rejects_bad_order():
    for n in (1, 11, 0, -3):
        with pytest.raises(sem.SemError) as ei:
            sem.sem_gll(n)
        assert ei.value.code == -1


@pytest.mark.parametrize("ngll", [2, 3, 5, 7, 10])
def test_geometry_matches_oracle(oracle, ngll):
    """Library geometry (GLL positions differentiated with hprime, inverse by cofactors)
    equals the oracle's (analytic derivatives of the trilinear map, numpy inverse and
    determinant) on a strongly jittered mesh, in double precision."""
    mesh = inputs.structured_hex_mesh(3, ngll, 1000.0, jitter=0.2, seed=11)
    xyz, g, jac = sem.sem_geometry(mesh.ctrl, ngll)
    ox, og, oj = oracle.element_geometry(mesh.ctrl, oracle.Basis(ngll))
    nspec = mesh.nspec
    ox = ox.reshape(nspec, 3, -1).transpose(0, 2, 1)
    og = og.reshape(nspec, 3, 3, -1).transpose(0, 3, 1, 2)
    oj = oj.reshape(nspec, -1)
    for lib_v, ora_v in ((xyz, ox), (g, og), (jac, oj)):
        assert np.abs(lib_v - ora_v).max() <= 1e-12 * np.abs(ora_v).max()


def test_geometry_regular_lattice_closed_form():
    """On a regular lattice of spacing h: d xi / d x = 2/h on the diagonal, 0 elsewhere,
    J = (h/2)^3 at every point, and the GLL points of an edge are h/2 (1 + xi) apart from
    its first corner."""
    h = 250.0
    mesh = inputs.structured_hex_mesh(2, 4, 2 * h)
    xyz, g, jac = sem.sem_geometry(mesh.ctrl, 4)
    np.testing.assert_allclose(g, np.broadcast_to(np.eye(3) * 2 / h, g.shape), rtol=0, atol=1e-15)
    np.testing.assert_allclose(jac, (h / 2) ** 3, rtol=1e-13)
    xi, _, _ = sem.sem_gll(4)
    e0 = xyz[0].reshape(4, 4, 4, 3)
    np.testing.assert_allclose(e0[0, 0, :, 0] - mesh.ctrl[0, 0, 0], h / 2 * (1 + xi), rtol=0, atol=1e-12)


def test_geometry_rejects_inverted_and_non_finite():
    mesh = inputs.structured_hex_mesh(2, 3, 1.0)
    ctrl = mesh.ctrl.copy()
    ctrl[5] = ctrl[5][[1, 0, 3, 2, 5, 4, 7, 6]]  # mirror element 5 in x: J < 0
    with pytest.raises(sem.SemError) as ei:
        sem.sem_geometry(ctrl, 3)
    assert ei.value.code == -1 and "element 5" in str(ei.value)
    ctrl = mesh.ctrl.copy()
    ctrl[2, 3, 1] = np.nan
    with pytest.raises(sem.SemError, match="non-finite"):
        sem.sem_geometry(ctrl, 3)


def _trilinear_point(X, ref):
    x = np.zeros(3)
    for c in range(8):
        sa, sb, sd = (1 if c & 1 else -1), (1 if c & 2 else -1), (1 if c & 4 else -1)
        x += (1 + sa * ref[0]) * (1 + sb * ref[1]) * (1 + sd * ref[2]) / 8.0 * X[c]
    return x


@pytest.fixture(scope="module")
def jittered(oracle):
    mesh = inputs.structured_hex_mesh(3, 5, 900.0, jitter=0.2, seed=11)
    ones = np.ones(mesh.ibool.shape)
    return mesh, oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, 2500 * ones, 4000 * ones, 2300 * ones, 5)


def test_locate_points_matches_oracle(oracle, jittered):
    """Library point location (Newton on the trilinear map in C++) equals the oracle's:
    same element (lowest index on shared faces) and reference coordinates within 1e-12;
    points outside the mesh get -1."""
    mesh, m = jittered
    pts = [_trilinear_point(mesh.ctrl[e], inputs.uniform(7 + e, (3,), -0.99, 0.99)) for e in range(mesh.nspec)]
    pts += [_trilinear_point(mesh.ctrl[13], np.array([-1.0, 0.2, 0.4])), m.node_xyz[17]]
    pts += list(inputs.uniform(3, (10, 3), 0.0, 900.0))
    elem, ref = sem.sem_locate_points(mesh.ctrl, np.array(pts))
    for x, e, r in zip(pts, elem, ref):
        e2, r2 = oracle.locate_point(m, x)
        assert e == e2
        np.testing.assert_allclose(r, r2, rtol=0, atol=1e-12)
    elem, _ = sem.sem_locate_points(mesh.ctrl, [[-5.0, 100.0, 100.0], [100.0, 100.0, 901.0]])
    assert list(elem) == [-1, -1]


def test_locate_points_buckets_equal_the_element_scan(oracle):
    """Many points on a larger mesh go through the bucket grid; the result equals the plain
    scan over all elements (one point per call) and the oracle, including points on the
    vertices, edges and faces that several elements share (lowest index) and points outside."""
    mesh = inputs.structured_hex_mesh(6, 2, 1200.0, jitter=0.2, seed=4)
    ones = np.ones(mesh.ibool.shape)
    m = oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, ones, 2 * ones, ones, 2)
    pts = list(inputs.uniform(21, (300, 3), -20.0, 1220.0))
    pts += [mesh.ctrl[e, c] for e in (43, 86, 129) for c in range(8)]  # vertices shared by up to 8
    pts += [0.5 * (mesh.ctrl[100, 0] + mesh.ctrl[100, 7])]  # element centre
    pts += [0.5 * (mesh.ctrl[100, 1] + mesh.ctrl[100, 7])]  # on a face
    pts = np.array(pts)
    elem, ref = sem.sem_locate_points(mesh.ctrl, pts)
    assert (elem >= 0).sum() > 200 and (elem < 0).sum() > 0
    for q in range(len(pts)):
        e1, r1 = sem.sem_locate_points(mesh.ctrl, pts[q:q + 1])
        assert e1[0] == elem[q]
        np.testing.assert_array_equal(r1[0], ref[q])
    for q in range(0, len(pts), 7):
        if elem[q] >= 0:
            e2, r2 = oracle.locate_point(m, pts[q])
            assert e2 == elem[q]
            np.testing.assert_allclose(ref[q], r2, rtol=0, atol=1e-12)
        else:
            with pytest.raises(ValueError):
                oracle.locate_point(m, pts[q])


@pytest.mark.parametrize("kind", ["force", "moment"])
@pytest.mark.parametrize("ngll", [2, 5, 8])
def test_point_source_forces_match_oracle(oracle, kind, ngll):
    """Library interpolated source forces (barycentric Lagrange values, derivatives through
    the nodal derivative matrix) equal the oracle's (product formula and its derivative)
    within 1e-12 of the largest force, at random points, a face and a node."""
    mesh = inputs.structured_hex_mesh(3, ngll, 900.0, jitter=0.2, seed=11)
    ones = np.ones(mesh.ibool.shape)
    m = oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, 2500 * ones, 4000 * ones, 2300 * ones, ngll)
    value = np.array([0.3, -1.2, 2.0]) if kind == "force" else inputs.uniform(5, (6,), -1.0, 1.0, stream=9)
    refs = [inputs.uniform(50 + q, (3,), -0.95, 0.95) for q in range(3)] + [np.array([1.0, -0.3, 0.5])]
    pts = [_trilinear_point(mesh.ctrl[13], r) for r in refs] + [m.node_xyz[int(mesh.ibool[13, ngll])]]
    for x in pts:
        e, ref, nodes, f = oracle.point_source_forces(m, x, **{kind: value})
        lib_f = sem.sem_point_source_forces(ngll, mesh.ctrl[e], ref, **{kind: value})
        dense_lib = np.zeros((mesh.nglob, 3))
        np.add.at(dense_lib, mesh.ibool[e], lib_f)
        dense_ora = np.zeros((mesh.nglob, 3))
        np.add.at(dense_ora, nodes, f)
        np.testing.assert_allclose(dense_lib, dense_ora, rtol=0, atol=1e-12 * np.abs(dense_ora).max())


def test_point_source_forces_reject_bad_arguments():
    ctrl = inputs.structured_hex_mesh(1, 3, 1.0).ctrl[0]
    with pytest.raises(sem.SemError):
        sem.sem_point_source_forces(3, ctrl, [0.0, 0.0, 0.0])  # neither force nor moment
    with pytest.raises(sem.SemError):
        sem.sem_point_source_forces(3, ctrl, [0.0, 0.0, 0.0], force=[1, 0, 0], moment=np.ones(6))
    with pytest.raises(sem.SemError):
        sem.sem_point_source_forces(3, ctrl, [1.5, 0.0, 0.0], force=[1, 0, 0])


def _check_coloring(ibool, color, ncolors):
    assert color.min() == 0 and color.max() == ncolors - 1
    for c in range(ncolors):
        nodes = ibool[color == c].reshape(-1)
        assert len(np.unique(nodes)) == nodes.size, f"colour {c} shares a node"


@pytest.mark.parametrize("n,ngll,jitter,periodic,expect", [
    (8, 5, 0.0, False, 8),
    (5, 3, 0.1, False, 8),
    ((3, 4, 5), 4, 0.0, False, 8),
    (4, 2, 0.0, True, 8),
    (1, 5, 0.0, False, 1),
    ((7, 1, 1), 6, 0.0, False, 2),
])
def test_coloring_valid(n, ngll, jitter, periodic, expect):
    """Sec. IV-C: within a colour no two elements share a node; a structured lattice gets
    the 8-colour parity pattern (2 for a line of elements, 1 for a single element)."""
    mesh = inputs.structured_hex_mesh(n, ngll, 1000.0, jitter=jitter, periodic=periodic)
    color, nc = sem.sem_color_elements(mesh.ibool, ngll, mesh.nglob)
    _check_coloring(mesh.ibool, color, nc)
    assert nc == expect


def test_coloring_periodic_odd():
    """A periodic lattice with an odd element count cannot use the parity pattern; the
    greedy colouring still yields a valid colouring."""
    mesh = inputs.structured_hex_mesh(3, 3, 1.0, periodic=True)
    color, nc = sem.sem_color_elements(mesh.ibool, 3, mesh.nglob)
    _check_coloring(mesh.ibool, color, nc)
    assert nc == 27  # every pair of the 27 elements shares a node


def test_coloring_rejects_repeated_node():
    """A periodic line of a single element repeats its own nodes: rejected (its own
    scatter would race)."""
    mesh = inputs.structured_hex_mesh((1, 2, 2), 3, 1.0, periodic=True)
    with pytest.raises(sem.SemError) as ei:
        sem.sem_color_elements(mesh.ibool, 3, mesh.nglob)
    assert ei.value.code == -1 and "repeats node" in str(ei.value)


def test_coloring_rejects_out_of_range():
    mesh = inputs.structured_hex_mesh(2, 3, 1.0)
    bad = mesh.ibool.copy()
    bad[1, 4] = mesh.nglob
    with pytest.raises(sem.SemError):
        sem.sem_color_elements(bad, 3, mesh.nglob)


def test_binding_checks_array_sizes():
    """The binding refuses arrays whose size does not match the declared layout before the
    library reads them."""
    mesh = inputs.structured_hex_mesh(2, 3, 1.0)
    with pytest.raises(ValueError):
        sem.sem_color_elements(mesh.ibool.reshape(-1)[:-1], 3, mesh.nglob)
    with pytest.raises(ValueError):
        sem.sem_geometry(mesh.ctrl.reshape(-1)[:-2], 3)
    ctx = sem.Ctx(0, 3)  # a null handle: nothing reaches the library
    with pytest.raises(ValueError):
        sem.sem_set_mesh_corners(ctx, mesh.ibool.reshape(-1)[:-1], mesh.ctrl, mesh.nglob)
    with pytest.raises(ValueError):
        sem.sem_set_mesh_corners(ctx, mesh.ibool, mesh.ctrl[:-1], mesh.nglob)


def test_missing_library_fails_loudly(monkeypatch):
    """No CPU fallback: with the library absent, the binding raises."""
    monkeypatch.setattr(sem, "_lib", None)
    monkeypatch.setattr(build, "LIB", "/nonexistent/libsemgb.so")
    with pytest.raises(RuntimeError, match="not built"):
        sem.lib()


def test_create_without_gpu_reports_cuda_error():
    """On a machine without a GPU, creating a context returns SEM_ECUDA, it does not
    crash or fall back to the CPU."""
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        pytest.skip("a GPU is present")
    with pytest.raises(sem.SemError) as ei:
        sem.sem_create(5)
    assert ei.value.code == -3


@pytest.mark.parametrize("ngll", [3, 5, 7])
def test_library_geometry_from_points_matches_oracle(ngll):
    """sem_geometry_points (the isoparametric route of sem_set_mesh) on a bent mesh against the
    oracle's isoparametric_geometry; each side builds its own GLL point positions (library:
    sem_geometry's trilinear points; oracle: its element_geometry) and bends them with the
    same map from the input module."""
    from oracle import sem_oracle as so
    mesh = inputs.structured_hex_mesh((2, 3, 2), ngll, (1.0, 1.5, 0.8), jitter=0.1, seed=3)
    amp = (0.2, 0.1, 0.15)
    lib_xyz, _, _ = sem.sem_geometry(mesh.ctrl, ngll)
    lib_pts = inputs.bent_map(lib_xyz, mesh.lengths, amp)
    G, J = sem.sem_geometry_points(ngll, lib_pts)
    xyz_o, _, _ = so.element_geometry(mesh.ctrl, so.Basis(ngll))
    pts_o = inputs.bent_map(np.moveaxis(xyz_o, 1, 4).reshape(mesh.nspec, -1, 3), mesh.lengths, amp)
    dxi_o, jac_o = so.isoparametric_geometry(np.moveaxis(pts_o.reshape(mesh.nspec, ngll, ngll, ngll, 3), 4, 1),
                                             so.Basis(ngll))
    J_o = jac_o.reshape(mesh.nspec, -1)
    G_o = np.moveaxis(dxi_o.reshape(mesh.nspec, 3, 3, -1), 3, 1)  # [e, p, r, d]
    assert np.max(np.abs(J - J_o)) <= 1e-12 * np.max(np.abs(J_o))
    assert np.max(np.abs(G - G_o)) <= 1e-12 * np.max(np.abs(G_o))
    bad = lib_pts.copy()
    bad[0, 0] = bad[0, -1]  # folds the first element
    with pytest.raises(sem.SemError):
        sem.sem_geometry_points(ngll, bad)


def test_surrogate_argument_errors_before_any_device_call():
    """Host-side checks of the surrogate ABI that fail before any CUDA call: options on a null
    model, an unknown option, and a batch whose sample indices (max_batch x output length)
    reach 2^24, past which the products' float-reciprocal division is not exact."""
    import ctypes

    from paper_2606_12850_gb300 import sem, surrogate
    lib = surrogate.lib()
    val = ctypes.c_int(7)
    assert lib.sg_set_option(None, surrogate.SG_OPT_PRODUCT, 1) == -1
    assert lib.sg_get_option(None, surrogate.SG_OPT_PRODUCT, ctypes.byref(val)) == -1
    assert val.value == 7
    spec = surrogate.Spec()
    co = np.asarray(spec.stage_cout, dtype=np.int32)
    up = np.asarray(spec.stage_up, dtype=np.int32)
    out = ctypes.c_void_p()
    too_big = (1 << 24) // spec.out_l + 1  # max_batch x 1000 samples >= 2^24
    code = lib.sg_create(ctypes.byref(out), 0, None, spec.in_dim, spec.hidden, spec.c0, spec.l0, len(co),
                         co.ctypes.data_as(ctypes.c_void_p), up.ctypes.data_as(ctypes.c_void_p), int(spec.contract),
                         too_big)
    assert code == -1 and out.value is None
    assert b"2^24" in lib.sg_last_error(None)
    with pytest.raises(sem.SemError):
        surrogate.Model(spec, max_batch=too_big)
