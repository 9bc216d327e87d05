"""CPU checks of the patch plan the library builds for the force sweep (host only, no GPU):
patches are bricks of the mesh's lattice, their colouring keeps the Sec. IV-C invariant (no
two patches of one colour share a node), and the plan does not depend on the order in
which the caller numbers its elements."""
import numpy as np
import pytest

from paper_2606_12850_gb300 import build, inputs, sem

BRICK = {2: (4, 4, 4), 3: (3, 3, 3), 4: (4, 2, 2), 5: (1, 4, 2), 6: (2, 2, 1), 7: (1, 2, 2), 8: (2, 2, 1),
         9: (3, 1, 1), 10: (2, 1, 1)}


@pytest.fixture(scope="module", autouse=True)
def library():
    build.build()
    return sem.lib()


def colour_valid(ibool, patch_of, color_of):
    """No node is touched by two different patches of the same colour."""
    np_ = ibool.shape[1]
    owner = {}
    for e in range(ibool.shape[0]):
        P = patch_of[e]
        c = color_of[P]
        for g in ibool[e]:
            key = (int(g), int(c))
            if owner.setdefault(key, P) != P:
                return False
    return True


@pytest.mark.parametrize("ngll", [2, 3, 4, 5, 6, 7, 8, 9, 10])
def test_bricks_on_a_lattice(ngll):
    bx, by, bz = BRICK[ngll]
    n = (2 * bx, 2 * by, 2 * bz)
    mesh = inputs.structured_hex_mesh(n, ngll, (1.0, 1.0, 1.0), jitter=0.1)
    patch_of, color_of, info = sem.sem_patch_plan(ngll, mesh.ibool, mesh.nglob)
    assert (info["bx"], info["by"], info["bz"]) == (bx, by, bz)
    assert info["patches"] == 8 and info["colors"] == 8 and info["tables"] == 1
    assert info["max_nodes"] == (bx * (ngll - 1) + 1) * (by * (ngll - 1) + 1) * (bz * (ngll - 1) + 1)
    # every patch is one brick of lattice cells
    ijk = mesh.elem_ijk
    for P in range(info["patches"]):
        cells = ijk[patch_of == P]
        assert len(cells) == bx * by * bz
        lo = cells.min(axis=0)
        assert np.all(lo % np.array([bx, by, bz]) == 0)
        assert np.all(cells.max(axis=0) - lo == np.array([bx - 1, by - 1, bz - 1]))
    assert colour_valid(mesh.ibool, patch_of, color_of)


def test_plan_independent_of_element_numbering():
    mesh = inputs.structured_hex_mesh((6, 4, 5), 5, (3.0, 2.0, 2.5), jitter=0.1)
    p0, c0, i0 = sem.sem_patch_plan(5, mesh.ibool, mesh.nglob)
    perm = np.random.default_rng(4).permutation(mesh.nspec)
    p1, c1, i1 = sem.sem_patch_plan(5, mesh.ibool[perm], mesh.nglob)
    assert i0["patches"] == i1["patches"] == 6 * 1 * 3  # bricks of 1 x 4 x 2 over 6 x 4 x 5
    # the same groups of elements (as sets of lattice cells), whatever their numbering
    groups0 = sorted(tuple(sorted(map(tuple, mesh.elem_ijk[p0 == P]))) for P in range(i0["patches"]))
    ijk1 = mesh.elem_ijk[perm]
    groups1 = sorted(tuple(sorted(map(tuple, ijk1[p1 == P]))) for P in range(i1["patches"]))
    assert groups0 == groups1
    assert colour_valid(mesh.ibool[perm], p1, c1)
    assert colour_valid(mesh.ibool, p0, c0)


def test_ragged_periodic_and_single_element_meshes():
    for n, periodic in (((5, 3, 7), False), ((4, 4, 4), True), ((3, 5, 2), True), ((1, 1, 1), False)):
        mesh = inputs.structured_hex_mesh(n, 5, (1.0, 1.0, 1.0), periodic=periodic)
        patch_of, color_of, info = sem.sem_patch_plan(5, mesh.ibool, mesh.nglob)
        assert colour_valid(mesh.ibool, patch_of, color_of), (n, periodic)
        sizes = np.bincount(patch_of, minlength=info["patches"])
        assert sizes.min() >= 1 and sizes.max() <= 8
        assert info["patches"] >= int(np.ceil(mesh.nspec / 8))
        # colours are numbered in sweep order: patch colours never decrease
        assert np.all(np.diff(color_of) >= 0)


def test_disconnected_components_and_bad_input():
    a = inputs.structured_hex_mesh((2, 2, 2), 3, (1.0, 1.0, 1.0))
    ib = np.concatenate([a.ibool, a.ibool + a.nglob])  # two separate cubes
    patch_of, color_of, info = sem.sem_patch_plan(3, ib, 2 * a.nglob)
    assert colour_valid(ib, patch_of, color_of)
    assert set(patch_of[:8]).isdisjoint(set(patch_of[8:]))
    with pytest.raises(sem.SemError):
        sem.sem_patch_plan(3, np.where(ib == 5, 10 ** 6, ib), 2 * a.nglob)
