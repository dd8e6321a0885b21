"""CPU checks of the C-ABI library: it loads, exports every declared symbol, and its
host-side mesh/DoF/constraint tables match the oracle bit-exactly (no GPU needed)."""
import os
import re

import numpy as np
import pytest

from oracle import mesh as omesh
from paper_1910_13247_gb300 import build as mbuild
from paper_1910_13247_gb300 import mfx, synthetic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    mbuild.build()
    mfx.lib()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(mfx_[a-z0-9_]+)\s*\(", src, re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert len(names) >= 20
    L = mfx.lib()
    for n in names:
        assert hasattr(L, n), n


def test_version_and_error_strings():
    assert b"sm_103a" in mfx.lib().mfx_version()
    with pytest.raises(mfx.MfxError) as e:
        mfx.Mesh.structured_box(0, 1, 1)
    assert e.value.code == mfx.EINVAL


@pytest.mark.parametrize("k", range(1, 9))
def test_structured_tables_bit_exact(k):
    nx, ny, nz = 3, 2, 4
    T = mfx.Mesh.structured_box(nx, ny, nz).tables(k)
    om = omesh.structured_mesh(nx, ny, nz, k)
    assert T["n_dofs"] == om.n_dofs
    assert np.array_equal(T["cell_dofs"], om.cell_dofs)
    assert np.array_equal(T["constrained"], om.constrained)
    assert np.array_equal(T["cptr"], om.cptr)


# octrees: (seed, coarse cells per direction, refinement levels, ball centre or None = seeded, radius or None)
OCTREES = {
    "seeded4x2a": (0, 4, 2, None, None), "seeded4x2b": (1, 4, 2, None, None), "seeded3x1": (2, 3, 1, None, None),
    "seeded4x3": (3, 4, 3, None, None),
    # small meshes that the oracle tabulates in seconds at every degree
    "seeded2x2": (5, 2, 2, None, 0.3),
    # three levels (leaves on levels 0..3): a ball around nested cell centres of levels 0, 1 and 2
    "nested2x3": (0, 2, 3, (0.3125, 0.3125, 0.3125), 0.12),
}
OCTREE_CASES = ([(k, c) for k in range(1, 6) for c in ("seeded4x2a", "seeded4x2b", "seeded3x1")] +
                [(k, "seeded4x3") for k in (1, 2, 3)] + [(k, "seeded2x2") for k in (6, 7, 8)] +
                [(k, "nested2x3") for k in range(1, 9)])


def octree_case(name):
    seed, nb, levels, centre, radius = OCTREES[name]
    g = synthetic.rng(100 + seed)
    c, r = g.uniform(0.25, 0.75, 3), float(g.uniform(0.15, 0.35))
    leaves = synthetic.octree_leaves(nb, levels, np.asarray(centre) if centre else c, radius if radius else r)
    return nb, leaves


@pytest.mark.parametrize("k,case", OCTREE_CASES)
def test_octree_tables_bit_exact(k, case):
    """DoF numbering, constrained DoFs, constraint rows, masters and weights of octree meshes (1-3 levels of
    refinement, hanging faces and edges, Dirichlet faces) equal the oracle's bit for bit at every degree."""
    nb, leaves = octree_case(case)
    if case == "nested2x3":
        assert set(leaves[:, 0]) == {0, 1, 2, 3}
    T = mfx.Mesh.octree(nb, nb, nb, leaves).tables(k)
    om = omesh.octree_mesh(nb, nb, nb, k, leaves)
    assert T["n_dofs"] == om.n_dofs
    assert np.array_equal(T["cell_dofs"], om.cell_dofs)
    assert np.array_equal(T["constrained"], om.constrained)
    assert np.array_equal(T["cptr"], om.cptr)
    assert np.array_equal(T["cmaster"], om.cmaster)
    # weights: same product formula in the same order on both sides
    assert np.array_equal(T["cweight"], om.cweight)


def test_octree_cell_order_matches_oracle_for_shuffled_leaves():
    leaves = synthetic.octree_leaves(3, 2, (0.5, 0.4, 0.6), 0.3)
    perm = np.random.default_rng(0).permutation(len(leaves))
    T = mfx.Mesh.octree(3, 3, 3, leaves[perm]).tables(2)
    om = omesh.octree_mesh(3, 3, 3, 2, leaves)
    assert np.array_equal(T["cell_dofs"], om.cell_dofs)


def test_invalid_octrees_rejected_with_emesh():
    good = synthetic.octree_leaves(2, 1, (0.25, 0.25, 0.25), 0.1)
    mfx.Mesh.octree(2, 2, 2, good)
    cases = {
        "hole": good[1:],
        "overlap": np.vstack([good, [[0, 1, 1, 1]]]),
        "duplicate": np.vstack([good, good[:1]]),
        "out of range": np.vstack([good[:-1], [[0, 2, 1, 1]]]),
    }
    # level-2 leaves next to a level-0 leaf
    unbalanced = [lf for lf in good.tolist() if not (lf[0] == 1 and lf[1:] == [1, 0, 0])]
    unbalanced += [[2, 2 + a, b, c] for c in (0, 1) for b in (0, 1) for a in (0, 1)]
    cases["unbalanced"] = np.array(unbalanced)
    for name, lv in cases.items():
        with pytest.raises(mfx.MfxError) as e:
            mfx.Mesh.octree(2, 2, 2, lv)
        assert e.value.code in (mfx.EMESH, mfx.EINVAL), name
    with pytest.raises(omesh.MeshError):
        omesh.octree_mesh(2, 2, 2, 1, cases["unbalanced"])


def test_bad_degree_rejected():
    m = mfx.Mesh.structured_box(2, 2, 2)
    with pytest.raises(mfx.MfxError) as e:
        m.tables(9)
    assert e.value.code == mfx.EUNSUPPORTED


@pytest.mark.parametrize("faces", [0, 0b000011, 0b110100, 0b101010])
def test_tables_with_dirichlet_face_masks_bit_exact(faces):
    """Dirichlet on a subset of the box faces: the constrained set and the hanging constraints (masters
    on natural faces kept, masters on Dirichlet faces dropped) match the oracle bit for bit."""
    T = mfx.Mesh.structured_box(4, 3, 2, dirichlet=faces).tables(2)
    om = omesh.structured_mesh(4, 3, 2, 2, dirichlet=faces)
    assert np.array_equal(T["constrained"], om.constrained) and np.array_equal(T["cell_dofs"], om.cell_dofs)
    # closed form: lattice points on no Dirichlet face
    Mx, My, Mz = 9, 7, 5
    free = 1
    for M, b in ((Mx, 0), (My, 2), (Mz, 4)):
        free *= M - (faces >> b & 1) - (faces >> (b + 1) & 1)
    assert len(T["constrained"]) == Mx * My * Mz - free
    # the refined ball touches the x = 0 and y = 0 faces of the box
    leaves = synthetic.octree_leaves(3, 2, np.array([0.15, 0.2, 0.5]), 0.3)
    for k in (1, 3):
        T = mfx.Mesh.octree(3, 3, 3, leaves, dirichlet=faces).tables(k)
        om = omesh.octree_mesh(3, 3, 3, k, leaves, dirichlet=faces)
        assert T["n_dofs"] == om.n_dofs
        assert np.array_equal(T["constrained"], om.constrained)
        assert np.array_equal(T["cptr"], om.cptr)
        assert np.array_equal(T["cmaster"], om.cmaster)
        assert np.array_equal(T["cweight"], om.cweight)
    with pytest.raises(mfx.MfxError):
        mfx.Mesh.structured_box(2, 2, 2, dirichlet=64)


def test_host_exceptions_become_status_codes():
    """A host-side failure inside an entry point (here a lattice too large to allocate) is returned as a
    status code with a message; no C++ exception crosses the C-ABI and the library stays usable."""
    with pytest.raises(mfx.MfxError) as e:
        mfx.Mesh.structured_box(1 << 20, 1 << 20, 1 << 20)
    assert e.value.code in (mfx.EINVAL, mfx.ENOMEM)
    assert mfx.Mesh.structured_box(2, 2, 2).tables(1)["n_dofs"] == 27
