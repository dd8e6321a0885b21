"""CPU check of the premise of the k = 1 octant vmult: on the library's own cell order, a window of eight
consecutive cells passes the kernel's index-table rule (every node position of the 3 x 3 x 3 block gets
one entry, child c at (c & 1, (c >> 1) & 1, c >> 2)) exactly when the eight cells are the children of one
octant (found here from the oracle's cell geometry, independently of the tables), and passing windows
never overlap.  No GPU needed: the tables come from the library's host builder."""
import numpy as np
import pytest

from oracle import mesh as omesh
from paper_1910_13247_gb300 import build as mbuild
from paper_1910_13247_gb300 import mfx, synthetic


@pytest.fixture(scope="module", autouse=True)
def _built():
    mbuild.build()
    mfx.lib()


def octant_pos(c, n):
    return ((c & 1) + (n & 1)) + 3 * (((c >> 1) & 1) + ((n >> 1) & 1)) + 9 * ((c >> 2) + (n >> 2))


def window_passes(cd, i):
    """The rule of the set-up kernel: the eight cells' entries agree wherever two meet one position."""
    slot = {}
    for c in range(8):
        for n in range(8):
            p = octant_pos(c, n)
            v = int(cd[i + c, n])
            if slot.setdefault(p, v) != v:
                return False
    return True


def sibling_group(cv, i):
    """Cells i .. i + 7 are the eight children of one octant, child c at offset (c & 1, (c >> 1) & 1,
    c >> 2) times the children's size, the parent's corner on the parent's lattice."""
    lo = cv[i:i + 8, 0, :]
    size = cv[i:i + 8, 7, :] - lo
    h = size[0]
    if not np.allclose(size, h, rtol=0, atol=1e-12):
        return False
    corner = lo[0]
    if not np.allclose(np.round(corner / (2 * h)) * (2 * h), corner, rtol=0, atol=1e-9):
        return False
    for c in range(8):
        off = np.array([c & 1, (c >> 1) & 1, c >> 2], dtype=np.float64) * h
        if not np.allclose(lo[c], corner + off, rtol=0, atol=1e-12):
            return False
    return True


@pytest.mark.parametrize("nb,levels,center,radius", [(4, 1, (0.5, 0.5, 0.5), 0.3), (3, 2, (0.3, 0.6, 0.5), 0.3),
                                                     (2, 3, (0.25, 0.25, 0.75), 0.2), (5, 2, (0.7, 0.4, 0.3), 0.25)])
def test_octant_windows_are_the_sibling_groups(nb, levels, center, radius):
    leaves = synthetic.octree_leaves(nb, levels, np.array(center), radius)
    mesh = mfx.Mesh.octree(nb, nb, nb, leaves)
    cd = mesh.tables(1)["cell_dofs"]
    om = omesh.octree_mesh(nb, nb, nb, 1, leaves)
    C = cd.shape[0]
    assert om.cell_vertices.shape[0] == C
    passing = [i for i in range(C - 7) if window_passes(cd, i)]
    siblings = [i for i in range(C - 7) if sibling_group(om.cell_vertices, i)]
    assert passing == siblings
    assert len(passing) > 0
    assert all(b - a >= 8 for a, b in zip(passing, passing[1:]))
