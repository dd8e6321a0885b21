"""Pins of the oracle's octree meshes: numbering, hanging-node constraints, validation.

Hanging nodes arise from local refinement (Sec. 3.1, Sec. 3.3, Fig. 2); the
constraint values are fixed by continuity of the Q_k space.  The pins use
facts the mathematics fixes: a uniformly refined octree is the structured
mesh up to a renumbering; Q1 constraints have weights 1/2 (edge midpoints)
and 1/4 (face centres); constraints reproduce every global polynomial of
degree <= k; and the condensed operator gives the exact energy of conforming
polynomials.
"""
import numpy as np
import pytest

from oracle import fem, mesh, rules
from paper_1910_13247_gb300 import synthetic


def node_positions(m):
    """Physical position of every DoF, from the cells' trilinear maps at GLL points."""
    k = m.k
    n = k + 1
    g = rules.gauss_lobatto(k)
    pos = np.zeros((m.n_dofs, 3))
    for c in range(m.n_cells):
        V = m.cell_vertices[c]
        for a3 in range(n):
            for a2 in range(n):
                for a1 in range(n):
                    s, t, u = g[a1], g[a2], g[a3]
                    p = np.zeros(3)
                    for v in range(8):
                        a, b, e = v & 1, (v >> 1) & 1, (v >> 2) & 1
                        p += (s if a else 1 - s) * (t if b else 1 - t) * (u if e else 1 - u) * V[v]
                    pos[m.cell_dofs[c, a1 + n * (a2 + n * a3)]] = p
    return pos


def small_octree(nb=2, refine=((0, 0, 0),), extra=()):
    """Coarse nb^3 grid; listed coarse cells refined once; `extra` level-1 cells refined again."""
    leaves = []
    for l in range(nb):
        for j in range(nb):
            for i in range(nb):
                if (i, j, l) in refine:
                    for c in range(2):
                        for b in range(2):
                            for a in range(2):
                                ch = (2 * i + a, 2 * j + b, 2 * l + c)
                                if ch in extra:
                                    for cc in range(2):
                                        for bb in range(2):
                                            for aa in range(2):
                                                leaves.append((2, 2 * ch[0] + aa, 2 * ch[1] + bb, 2 * ch[2] + cc))
                                else:
                                    leaves.append((1,) + ch)
                else:
                    leaves.append((0, i, j, l))
    return np.array(leaves)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_uniform_octree_equals_structured_mesh(k):
    leaves = [(1, i, j, l) for l in range(4) for j in range(4) for i in range(4)]
    mo = mesh.octree_mesh(2, 2, 2, k, leaves)
    ms = mesh.structured_mesh(4, 4, 4, k)
    assert mo.n_dofs == ms.n_dofs and len(mo.cmaster) == 0
    assert len(mo.constrained) == len(ms.constrained)
    po, ps = node_positions(mo), node_positions(ms)
    # permutation between the two numberings by exact node position
    key = lambda p: tuple(np.round(p * 1e9).astype(np.int64))
    idx = {key(p): i for i, p in enumerate(ps)}
    perm = np.array([idx[key(p)] for p in po])
    assert sorted(perm) == list(range(ms.n_dofs))
    Ko = fem.assemble(mo, k + 1).toarray()
    Ks = fem.assemble(ms, k + 1).toarray()
    assert np.allclose(Ko, Ks[np.ix_(perm, perm)], atol=1e-13)


def test_q1_hanging_weights_are_halves_and_quarters():
    m = mesh.octree_mesh(3, 3, 3, 1, small_octree(3, refine=((1, 1, 1),)))
    hang = [t for t in range(len(m.constrained)) if m.cptr[t + 1] > m.cptr[t]]
    assert hang
    seen = set()
    for t in hang:
        w = sorted(m.cweight[m.cptr[t]:m.cptr[t + 1]])
        assert w in ([0.5, 0.5], [0.25, 0.25, 0.25, 0.25]), w
        seen.add(len(w))
    assert seen == {2, 4}


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_constraints_reproduce_polynomials(k):
    leaves = synthetic.octree_leaves(4, 2, (0.45, 0.5, 0.55), 0.3)
    m = mesh.octree_mesh(4, 4, 4, k, leaves)
    assert len(m.cmaster) > 0
    pos = node_positions(m)
    x, y, z = pos.T
    # a polynomial of degree <= k in each variable that vanishes on the boundary where k >= 2;
    # for k = 1 a general trilinear function (checked away from Dirichlet masters)
    if k >= 2:
        u = x * (1 - x) * y * (1 - y) * z * (1 - z) * (1 + (x - 0.3) ** (k - 2))
    else:
        u = 1 + 2 * x - 3 * y + 0.5 * z + x * y * z
    checked = 0
    for t, dof in enumerate(m.constrained):
        lo, hi = m.cptr[t], m.cptr[t + 1]
        if hi == lo:
            continue
        masters = m.cmaster[lo:hi]
        w = m.cweight[lo:hi]
        # for k = 1, u does not vanish on the boundary: use rows whose Dirichlet masters
        # were not dropped (their weights sum to one: partition of unity)
        if k == 1 and abs(w.sum() - 1.0) > 1e-14:
            continue
        checked += 1
        val = float(np.dot(w, u[masters]))
        assert abs(val - u[dof]) < 1e-13, (dof, val, u[dof])
    assert checked > 10


@pytest.mark.parametrize("k", [2, 3])
def test_condensed_energy_of_conforming_polynomial_is_exact(k):
    # u = x(1-x) y(1-y) z(1-z) lies in the conforming Q_k space (k >= 2) and vanishes on the
    # boundary; with constant coefficient a = 1 its energy is 3 * (1/3) * (1/30)^2 = 1/900
    leaves = synthetic.octree_leaves(4, 2, (0.4, 0.6, 0.5), 0.35)
    m = mesh.octree_mesh(4, 4, 4, k, leaves)
    pos = node_positions(m)
    x, y, z = pos.T
    u = x * (1 - x) * y * (1 - y) * z * (1 - z)
    u[m.constrained] = 0.0
    K = fem.assemble(m, k + 1)
    assert abs(u @ (K @ u) - 1.0 / 900.0) < 1e-13
    # and distributing the free values recovers the interpolant at the hanging nodes
    full = fem.distribute(m, u)
    assert np.allclose(full, x * (1 - x) * y * (1 - y) * z * (1 - z), atol=1e-14)


def test_octree_order_and_first_encounter_numbering():
    m = mesh.octree_mesh(2, 2, 2, 2, small_octree(2))
    # the first cell is the first Morton child of coarse cell (0,0,0); its nodes get DoFs 0..26
    assert list(m.cell_dofs[0]) == list(range(27))
    # every DoF number appears, and first appearances are increasing in cell/local order
    seen = []
    for row in m.cell_dofs:
        for d in row:
            if d not in seen:
                seen.append(d)
    assert seen == list(range(m.n_dofs))


def test_invalid_octrees_are_rejected():
    good = small_octree(2)
    mesh.octree_mesh(2, 2, 2, 1, good)
    with pytest.raises(mesh.MeshError):
        mesh.octree_mesh(2, 2, 2, 1, good[1:])                      # hole
    with pytest.raises(mesh.MeshError):
        mesh.octree_mesh(2, 2, 2, 1, np.vstack([good, [[0, 1, 1, 1]]]))  # overlap
    # level-2 cells next to a level-0 cell across a face
    bad = small_octree(2, refine=((0, 0, 0),), extra=((1, 0, 0),))
    with pytest.raises(mesh.MeshError):
        mesh.octree_mesh(2, 2, 2, 1, bad)
    # across an edge only: refine the child touching the edge shared with the diagonal coarse cell
    bad_edge = small_octree(2, refine=((0, 0, 0),), extra=((1, 1, 0),))
    with pytest.raises(mesh.MeshError):
        mesh.octree_mesh(2, 2, 2, 1, bad_edge)


def test_octree_manufactured_solution_converges():
    errs = []
    for nb in (2, 4):
        leaves = synthetic.octree_leaves(nb, 1, (0.5, 0.5, 0.5), 0.3)
        m = mesh.octree_mesh(nb, nb, nb, 2, leaves)
        K = fem.assemble(m, 3)
        b = fem.rhs(m, 3)
        import scipy.sparse.linalg as spla
        errs.append(fem.l2_error(m, spla.spsolve(K.tocsc(), b)))
    assert errs[1] < errs[0] / 5
