"""CPU checks of the tensor-product form of the hanging-node constraints that the octree vmult applies
for k >= 3 (Sec. 3.3, Fig. 2): rebuilt node by node from the library's per-cell face/edge words and
coarse-DoF lists with the GLL Lagrange basis, every constrained node of every cell equals the oracle's
constraint row, and every node that is not constrained is reproduced by its own coarse DoF."""
import itertools

import numpy as np
import pytest

from oracle import mesh as omesh
from oracle import rules
from paper_1910_13247_gb300 import build as mbuild
from paper_1910_13247_gb300 import mfx, synthetic


@pytest.fixture(scope="module", autouse=True)
def _built():
    mbuild.build()
    mfx.lib()


def _axes(d):
    return (1, 2) if d == 0 else ((0, 2) if d == 1 else (0, 1))


def _owner(hf, he, a, k):
    """The first hanging face (f order) that holds local node a, else the first hanging edge."""
    for f in range(6):
        if hf >> f & 1 and a[f >> 1] == (f & 1) * k:
            return "f", f
    for e in range(12):
        if he >> e & 1:
            u, v = _axes(e >> 2)
            if a[u] == (e & 1) * k and a[v] == (e >> 1 & 1) * k:
                return "e", e
    return None


def _tensor_rows(H, n_cells, k):
    """(cell, local node) -> {coarse DoF: weight} for every node on a hanging face or edge."""
    n = k + 1
    x = rules.gauss_lobatto(k)
    # P[c, b, m] = l_m((c + x_b) / 2): the coarse basis at the fine nodes of half c
    P = np.array([[[float(rules.lagrange(x, m, (c + x[b]) / 2)) for m in range(n)] for b in range(n)]
                  for c in range(2)])
    ends = np.append(H["hoff"][1:], len(H["hdofs"]))
    out = {}
    for c in range(n_cells):
        hf, he = int(H["hface"][c]), int(H["hedge"][c])
        off = int(H["hoff"][c])
        faces, edges = {}, {}
        for f in range(6):
            if hf >> f & 1:
                faces[f] = H["hdofs"][off:off + n * n]
                off += n * n
        for e in range(12):
            if he >> e & 1:
                edges[e] = H["hdofs"][off:off + n]
                off += n
        assert off == ends[c]
        if not faces and not edges:
            continue
        for a3, a2, a1 in itertools.product(range(n), repeat=3):
            a = (a1, a2, a3)
            own = _owner(hf, he, a, k)
            if own is None:
                continue
            w = {}
            if own[0] == "f":
                f = own[1]
                u, v = _axes(f >> 1)
                cu, cv = hf >> (6 + 2 * f) & 1, hf >> (7 + 2 * f) & 1
                for mv in range(n):
                    for mu in range(n):
                        dof = int(faces[f][mu + n * mv])
                        if dof >= 0:
                            w[dof] = w.get(dof, 0.0) + P[cu, a[u], mu] * P[cv, a[v], mv]
            else:
                e = own[1]
                d = e >> 2
                cd = he >> (12 + e) & 1
                for md in range(n):
                    dof = int(edges[e][md])
                    if dof >= 0:
                        w[dof] = w.get(dof, 0.0) + P[cd, a[d], md]
            out[(c, a1 + n * (a2 + n * a3))] = w
    return out


def _oracle_rows(om):
    rows = {}
    for i, dof in enumerate(om.constrained):
        lo, hi = om.cptr[i], om.cptr[i + 1]
        rows[int(dof)] = {int(m): float(wt) for m, wt in zip(om.cmaster[lo:hi], om.cweight[lo:hi])}
    return rows


def _same(w, ref, tol=1e-13):
    keys = {m for m, x in w.items() if abs(x) > tol} | set(ref)
    return all(abs(w.get(m, 0.0) - ref.get(m, 0.0)) <= tol for m in keys)


@pytest.mark.parametrize("seed,nb,levels,dirichlet", [(0, 3, 2, 0x3F), (1, 3, 2, 0x3F), (2, 4, 1, 0x3F),
                                                      (3, 3, 2, 0b000011), (4, 3, 2, 0)])
@pytest.mark.parametrize("k", [3, 4, 6])
def test_tensor_product_constraints_equal_oracle_rows(seed, nb, levels, dirichlet, k):
    g = synthetic.rng(300 + seed)
    centre = g.uniform(0.15, 0.6, 3) if dirichlet != 0x3F else g.uniform(0.25, 0.75, 3)
    leaves = synthetic.octree_leaves(nb, levels, centre, float(g.uniform(0.2, 0.35)))
    mesh = mfx.Mesh.octree(nb, nb, nb, leaves, dirichlet=dirichlet)
    T = mesh.tables(k)
    H = mesh.hanging_tables(k)
    om = omesh.octree_mesh(nb, nb, nb, k, leaves, dirichlet=dirichlet)
    assert np.array_equal(T["cell_dofs"], om.cell_dofs)
    n_cells = T["cell_dofs"].shape[0]
    rows = _oracle_rows(om)
    hanging = {d for d, r in rows.items() if r}
    tensor = _tensor_rows(H, n_cells, k)
    assert tensor, "the refined ball leaves no hanging faces"
    covered = set()
    for (c, li), w in tensor.items():
        dof = int(om.cell_dofs[c, li])
        if dof in rows:  # constrained: hanging (oracle row) or Dirichlet (empty row, the value is 0)
            assert _same(w, rows[dof]), (c, li, dof)
            covered.add((c, dof))
        else:  # a coarse node itself
            assert _same(w, {dof: 1.0}), (c, li, dof)
    # every hanging node of every cell lies on one of the cell's hanging faces or edges
    for c in range(n_cells):
        for li, dof in enumerate(om.cell_dofs[c]):
            if int(dof) in hanging:
                assert (c, int(dof)) in covered, (c, li, int(dof))


def test_structured_mesh_has_no_hanging_tables():
    H = mfx.Mesh.structured_box(3, 2, 2).hanging_tables(4)
    assert not H["hface"].any() and not H["hedge"].any() and not H["hoff"].any() and len(H["hdofs"]) == 0


def test_uniform_octree_has_no_hanging_tables():
    leaves = synthetic.octree_leaves(2, 1, (0.5, 0.5, 0.5), 2.0)  # the ball covers the box: uniform refinement
    H = mfx.Mesh.octree(2, 2, 2, leaves).hanging_tables(3)
    assert not H["hface"].any() and not H["hedge"].any() and len(H["hdofs"]) == 0
