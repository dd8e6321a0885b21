"""Meshes, DoF numbering and constraints for the oracle (test infrastructure).

The paper's meshes are hexahedral (Sec. 3.1) with tensor-product Lagrange
elements; adaptive refinement produces hanging nodes (Sec. 3.1, Sec. 3.3,
Fig. 2) whose values are fixed by continuity.  The paper does not spell out
the numbering or the constraint tables, so the oracle follows these
readings (also implemented, independently, by the library):

Structured mesh (nx x ny x nz cells):
  * vertices lexicographic, x fastest; cells lexicographic, x fastest;
    cell vertex v = a + 2 b + 4 c for corner (a, b, c);
  * global DoF = I + Mx (J + My L) on the (k nx + 1) x (k ny + 1) x (k nz + 1)
    lattice of GLL nodes; local DoF = i1 + n (i2 + n i3), n = k + 1;
  * Dirichlet: every DoF on a Dirichlet face of the box is constrained to 0;
    by default all six faces, else the faces of the bit mask `dirichlet`
    (bit 2d: the face at coordinate 0 in direction d, bit 2d + 1: the far
    face); the other faces are natural boundaries of the weak form.

Octree mesh (leaves (level, i, j, l) over an nx x ny x nz coarse grid):
  * leaves must tile the coarse box and be 2:1 balanced across faces and
    edges; the cell order is (coarse cell lexicographic, Morton order of
    the leaf's lower corner within its tree, x bit lowest);
  * leaf vertices are the trilinear map of the coarse cell's vertices at
    the leaf's reference corners;
  * a node's identity is its exact position: per dimension either a
    rational position (GLL nodes 0, 1/2 (even k) and 1 of the cell) or an
    interior GLL node of one specific cell row (level, index, local node);
    DoFs are numbered on first encounter, walking cells in order and local
    nodes lexicographically;
  * hanging nodes: a node of a finer leaf that lies on a face or edge of a
    coarser leaf without being a node of it is constrained to that leaf's
    face (edge) nodes with weights l_m1(p1) l_m2(p2) (l_m(p) on edges),
    p its position in the coarse face (edge) coordinates;
  * Dirichlet takes precedence over hanging; Dirichlet masters and
    masters with weight exactly 0 are dropped; masters are sorted by DoF;
    a master that is itself constrained is an error.
"""
import numpy as np

from .rules import gauss_lobatto, lagrange


class Mesh:
    """Cells with 8 physical vertices each, plus the DoF tables of degree k.

    The triangulation with its DoF numbering and constraints (Sec. 3.1).
    """

    def __init__(self, cell_vertices, cell_dofs, n_dofs, constrained, cptr, cmaster,
                 cweight, k):
        self.cell_vertices = cell_vertices      # (C, 8, 3) float64
        self.cell_dofs = cell_dofs              # (C, n^3) int64
        self.n_dofs = int(n_dofs)
        self.constrained = constrained          # sorted int64
        self.cptr = cptr                        # int64, len = len(constrained) + 1
        self.cmaster = cmaster                  # int64
        self.cweight = cweight                  # float64
        self.k = k

    @property
    def n_cells(self):
        return self.cell_vertices.shape[0]


def unit_vertices(nx, ny, nz):
    """Vertex coordinates (i/nx, j/ny, l/nz), lexicographic, x fastest.

    Vertices of the structured box (Sec. 3.1).
    """
    i = np.arange(nx + 1) / nx
    j = np.arange(ny + 1) / ny
    l = np.arange(nz + 1) / nz
    Z, Y, X = np.meshgrid(l, j, i, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def structured_mesh(nx, ny, nz, k, vertices=None, dirichlet=0x3F):
    """Structured box mesh of nx*ny*nz cells with degree-k lexicographic DoFs.

    Tensor-product Q_k DoFs of a structured box (Sec. 3.1).
    """
    if vertices is None:
        vertices = unit_vertices(nx, ny, nz)
    vertices = np.asarray(vertices, dtype=np.float64).reshape(-1, 3)
    n = k + 1
    C = nx * ny * nz
    cv = np.zeros((C, 8, 3))
    cd = np.zeros((C, n ** 3), dtype=np.int64)
    Mx, My, Mz = k * nx + 1, k * ny + 1, k * nz + 1
    c = 0
    for cz in range(nz):
        for cy in range(ny):
            for cx in range(nx):
                for v in range(8):
                    a, b, e = v & 1, (v >> 1) & 1, (v >> 2) & 1
                    cv[c, v] = vertices[(cx + a) + (nx + 1) * ((cy + b) + (ny + 1) * (cz + e))]
                for i3 in range(n):
                    for i2 in range(n):
                        for i1 in range(n):
                            I, J, L = k * cx + i1, k * cy + i2, k * cz + i3
                            cd[c, i1 + n * (i2 + n * i3)] = I + Mx * (J + My * L)
                c += 1
    N = Mx * My * Mz
    I = np.arange(N) % Mx
    J = (np.arange(N) // Mx) % My
    L = np.arange(N) // (Mx * My)
    f = [bool(dirichlet >> b & 1) for b in range(6)]
    bnd = ((I == 0) & f[0]) | ((I == Mx - 1) & f[1]) | ((J == 0) & f[2]) | ((J == My - 1) & f[3]) | \
          ((L == 0) & f[4]) | ((L == Mz - 1) & f[5])
    constrained = np.nonzero(bnd)[0].astype(np.int64)
    cptr = np.zeros(len(constrained) + 1, dtype=np.int64)
    return Mesh(cv, cd, N, constrained, cptr, np.zeros(0, np.int64), np.zeros(0), k)


# ----------------------------------------------------------------------------
# octree meshes
# ----------------------------------------------------------------------------

class MeshError(ValueError):
    """An octree that violates the 2:1 balance or does not tile its box (Sec. 3.1)."""
    pass


def _morton(x, y, z, bits):
    m = 0
    for b in range(bits):
        m |= ((x >> b) & 1) << (3 * b)
        m |= ((y >> b) & 1) << (3 * b + 1)
        m |= ((z >> b) & 1) << (3 * b + 2)
    return m


def _leaf_owner_grid(nx, ny, nz, leaves, Lmax):
    """Finest-level voxel grid holding the index of the covering leaf; checks tiling."""
    R = 1 << Lmax
    owner = -np.ones((nz * R, ny * R, nx * R), dtype=np.int64)
    for idx, (L, i, j, l) in enumerate(leaves):
        s = 1 << (Lmax - L)
        blk = owner[l * s:(l + 1) * s, j * s:(j + 1) * s, i * s:(i + 1) * s]
        if np.any(blk >= 0):
            raise MeshError("leaves overlap")
        blk[...] = idx
    if np.any(owner < 0):
        raise MeshError("leaves do not cover the domain")
    return owner


def _check_balance(owner, levels):
    """2:1 balance across faces and edges, via neighbouring finest voxels."""
    lev = levels[owner]
    shifts = []
    for d in range(3):
        s = [0, 0, 0]
        s[d] = 1
        shifts.append(tuple(s))
    for d1 in range(3):
        for d2 in range(d1 + 1, 3):
            for sgn in (1, -1):
                s = [0, 0, 0]
                s[d1] = 1
                s[d2] = sgn
                shifts.append(tuple(s))
    Z, Y, X = lev.shape
    for sz, sy, sx in [(s[2], s[1], s[0]) for s in shifts]:
        a = lev[max(0, -sz):Z - max(0, sz), max(0, -sy):Y - max(0, sy), max(0, -sx):X - max(0, sx)]
        b = lev[max(0, sz):Z + min(0, sz), max(0, sy):Y + min(0, sy), max(0, sx):X + min(0, sx)]
        if np.any(np.abs(a - b) > 1):
            raise MeshError("mesh is not 2:1 balanced across faces and edges")


def octree_mesh(nx, ny, nz, k, leaves, coarse_vertices=None, dirichlet=0x3F):
    """Octree mesh from leaves (level, i, j, l), with DoF tables and constraints.

    Locally refined mesh with hanging nodes (Sec. 3.1, Fig. 2; constraints as in Sec. 3.3).
    """
    faces = int(dirichlet)  # Dirichlet face mask (the name is reused below for the Dirichlet DoF set)
    leaves = [tuple(int(v) for v in lf) for lf in np.asarray(leaves).reshape(-1, 4)]
    if not leaves:
        raise MeshError("no leaves")
    for L, i, j, l in leaves:
        if L < 0 or L > 8:
            raise MeshError("level out of range")
        if not (0 <= i < nx << L and 0 <= j < ny << L and 0 <= l < nz << L):
            raise MeshError("leaf index out of range")
    Lmax = max(lf[0] for lf in leaves)
    owner = _leaf_owner_grid(nx, ny, nz, leaves, Lmax)
    levels = np.array([lf[0] for lf in leaves], dtype=np.int64)
    _check_balance(owner, levels)

    # cell order: coarse cell lexicographic, then Morton order within the tree
    def order_key(lf):
        L, i, j, l = lf
        ci, cj, cl = i >> L, j >> L, l >> L
        sh = Lmax - L
        m = _morton((i - (ci << L)) << sh, (j - (cj << L)) << sh, (l - (cl << L)) << sh, Lmax)
        return (ci + nx * (cj + ny * cl), m)

    order = sorted(range(len(leaves)), key=lambda t: order_key(leaves[t]))
    leaves = [leaves[t] for t in order]
    remap = np.empty(len(order), dtype=np.int64)
    remap[np.array(order)] = np.arange(len(order))
    owner = remap[owner]

    if coarse_vertices is None:
        coarse_vertices = unit_vertices(nx, ny, nz)
    coarse_vertices = np.asarray(coarse_vertices, dtype=np.float64).reshape(-1, 3)
    n = k + 1
    g = gauss_lobatto(k)
    C = len(leaves)
    cv = np.zeros((C, 8, 3))
    for c, (L, i, j, l) in enumerate(leaves):
        ci, cj, cl = i >> L, j >> L, l >> L
        X = [coarse_vertices[(ci + a) + (nx + 1) * ((cj + b) + (ny + 1) * (cl + e))]
             for e in (0, 1) for b in (0, 1) for a in (0, 1)]
        for v in range(8):
            a, b, e = v & 1, (v >> 1) & 1, (v >> 2) & 1
            s = ((i - (ci << L)) + a) / (1 << L)
            t = ((j - (cj << L)) + b) / (1 << L)
            u = ((l - (cl << L)) + e) / (1 << L)
            p = np.zeros(3)
            for w in range(8):
                wa, wb, we = w & 1, (w >> 1) & 1, (w >> 2) & 1
                p = p + ((s if wa else 1 - s) * (t if wb else 1 - t) * (u if we else 1 - u)) * X[w]
            cv[c, v] = p

    R2 = 1 << (Lmax + 1)   # rational positions in units of 1/(2^(Lmax+1)) coarse cells
    ext = (nx * R2, ny * R2, nz * R2)

    def dim_key(L, I, a):
        if a == 0:
            return (0, I * (R2 >> L))
        if a == k:
            return (0, (I + 1) * (R2 >> L))
        if 2 * a == k:
            return (0, (2 * I + 1) * (R2 >> (L + 1)))
        return (1, L, I, a)

    def node_key(c, a1, a2, a3):
        L, i, j, l = leaves[c]
        return (dim_key(L, i, a1), dim_key(L, j, a2), dim_key(L, l, a3))

    dof_of = {}
    cd = np.zeros((C, n ** 3), dtype=np.int64)
    keys_of_cell = []
    for c in range(C):
        kc = []
        for a3 in range(n):
            for a2 in range(n):
                for a1 in range(n):
                    key = node_key(c, a1, a2, a3)
                    if key not in dof_of:
                        dof_of[key] = len(dof_of)
                    cd[c, a1 + n * (a2 + n * a3)] = dof_of[key]
                    kc.append(key)
        keys_of_cell.append(kc)
    key_sets = [set(kc) for kc in keys_of_cell]
    N = len(dof_of)

    def on_boundary(key):
        # on a Dirichlet face: a rational position at 0 or at the far end of the box
        for d in range(3):
            kd = key[d]
            if kd[0] == 0 and ((kd[1] == 0 and faces >> (2 * d) & 1) or
                               (kd[1] == ext[d] and faces >> (2 * d + 1) & 1)):
                return True
        return False

    dirichlet = set()
    for key, dof in dof_of.items():
        if on_boundary(key):
            dirichlet.add(dof)

    hanging = {}   # dof -> dict master -> weight

    def add_constraint(dof, masters):
        if dof in dirichlet:
            return
        clean = {}
        for m, w in masters:
            if w == 0.0 or m in dirichlet:
                continue
            clean[m] = w
        if dof in hanging:
            old = hanging[dof]
            if set(old) != set(clean) or any(abs(old[m] - clean[m]) > 1e-12 for m in old):
                raise MeshError("inconsistent hanging-node constraints")
            return
        hanging[dof] = clean

    Rf = 1 << Lmax

    def leaf_at(v):
        z, y, x = v
        if 0 <= x < nx * Rf and 0 <= y < ny * Rf and 0 <= z < nz * Rf:
            return owner[z, y, x]
        return -1

    for c, (L, i, j, l) in enumerate(leaves):
        s = 1 << (Lmax - L)
        lo = (i * s, j * s, l * s)
        idx = (i, j, l)
        # faces: dim d, side sd; look at voxels just across
        for d in range(3):
            u, v = [e for e in range(3) if e != d]
            for sd in (0, 1):
                across = lo[d] - 1 if sd == 0 else lo[d] + s
                fine = set()
                for pu in range(s):
                    for pv in range(s):
                        vox = [0, 0, 0]
                        vox[d] = across
                        vox[u] = lo[u] + pu
                        vox[v] = lo[v] + pv
                        o = leaf_at((vox[2], vox[1], vox[0]))
                        if o >= 0 and leaves[o][0] > L:
                            fine.add(o)
                for e in sorted(fine):
                    Le, ie, je, le = leaves[e]
                    if Le != L + 1:
                        raise MeshError("mesh is not 2:1 balanced")
                    eidx = (ie, je, le)
                    ou, ov = eidx[u] - 2 * idx[u], eidx[v] - 2 * idx[v]
                    ae_d = k if sd == 0 else 0   # fine leaf's face on our side
                    ac_d = 0 if sd == 0 else k
                    for bv in range(n):
                        for bu in range(n):
                            ae = [0, 0, 0]
                            ae[d], ae[u], ae[v] = ae_d, bu, bv
                            fdof = cd[e, ae[0] + n * (ae[1] + n * ae[2])]
                            if keys_of_cell[e][ae[0] + n * (ae[1] + n * ae[2])] in key_sets[c]:
                                continue
                            pu_ = (ou + g[bu]) * 0.5
                            pv_ = (ov + g[bv]) * 0.5
                            masters = []
                            for mv in range(n):
                                for mu in range(n):
                                    ac = [0, 0, 0]
                                    ac[d], ac[u], ac[v] = ac_d, mu, mv
                                    w = float(lagrange(g, mu, pu_)) * float(lagrange(g, mv, pv_))
                                    masters.append((int(cd[c, ac[0] + n * (ac[1] + n * ac[2])]), w))
                            add_constraint(int(fdof), masters)
        # edges: direction d, the two other dims at sides (su, sv)
        for d in range(3):
            u, v = [e for e in range(3) if e != d]
            for sv in (0, 1):
                for su in (0, 1):
                    fine = set()
                    for du in ((-1,) if su == 0 else (s,)):
                        for dv in ((-1,) if sv == 0 else (s,)):
                            for (xu, xv) in ((du, dv), (du, 0 if sv == 0 else s - 1),
                                             (0 if su == 0 else s - 1, dv)):
                                for pd in range(s):
                                    vox = [0, 0, 0]
                                    vox[d] = lo[d] + pd
                                    vox[u] = lo[u] + xu
                                    vox[v] = lo[v] + xv
                                    o = leaf_at((vox[2], vox[1], vox[0]))
                                    if o >= 0 and o != c and leaves[o][0] > L:
                                        fine.add(o)
                    for e in sorted(fine):
                        Le, ie, je, le = leaves[e]
                        if Le != L + 1:
                            raise MeshError("mesh is not 2:1 balanced")
                        eidx = (ie, je, le)
                        od = eidx[d] - 2 * idx[d]
                        # the fine leaf's nodes on our edge: positions along d, with the
                        # u/v coordinates on the edge line
                        edge_u = (idx[u] + su) * 2   # in fine-level units
                        edge_v = (idx[v] + sv) * 2
                        if edge_u == eidx[u]:
                            au = 0
                        elif edge_u == eidx[u] + 1:
                            au = k
                        else:
                            continue
                        if edge_v == eidx[v]:
                            av = 0
                        elif edge_v == eidx[v] + 1:
                            av = k
                        else:
                            continue
                        for bd in range(n):
                            ae = [0, 0, 0]
                            ae[d], ae[u], ae[v] = bd, au, av
                            li = ae[0] + n * (ae[1] + n * ae[2])
                            if keys_of_cell[e][li] in key_sets[c]:
                                continue
                            pd_ = (od + g[bd]) * 0.5
                            masters = []
                            for md in range(n):
                                ac = [0, 0, 0]
                                ac[d], ac[u], ac[v] = md, su * k, sv * k
                                w = float(lagrange(g, md, pd_))
                                masters.append((int(cd[c, ac[0] + n * (ac[1] + n * ac[2])]), w))
                            add_constraint(int(cd[e, li]), masters)

    constrained = sorted(dirichlet | set(hanging))
    cptr = [0]
    cmaster, cweight = [], []
    for dof in constrained:
        if dof in hanging:
            for m in sorted(hanging[dof]):
                if m in hanging:
                    raise MeshError("constraint master is itself constrained")
                cmaster.append(m)
                cweight.append(hanging[dof][m])
        cptr.append(len(cmaster))
    return Mesh(cv, cd, N, np.array(constrained, dtype=np.int64), np.array(cptr, dtype=np.int64),
                np.array(cmaster, dtype=np.int64), np.array(cweight, dtype=np.float64), k)
