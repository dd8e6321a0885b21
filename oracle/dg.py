"""Symmetric interior penalty discontinuous Galerkin (SIPG) Laplacian for the oracle (test infrastructure).

The paper's multigrid benchmark discretises the 3D Laplacian with SIPG of degree p = 4 on a
hyper-rectangle (Sec. 6.1).  The oracle assembles that operator by full quadrature on a uniform
Cartesian box, in this reading (the paper gives no formulas):

  * space: discontinuous tensor-product Q_k on Gauss-Lobatto nodes, DoFs cell-major
    (cell c, local node i1 + n (i2 + n i3), n = k + 1), cells lexicographic (x fastest);
  * a(u, v) = sum_K int_K a grad u . grad v
             + sum_{interior F} int_F a ( -{d_n u} [v] - [u] {d_n v} + sigma_F [u] [v] )
             + sum_{Dirichlet F} int_F a ( -(d_n u) v - u (d_n v) + sigma_F u v ),
    with n the normal from the lower to the upper cell (outward on the boundary), [w] = w^- - w^+,
    {w} = (w^- + w^+) / 2, a a constant coefficient, homogeneous Dirichlet data imposed weakly on
    the faces in the Dirichlet mask (the others are natural boundaries, no face term);
  * penalty sigma_F = eta (k + 1)^2 (1/h^- + 1/h^+) / 2 on interior faces and eta (k + 1)^2 2/h on
    boundary faces, h the cell size normal to the face, eta = 1 unless given;
  * (k + 1)-point Gauss quadrature per direction on cells and faces.
"""
import numpy as np
import scipy.sparse as sp

from .mesh import Mesh
from .rules import gauss_legendre, gauss_lobatto, lagrange, lagrange_deriv


def _tables(k, nq):
    x = gauss_lobatto(k)
    xq, wq = gauss_legendre(nq)
    n = k + 1
    V = np.array([[float(lagrange(x, i, t)) for i in range(n)] for t in xq])          # [q][i]
    Dv = np.array([[float(lagrange_deriv(x, i, t)) for i in range(n)] for t in xq])
    e = {s: np.array([float(lagrange(x, i, float(s))) for i in range(n)]) for s in (0, 1)}
    de = {s: np.array([float(lagrange_deriv(x, i, float(s))) for i in range(n)]) for s in (0, 1)}
    return x, xq, wq, V, Dv, e, de


def dg_operator(nx, ny, nz, k, lengths=(1.0, 1.0, 1.0), dirichlet=0x3F, eta=1.0, coef=1.0):
    """Sparse SIPG matrix of the uniform box [0, Lx] x [0, Ly] x [0, Lz] with nx x ny x nz cells.

    The symmetric interior penalty discretisation of the multigrid benchmark of Sec. 6.1.
    """
    n, n3 = k + 1, (k + 1) ** 3
    h = np.array([lengths[0] / nx, lengths[1] / ny, lengths[2] / nz])
    x, xq, wq, V, Dv, e, de = _tables(k, n)
    vol = h[0] * h[1] * h[2]
    # cell matrix by the literal loop over 3D quadrature points
    loc = [(i % n, (i // n) % n, i // (n * n)) for i in range(n3)]
    A = np.zeros((n3, n3))
    for q3 in range(n):
        for q2 in range(n):
            for q1 in range(n):
                qq = (q1, q2, q3)
                w = wq[q1] * wq[q2] * wq[q3] * vol
                grads = np.zeros((n3, 3))
                for i, ii in enumerate(loc):
                    for d in range(3):
                        g = 1.0
                        for t in range(3):
                            g *= (Dv[qq[t], ii[t]] / h[t]) if t == d else V[qq[t], ii[t]]
                        grads[i, d] = g
                A += coef * w * grads @ grads.T
    C = nx * ny * nz
    rows, cols, vals = [], [], []

    def add_block(ca, cb, B):
        ra = ca * n3 + np.arange(n3)
        rb = cb * n3 + np.arange(n3)
        rows.append(np.repeat(ra, n3))
        cols.append(np.tile(rb, n3))
        vals.append(B.ravel())

    for c in range(C):
        add_block(c, c, A)

    def cell_index(ix, iy, iz):
        return ix + nx * (iy + ny * iz)

    pen = eta * (k + 1) ** 2

    def face_traces(d, s):
        """Values and d-derivatives (physical, along +e_d) at the face's Gauss points (n^2), of every
        local basis function of a cell whose face xi_d = s it is."""
        others = [t for t in range(3) if t != d]
        val = np.zeros((n * n, n3))
        der = np.zeros((n * n, n3))
        wts = np.zeros(n * n)
        for qb in range(n):
            for qa in range(n):
                qi = qa + n * qb
                wts[qi] = wq[qa] * wq[qb] * h[others[0]] * h[others[1]]
                for i, ii in enumerate(loc):
                    tang = V[qa, ii[others[0]]] * V[qb, ii[others[1]]]
                    val[qi, i] = e[s][ii[d]] * tang
                    der[qi, i] = de[s][ii[d]] / h[d] * tang
        return val, der, wts

    traces = {(d, s): face_traces(d, s) for d in range(3) for s in (0, 1)}
    dims = (nx, ny, nz)
    for iz in range(nz):
        for iy in range(ny):
            for ix in range(nx):
                c = cell_index(ix, iy, iz)
                idx = (ix, iy, iz)
                for d in range(3):
                    # interior face above this cell in direction d: this cell is "-", the neighbour "+"
                    if idx[d] + 1 < dims[d]:
                        nb = list(idx)
                        nb[d] += 1
                        cp = cell_index(*nb)
                        vm, dm, w = traces[(d, 1)]   # lower cell at xi_d = 1
                        vp, dp, _ = traces[(d, 0)]   # upper cell at xi_d = 0
                        sig = pen * (1.0 / h[d] + 1.0 / h[d]) / 2.0
                        # jump [phi] = phi (for "-" functions), -phi (for "+"); average of d_n = d / 2
                        J = {"m": vm, "p": -vp}
                        Dn = {"m": dm / 2.0, "p": dp / 2.0}
                        for a, ca in (("m", c), ("p", cp)):
                            for b, cb in (("m", c), ("p", cp)):
                                # rows: test functions of side a, columns: trial functions of side b
                                B = -(J[a].T * w) @ Dn[b] - (Dn[a].T * w) @ J[b] + sig * (J[a].T * w) @ J[b]
                                add_block(ca, cb, coef * B)
                    # boundary faces
                    for s in (0, 1):
                        on_bnd = (idx[d] == 0 and s == 0) or (idx[d] == dims[d] - 1 and s == 1)
                        if not on_bnd or not (dirichlet >> (2 * d + s)) & 1:
                            continue
                        v, dd, w = traces[(d, s)]
                        dn = dd if s == 1 else -dd   # outward normal derivative
                        sig = pen * 2.0 / h[d]
                        B = -(v.T * w) @ dn - (dn.T * w) @ v + sig * (v.T * w) @ v
                        add_block(c, c, coef * B)
    K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(C * n3, C * n3))
    K.sum_duplicates()
    return K


def dg_mesh(nx, ny, nz, k, lengths=(1.0, 1.0, 1.0)):
    """The DG space as an oracle Mesh (cell-major DoFs, no constraints), for the L2 error and the
    right-hand side routines.
    The discontinuous space of Sec. 6.1."""
    n3 = (k + 1) ** 3
    C = nx * ny * nz
    cv = np.zeros((C, 8, 3))
    h = (lengths[0] / nx, lengths[1] / ny, lengths[2] / nz)
    c = 0
    for iz in range(nz):
        for iy in range(ny):
            for ix in range(nx):
                for v in range(8):
                    a, b, e = v & 1, (v >> 1) & 1, (v >> 2) & 1
                    cv[c, v] = ((ix + a) * h[0], (iy + b) * h[1], (iz + e) * h[2])
                c += 1
    cd = np.arange(C * n3, dtype=np.int64).reshape(C, n3)
    empty = np.zeros(0, dtype=np.int64)
    return Mesh(cv, cd, C * n3, empty, np.zeros(1, dtype=np.int64), empty, np.zeros(0), k)


def injection(cg_mesh, k):
    """Matrix of the continuous space in the discontinuous one on the same structured mesh: DG DoF
    (c, i) takes the CG value at the same node (0 for Dirichlet CG DoFs).
    The switch from the discontinuous to the continuous space in the hierarchy of Sec. 6.1."""
    C, n3 = cg_mesh.cell_dofs.shape
    keep = np.ones(cg_mesh.n_dofs)
    keep[cg_mesh.constrained] = 0.0
    r = np.arange(C * n3)
    cidx = cg_mesh.cell_dofs.ravel()
    return sp.csr_matrix((keep[cidx], (r, cidx)), shape=(C * n3, cg_mesh.n_dofs))
