"""Geometric multigrid V-cycle for the oracle (test infrastructure only).

The paper's large-scale solver is conjugate gradients preconditioned by a geometric multigrid V-cycle
with Chebyshev smoothing and matrix-free level transfers (Sec. 3.5, Sec. 6.1).  The oracle writes the
cycle out with assembled matrices, in this reading (the paper fixes none of these details):

  * h-multigrid on structured boxes: level l - 1 has half the cells per direction of level l, every
    level the same degree k; a level's vertices are every other vertex of the next finer level's
    lattice (so each level keeps the trilinear map of its own cells);
  * prolongation P: the coarse Q_k function evaluated at the fine nodes; in logical coordinates a fine
    lattice point I lies in coarse cell c = min(I // (2k), n_c - 1) at the reference position
    x_i / 2 (i = I - 2k c <= k) or (1 + x_{i-k}) / 2 (i > k), x the GLL nodes, so along one direction
    P1[I, c k + j] = l_j(position) and P = Pz (x) Py (x) Px (x fastest); rows of fine Dirichlet DoFs
    and columns of coarse Dirichlet DoFs are dropped (the condensed spaces); restriction is P^T;
  * the cycle on level l for K_l x = b: pre-smoothing x = S(b) with S the Chebyshev(m) polynomial in
    D^-1 K of fem.chebyshev on [lo_l, hi_l]; residual r = b - K x; coarse correction
    x += P V_{l-1}(P^T r); post-smoothing x += S(b - K x); on the coarsest level V_0 = K_0^-1 on the
    free DoFs (direct solve);
  * as a preconditioner of the condensed operator (identity on constrained rows, decoupled from the
    free ones) the cycle runs on the free DoFs and returns the residual itself on constrained rows;
  * optionally a discontinuous (SIPG, oracle/dg.py) level on top of the finest continuous one, on the
    same mesh and degree, reached by the injection of the continuous space (its transpose restricts),
    as in the paper's benchmark hierarchy.

Both smoothing steps use the same symmetric polynomial and the coarse solve is exact, so the cycle is
a symmetric linear operator.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem
from .mesh import structured_mesh, unit_vertices
from .rules import gauss_lobatto, lagrange


def coarsen_vertices(vertices, nx, ny, nz):
    """Every other vertex of an (nx+1)(ny+1)(nz+1) lattice (x fastest): the next coarser level's.

    The geometric multigrid hierarchy of Sec. 3.5.
    """
    v = np.asarray(vertices, dtype=np.float64).reshape(nz + 1, ny + 1, nx + 1, 3)
    return v[::2, ::2, ::2].reshape(-1, 3).copy()


def level_sizes(nx, ny, nz, max_levels=0):
    """Cells per direction of every level, coarse to fine: halve while all three counts are even (a
    2:1:1 box of 2^(l+1) x 2^l x 2^l cells ends on 2 x 1 x 1 cells, the coarse mesh of the paper's
    benchmark, Sec. 6.1), up to max_levels levels."""
    sizes = [(nx, ny, nz)]
    while all(s % 2 == 0 for s in sizes[0]) and (max_levels <= 0 or len(sizes) < max_levels):
        sizes.insert(0, tuple(s // 2 for s in sizes[0]))
    return sizes


def level_meshes(nx, ny, nz, k, vertices=None, max_levels=0, dirichlet=0x3F):
    """Levels of the geometric multigrid hierarchy of Sec. 3.5 (coarsest: the 2 x 1 x 1 mesh of Sec. 6.1 for the 2:1:1 box)."""
    sizes = level_sizes(nx, ny, nz, max_levels)
    if vertices is None:
        vertices = unit_vertices(nx, ny, nz)
    verts = [np.asarray(vertices, dtype=np.float64).reshape(-1, 3)]
    for (cx, cy, cz), (fx, fy, fz) in zip(reversed(sizes[:-1]), reversed(sizes[1:])):
        verts.insert(0, coarsen_vertices(verts[0], fx, fy, fz))
    return [structured_mesh(sx, sy, sz, k, v, dirichlet=dirichlet) for (sx, sy, sz), v in zip(sizes, verts)], sizes


def prolongation_1d(nc, k):
    """Fine lattice (2 k nc + 1 points) from coarse lattice (k nc + 1 points), one direction.

    The transfer between multigrid levels (Sec. 3.5).
    """
    x = gauss_lobatto(k)
    Mf, Mc = 2 * k * nc + 1, k * nc + 1
    P = np.zeros((Mf, Mc))
    for I in range(Mf):
        c = min(I // (2 * k), nc - 1)
        i = I - 2 * k * c
        pos = x[i] / 2.0 if i <= k else (1.0 + x[i - k]) / 2.0
        for j in range(k + 1):
            P[I, c * k + j] = float(lagrange(x, j, pos))
    return P


def prolongation(mc, mf, size_c, k, condensed=True):
    """The transfer between multigrid levels (Sec. 3.5)."""
    nxc, nyc, nzc = size_c
    P = sp.kron(sp.csr_matrix(prolongation_1d(nzc, k)),
                sp.kron(sp.csr_matrix(prolongation_1d(nyc, k)), sp.csr_matrix(prolongation_1d(nxc, k))))
    P = P.tocsr()
    if condensed:
        keep_f = np.ones(mf.n_dofs)
        keep_f[mf.constrained] = 0.0
        keep_c = np.ones(mc.n_dofs)
        keep_c[mc.constrained] = 0.0
        P = (sp.diags(keep_f) @ P @ sp.diags(keep_c)).tocsr()
        P.eliminate_zeros()
    return P


class Hierarchy:
    """Assembled levels: condensed K, inverse diagonal, Chebyshev interval, prolongation from below.

    The geometric multigrid V-cycle with Chebyshev smoothing (Sec. 3.5), the CG preconditioner of Sec. 6.1.
    """

    def __init__(self, meshes, sizes, k, coef_kind=fem.COEF_CONSTANT, coef_par=(1.0, 0.0), degree=6,
                 bounds=None, smoothing_range=20.0, lanczos_steps=15, dg_top=None):
        """dg_top = (K_dg, P): a discontinuous level above the finest continuous one, reached by the
        injection P of the continuous space (the paper's hierarchy switches from SIPG to the
        continuous space of the same degree on the same mesh before it coarsens)."""
        self.meshes, self.k, self.degree = list(meshes), k, degree
        self.K = [fem.assemble(m, k + 1, coef_kind, coef_par) for m in meshes]
        self.free = []
        for m in meshes:
            f = np.ones(m.n_dofs, dtype=bool)
            f[m.constrained] = False
            self.free.append(f)
        self.P = [None] + [prolongation(meshes[l - 1], meshes[l], sizes[l - 1], k) for l in range(1, len(meshes))]
        if dg_top is not None:
            self.K.append(dg_top[0].tocsr())
            self.P.append(dg_top[1].tocsr())
            self.free.append(np.ones(dg_top[0].shape[0], dtype=bool))
            self.meshes.append(None)
        self.dinv = [1.0 / fem.diagonal(K) for K in self.K]
        self.bounds = []
        for l, (K, dinv) in enumerate(zip(self.K, self.dinv)):
            if bounds is not None:
                self.bounds.append(bounds[l])
                continue
            start = self.free[l].astype(np.float64)  # ones on the free DoFs
            lam = fem.lanczos_lambda_max(lambda v, K=K: K @ v, dinv, start, lanczos_steps)
            hi = 1.2 * lam
            self.bounds.append((hi / smoothing_range, hi))
        f0 = self.free[0]
        self.coarse = spla.splu(self.K[0][f0][:, f0].tocsc()) if f0.any() else None

    def cycle(self, l, b):
        if l == 0:
            x = np.zeros_like(b)
            if self.coarse is not None:
                x[self.free[0]] = self.coarse.solve(b[self.free[0]])
            return x
        K, dinv, (lo, hi) = self.K[l], self.dinv[l], self.bounds[l]
        A = lambda v: K @ v  # noqa: E731
        x = fem.chebyshev(A, dinv, b, self.degree, lo, hi)
        r = b - K @ x
        x = x + self.P[l] @ self.cycle(l - 1, self.P[l].T @ r)
        r = b - K @ x
        return x + fem.chebyshev(A, dinv, r, self.degree, lo, hi)

    def vcycle(self, r):
        """Preconditioner of the finest condensed operator: the cycle on the free DoFs, identity on
        the constrained ones."""
        L = len(self.K) - 1
        b = np.where(self.free[L], r, 0.0)
        z = self.cycle(L, b)
        return np.where(self.free[L], z, r)
