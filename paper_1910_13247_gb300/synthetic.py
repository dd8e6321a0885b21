"""Seeded synthetic inputs for the matrix-free Laplacian workloads.

This module only generates inputs (vectors, vertex coordinates, octree leaf
lists, request streams).  It holds none of the finite-element arithmetic and
is shared by the tests, the benchmark and the reference checker.

Recipes (numpy PCG64 generators, seed given by the caller):
* vectors: uniform on [-1, 1] or standard Gaussian, FP64 (FP32 inputs are the
  FP64 vector rounded to nearest);
* deformed cube: lattice vertex x on [0,1]^3 moved to
  x + amp sin(pi x) sin(pi y) sin(pi z) (1, 1, 1), amp = 0.05 (the same
  scalar added to every component; identity on the boundary);
* octree leaves: coarse nb^3 grid, cells whose centre lies within a seeded
  radius of a seeded centre are refined, level by level, then the leaves
  are refined until 2:1 balanced across faces and edges.
"""
import math

import numpy as np


def rng(seed):
    return np.random.default_rng(seed)


def uniform_vector(n, seed):
    return rng(seed).uniform(-1.0, 1.0, size=n)


def gaussian_vector(n, seed):
    return rng(seed).standard_normal(size=n)


def lattice_vertices(nx, ny, nz):
    """(i/nx, j/ny, l/nz), lexicographic with x fastest, shape ((nx+1)(ny+1)(nz+1), 3)."""
    i = np.arange(nx + 1) / nx
    j = np.arange(ny + 1) / ny
    l = np.arange(nz + 1) / nz
    Z, Y, X = np.meshgrid(l, j, i, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def deformed_vertices(nx, ny, nz, amp=0.05):
    v = lattice_vertices(nx, ny, nz)
    s = amp * np.sin(math.pi * v[:, 0]) * np.sin(math.pi * v[:, 1]) * np.sin(math.pi * v[:, 2])
    return v + s[:, None]


def _dilate_faces_edges(a):
    """out[v] = a[v] or a[w] for every face or edge neighbour w of v (same level)."""
    out = a.copy()
    Z, Y, X = a.shape
    for d1 in range(3):
        for s1 in (1, -1):
            sh = [0, 0, 0]
            sh[d1] = s1
            shifts = [tuple(sh)]
            for d2 in range(d1 + 1, 3):
                for s2 in (1, -1):
                    sh2 = list(sh)
                    sh2[d2] = s2
                    shifts.append(tuple(sh2))
            for sz, sy, sx in [(v[2], v[1], v[0]) for v in shifts]:
                src = a[max(0, sz):Z + min(0, sz), max(0, sy):Y + min(0, sy), max(0, sx):X + min(0, sx)]
                dst = out[max(0, -sz):Z - max(0, sz), max(0, -sy):Y - max(0, sy), max(0, -sx):X - max(0, sx)]
                np.logical_or(dst, src, out=dst)
    return out


def _children_any(a):
    """Level-L array: any of the 8 level-(L+1) children set."""
    Z, Y, X = a.shape
    return a.reshape(Z // 2, 2, Y // 2, 2, X // 2, 2).any(axis=(1, 3, 5))


def octree_leaves(nb, levels, center, radius):
    """Leaves (level, i, j, l) of an nb^3 grid refined `levels` times inside a ball, 2:1 balanced.

    ref[L] marks the level-L cells that are refined.  A leaf is refined when its centre lies within
    `radius` of `center` (level by level), then the smallest balanced refinement is taken: a level-L
    leaf is refined while a refined level-(L+1) cell touches it across a face or an edge.
    """
    center = np.asarray(center, dtype=np.float64)
    exists = [np.ones((nb, nb, nb), dtype=bool)]
    ref = []
    for L in range(levels + 1):
        n = nb << L
        c = (np.arange(n) + 0.5) / n
        Zc, Yc, Xc = np.meshgrid(c, c, c, indexing="ij")
        inside = (Xc - center[0]) ** 2 + (Yc - center[1]) ** 2 + (Zc - center[2]) ** 2 < radius * radius
        r = exists[L] & inside if L < levels else np.zeros_like(exists[L])
        ref.append(r)
        if L < levels:
            exists.append(np.repeat(np.repeat(np.repeat(r, 2, 0), 2, 1), 2, 2))
    # balance: fine to coarse, repeated until nothing changes
    changed = True
    while changed:
        changed = False
        for L in range(levels - 1, -1, -1):
            need = _children_any(_dilate_faces_edges(ref[L + 1])) & exists[L] & ~ref[L]
            if need.any():
                ref[L] |= need
                changed = True
                exists[L + 1] = np.repeat(np.repeat(np.repeat(ref[L], 2, 0), 2, 1), 2, 2)
                # children of newly refined cells exist; deeper levels keep their refinement marks
                for M in range(L + 1, levels):
                    ref[M] &= exists[M]
                    exists[M + 1] = np.repeat(np.repeat(np.repeat(ref[M], 2, 0), 2, 1), 2, 2)
    out = []
    for L in range(levels + 1):
        leaf = exists[L] & ~ref[L]
        lz, ly, lx = np.nonzero(leaf)
        out.append(np.stack([np.full(lx.shape, L), lx, ly, lz], axis=1))
    leaves = np.concatenate(out).astype(np.int64)
    order = np.lexsort((leaves[:, 3], leaves[:, 2], leaves[:, 1], leaves[:, 0]))
    return leaves[order]


def random_octree(seed, nb=8, max_levels=3):
    """Seeded octree: levels uniform in 1..max_levels, centre in [0.2, 0.8]^3, radius in [0.15, 0.35]."""
    g = rng(seed)
    levels = int(g.integers(1, max_levels + 1))
    center = g.uniform(0.2, 0.8, size=3)
    radius = float(g.uniform(0.15, 0.35))
    return octree_leaves(nb, levels, center, radius)
