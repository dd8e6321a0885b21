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


def _neighbour_shifts():
    shifts = []
    for d in range(3):
        for sgn in (1, -1):
            s = [0, 0, 0]
            s[d] = sgn
            shifts.append(s)
    for d1 in range(3):
        for d2 in range(d1 + 1, 3):
            for s1 in (1, -1):
                for s2 in (1, -1):
                    s = [0, 0, 0]
                    s[d1] = s1
                    s[d2] = s2
                    shifts.append(s)
    return shifts


def _max_neighbour_level(lev):
    """Per finest voxel, the largest level among its face/edge neighbour voxels."""
    out = lev.copy()
    Z, Y, X = lev.shape
    for sx, sy, sz in _neighbour_shifts():
        src = lev[max(0, sz):Z + min(0, sz), max(0, sy):Y + min(0, sy), max(0, sx):X + min(0, sx)]
        dst = out[max(0, -sz):Z - max(0, sz), max(0, -sy):Y - max(0, sy), max(0, -sx):X - max(0, sx)]
        np.maximum(dst, src, out=dst)
    return out


def octree_leaves(nb, levels, center, radius):
    """Leaves (level, i, j, l) of an nb^3 grid refined `levels` times inside a ball, 2:1 balanced."""
    leaves = {(0, i, j, l) for l in range(nb) for j in range(nb) for i in range(nb)}

    def centre(lf):
        L, i, j, l = lf
        h = 1.0 / (nb << L)
        return np.array([(i + 0.5) * h, (j + 0.5) * h, (l + 0.5) * h])

    def children(lf):
        L, i, j, l = lf
        return [(L + 1, 2 * i + a, 2 * j + b, 2 * l + c) for c in (0, 1) for b in (0, 1) for a in (0, 1)]

    center = np.asarray(center, dtype=np.float64)
    for L in range(levels):
        ref = [lf for lf in leaves if lf[0] == L and np.linalg.norm(centre(lf) - center) < radius]
        for lf in ref:
            leaves.remove(lf)
            leaves.update(children(lf))
    # 2:1 balance across faces and edges
    Lmax = max(lf[0] for lf in leaves)
    R = 1 << Lmax
    while True:
        lev = np.zeros((nb * R, nb * R, nb * R), dtype=np.int64)
        for (L, i, j, l) in leaves:
            s = 1 << (Lmax - L)
            lev[l * s:(l + 1) * s, j * s:(j + 1) * s, i * s:(i + 1) * s] = L
        mx = _max_neighbour_level(lev)
        bad = []
        for lf in leaves:
            L, i, j, l = lf
            s = 1 << (Lmax - L)
            if mx[l * s:(l + 1) * s, j * s:(j + 1) * s, i * s:(i + 1) * s].max() > L + 1:
                bad.append(lf)
        if not bad:
            break
        for lf in bad:
            leaves.remove(lf)
            leaves.update(children(lf))
    return np.array(sorted(leaves), dtype=np.int64)


def random_octree(seed, nb=8, max_levels=3):
    """Seeded octree: levels uniform in 1..max_levels, centre in [0.2, 0.8]^3, radius in [0.15, 0.35]."""
    g = rng(seed)
    levels = int(g.integers(1, max_levels + 1))
    center = g.uniform(0.2, 0.8, size=3)
    radius = float(g.uniform(0.15, 0.35))
    return octree_leaves(nb, levels, center, radius)
