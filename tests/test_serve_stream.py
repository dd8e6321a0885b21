"""CPU checks of the serving workload's seeded request stream: Poisson arrivals at the stated rate,
degrees 1..8, reproducible from the seed, and every request's octree a valid 2:1 balanced tiling of its
coarse box whose size follows the log-uniform target (up to the generator's clamp)."""
import math

import numpy as np
import pytest

from paper_1910_13247_gb300 import build as mbuild
from paper_1910_13247_gb300 import mfx, serve


@pytest.fixture(scope="module", autouse=True)
def _built():
    mbuild.build()
    mfx.lib()


def test_arrivals_degrees_and_reproducibility():
    rate = 200.0
    reqs = serve.make_requests(400, rate=rate, seed=7, size_range=(1e3, 3e4))
    t = np.array([r.arrival for r in reqs])
    gaps = np.diff(np.concatenate(([0.0], t)))
    assert (gaps > 0).all()
    # exponential gaps: mean 1/rate (3 standard errors at n = 400), coefficient of variation 1
    assert abs(gaps.mean() * rate - 1.0) < 3.0 / math.sqrt(len(gaps))
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.2
    ks = np.array([r.degree for r in reqs])
    assert set(ks.tolist()) == set(range(1, 9))
    again = serve.make_requests(400, rate=rate, seed=7, size_range=(1e3, 3e4))
    assert [r.arrival for r in again] == t.tolist()
    assert all(np.array_equal(a.leaves, b.leaves) and a.degree == b.degree for a, b in zip(reqs, again))
    other = serve.make_requests(400, rate=rate, seed=8, size_range=(1e3, 3e4))
    assert [r.arrival for r in other] != t.tolist()


def test_octrees_tile_the_box_and_follow_the_target_size():
    lo, hi = 1e3, 3e4
    reqs = serve.make_requests(24, rate=200.0, seed=9, size_range=(lo, hi))
    for r in reqs:
        lv = r.leaves
        assert lv.shape[1] == 4 and lv[:, 0].min() >= 0 and lv[:, 0].max() <= 3
        # leaves cover the nb^3 coarse cells exactly: volumes 8^-level sum to nb^3, no leaf outside
        assert np.isclose(np.sum(8.0 ** -lv[:, 0]), r.nb ** 3)
        assert (lv[:, 1:] < (r.nb << lv[:, :1])).all() and (lv[:, 1:] >= 0).all()
        # the library accepts the mesh (it rejects overlaps, holes and 2:1 violations with MFX_EMESH)
        mesh = mfx.Mesh.octree(r.nb, r.nb, r.nb, lv)
        n_dofs = mesh.tables(r.degree)["n_dofs"]
        if r.nb > 2:  # not clamped from below: the size is near the log-uniform target range
            assert lo / 8 <= n_dofs <= hi * 8, (r.rid, n_dofs)
