"""Checked mode: device-side validation of the index tables that the per-cell kernels read (in place of a
memory checker). The operators' own tables validate clean; entries planted out of range or inconsistent in
copies of sound tables are each counted; MFX_CHECKED=1 validates at operator creation."""
import numpy as np
import pytest

from paper_1910_13247_gb300 import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def mfx():
    from paper_1910_13247_gb300 import build, mfx as m
    build.build()
    m.lib()
    return m


def _octree_mesh(mfx):
    leaves = synthetic.octree_leaves(3, 2, np.array([0.4, 0.5, 0.6]), 0.3)
    return mfx.Mesh.octree(3, 3, 3, leaves, synthetic.deformed_vertices(3, 3, 3))


def test_operators_have_sound_tables(mfx):
    octree = _octree_mesh(mfx)
    ops = [mfx.Operator(mfx.Mesh.structured_box(4, 3, 2), 4),                # row-batch kernels: no tables
           mfx.Operator(mfx.Mesh.structured_box(3, 2, 2), 7),                # lattice table (k >= 6)
           mfx.Operator(octree, 2, mfx.COEF_TRIG, (1.0, 0.5)),              # per-node hanging constraints
           mfx.Operator(octree, 4, mfx.COEF_TRIG, (1.0, 0.5)),              # tensor-product constraints
           mfx.Operator(mfx.Mesh.structured_box(4, 2, 2), 3, discretization=mfx.SIPG)]
    assert ops[3].info()["n_hanging"] > 0
    for op in ops:
        assert op.validate() == 0


def test_checked_mode_at_creation(mfx, monkeypatch):
    monkeypatch.setenv("MFX_CHECKED", "1")
    op = mfx.Operator(_octree_mesh(mfx), 3, mfx.COEF_TRIG, (1.0, 0.5))
    x = torch.ones(op.n_dofs, dtype=torch.float64, device=DEV)
    y = torch.empty_like(x)
    op.vmult(x, y)
    op.device_check()
    assert op.validate() == 0


def _device_tables(mfx, k):
    """Sound tables of an octree in the device encoding, built from the host-only table calls."""
    mesh = _octree_mesh(mfx)
    T = mesh.tables(k)
    H = mesh.hanging_tables(k)
    cons = T["constrained"]
    cd = T["cell_dofs"].reshape(-1).astype(np.int64)
    pos = np.searchsorted(cons, cd)
    is_c = (pos < len(cons)) & (cons[np.minimum(pos, len(cons) - 1)] == cd)
    codes = np.where(is_c, -1 - pos, cd).astype(np.int32)
    hang = np.nonzero((H["hface"] & 0x3F) | (H["hedge"] & 0xFFF))[0].astype(np.int32)
    plain = np.setdiff1d(np.arange(T["cell_dofs"].shape[0], dtype=np.int32), hang)

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)

    tabs = {"cell_dofs": dev(codes), "cptr": dev(T["cptr"]), "cmaster": dev(T["cmaster"]),
            "hface": dev(H["hface"].view(np.int32)), "hedge": dev(H["hedge"].view(np.int32)),
            "hoff": dev(H["hoff"]), "hdofs": dev(H["hdofs"]), "lists": (dev(plain), dev(hang))}
    return T["cell_dofs"].shape[0], T["n_dofs"], len(cons), tabs


def _count(mfx, k, n_cells, n_dofs, n_rows, t):
    return mfx.validate_tables(n_cells, k + 1, n_dofs, t["cell_dofs"], n_rows=n_rows, cptr=t["cptr"],
                               cmaster=t["cmaster"], hface=t["hface"], hedge=t["hedge"], hoff=t["hoff"],
                               hdofs=t["hdofs"], cell_lists=t["lists"])


def test_planted_bad_entries_are_counted(mfx):
    k = 3
    n_cells, n_dofs, n_rows, good = _device_tables(mfx, k)
    assert _count(mfx, k, n_cells, n_dofs, n_rows, good) == 0
    plain_cell = int(good["lists"][0][0])
    hoff_cell = int(torch.nonzero(good["hoff"][1:] > good["hoff"][:-1])[0]) + 1  # a cell after one with slots

    def planted(name, fn):
        t = dict(good)
        if name == "lists":
            t["lists"] = (good["lists"][0].clone(), good["lists"][1])
            fn(t["lists"][0])
        else:
            t[name] = good[name].clone()
            fn(t[name])
        return _count(mfx, k, n_cells, n_dofs, n_rows, t)

    cases = [
        ("cell_dofs", lambda a: a.__setitem__(5, n_dofs), 1),              # DoF past the end
        ("cell_dofs", lambda a: a.__setitem__(7, -n_rows - 1), 1),         # constraint row past the end
        ("cptr", lambda a: a.__setitem__(-1, a[-1] + 1), 1),               # last pointer is not n_masters
        ("cptr", lambda a: a.__setitem__(0, 1), 1),                        # first pointer is not 0
        ("cmaster", lambda a: a.__setitem__(0, -1), 1),                    # negative master
        ("hdofs", lambda a: a.__setitem__(0, -2), 1),                      # below the "constrained" code
        ("hface", lambda a: a.__setitem__(plain_cell, 1 << 20), 1),        # undefined bit
        ("hedge", lambda a: a.__setitem__(plain_cell, 1 << 12), 1),        # half bit of an edge that is not hanging
        ("hoff", lambda a: a.__setitem__(hoff_cell, a[hoff_cell] + 1), 2),  # slots no longer contiguous
        ("lists", lambda a: a.__setitem__(0, n_cells), 1),                 # cell past the end
    ]
    for name, fn, expected in cases:
        assert planted(name, fn) == expected, name
    with pytest.raises(mfx.MfxError) as e:
        mfx.validate_tables(n_cells, k + 1, n_dofs, None)
    assert e.value.code == mfx.EINVAL
