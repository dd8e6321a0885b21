"""The allocation-free dot product (mfx_dot_noalloc) against the regular one (mfx_dot).

mfx_dot_noalloc exists for callers that may not allocate device memory (a plug-in whose
host application owns all device memory, or code inside another runtime's memory pool):
it keeps its reduction partials in a fixed array compiled into the library.  This file is collected
last so that a failure here cannot hide any other test's result.
"""
import numpy as np
import pytest

from paper_1910_13247_gb300 import synthetic

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mfx():
    from paper_1910_13247_gb300 import build, mfx as m
    build.build()
    m.lib()
    return m


@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_noalloc_dot_matches_operator_dot_on_two_calls(mfx, dtype):
    op = mfx.Operator(mfx.Mesh.structured_box(6, 5, 4), 3)
    n = op.n_dofs
    dt = getattr(torch, dtype)
    for call in range(2):
        a = torch.tensor(synthetic.uniform_vector(n, 40 + call), device="cuda", dtype=dt)
        b = torch.tensor(synthetic.uniform_vector(n, 50 + call), device="cuda", dtype=dt)
        ref = torch.zeros(1, dtype=torch.float64, device="cuda")
        got = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        op.dot(a, b, ref)
        mfx.dot_noalloc(a, b, got)
        torch.cuda.synchronize()
        scale = float((a.double().abs() * b.double().abs()).sum())
        assert abs(got.item() - ref.item()) <= 1e-12 * scale, (call, got.item(), ref.item())


def test_noalloc_dot_rejects_sizes_beyond_the_maximum(mfx):
    a = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(mfx.MfxError) as e:
        mfx.dot_noalloc(a, a, out, n=2 ** 31)
    assert e.value.code == mfx.EINVAL
