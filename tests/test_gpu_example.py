"""The committed Python usage example (paper_1910_13247_gb300/example.py) runs as written on the GPU."""
import runpy

import pytest

pytestmark = pytest.mark.gpu


def test_python_example_runs():
    pytest.importorskip("torch")
    from paper_1910_13247_gb300 import build
    build.build()
    env = runpy.run_module("paper_1910_13247_gb300.example", run_name="example")
    assert env["u_octree"].size > 0 and env["st"]["status"] == 0
