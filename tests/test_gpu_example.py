"""The Python usage example of the README runs as written (on the GPU)."""
import os
import re

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_python_example_runs():
    pytest.importorskip("torch")
    from paper_1910_13247_gb300 import build
    build.build()
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, re.S)
    assert blocks, "no python block in the README"
    env = {"__name__": "readme_example"}
    exec(compile(blocks[0], "README.md", "exec"), env)
    assert env["u_octree"].size > 0 and env["st"]["status"] == 0
