"""The C-ABI from plain C: include/mfx.h compiles as pedantic C99 and a C program linked against
libmfx.so builds a mesh and its host-only tables through it (no GPU needed)."""
import os
import shutil
import subprocess

import pytest

from paper_1910_13247_gb300 import build as mbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include "mfx.h"

int main(void) {
  mfx_mesh* mesh = NULL;
  int64_t n_cells = 0, n_dofs = 0, n_constrained = 0, n_masters = 0;
  int32_t leaves[8 * 4];
  int q;
  mfx_status st;
  printf("%s\n", mfx_version());
  /* 2 x 1 x 1 structured box, Q3: (3*2+1) x 4 x 4 lattice */
  st = mfx_mesh_create_structured(&mesh, 2, 1, 1, NULL);
  if (st != MFX_OK) { printf("error %d %s\n", (int)st, mfx_last_error()); return 1; }
  st = mfx_mesh_table_sizes(mesh, 3, &n_cells, &n_dofs, &n_constrained, &n_masters);
  if (st != MFX_OK) return 2;
  printf("structured %lld %lld %lld %lld\n", (long long)n_cells, (long long)n_dofs, (long long)n_constrained,
         (long long)n_masters);
  mfx_mesh_destroy(mesh);
  /* one coarse cell refined once: eight level-1 leaves, no hanging nodes */
  for (q = 0; q < 8; ++q) {
    leaves[4 * q] = 1;
    leaves[4 * q + 1] = q & 1;
    leaves[4 * q + 2] = (q >> 1) & 1;
    leaves[4 * q + 3] = (q >> 2) & 1;
  }
  st = mfx_mesh_create_octree(&mesh, 1, 1, 1, NULL, leaves, 8);
  if (st != MFX_OK) return 3;
  st = mfx_mesh_table_sizes(mesh, 2, &n_cells, &n_dofs, &n_constrained, &n_masters);
  if (st != MFX_OK) return 4;
  printf("octree %lld %lld %lld %lld\n", (long long)n_cells, (long long)n_dofs, (long long)n_constrained,
         (long long)n_masters);
  mfx_mesh_destroy(mesh);
  /* errors come back as status codes with a message */
  st = mfx_mesh_create_structured(&mesh, 0, 1, 1, NULL);
  printf("invalid %d %d\n", (int)st, mfx_last_error()[0] != 0);
  return 0;
}
"""


def test_header_is_pedantic_c99_and_a_c_program_links_and_runs(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = mbuild.build()
    src = tmp_path / "consumer.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "consumer"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe), lib, "-Wl,-rpath," + os.path.dirname(lib)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.stdout, r.stderr)
    out = r.stdout.splitlines()
    assert "sm_103a" in out[0]
    # 7 x 4 x 4 lattice, all boundary points Dirichlet: interior 5 x 2 x 2
    assert out[1].split() == ["structured", "2", str(7 * 4 * 4), str(7 * 4 * 4 - 5 * 2 * 2), "0"]
    # a uniformly refined cell at Q2 is the 2 x 2 x 2 box: 5^3 lattice, 3^3 interior
    assert out[2].split() == ["octree", "8", "125", str(125 - 27), "0"]
    assert out[3].split() == ["invalid", "-1", "1"]
