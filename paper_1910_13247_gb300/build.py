"""Build libmfx.so in-tree for sm_103a (nvcc + g++, translation units compiled in parallel).

    python -m paper_1910_13247_gb300.build [--force]
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmfx.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) +
                  [p for p in glob.glob(os.path.join(CSRC, "*.cpp")) if not p.endswith("gen_basis.cpp")])


def _gen_basis_header(cuda_inc):
    """Generate _build/basis_tables.h with the library's own host rules (compiled for the host)."""
    hdr = os.path.join(OUT, "basis_tables.h")
    deps = [os.path.join(CSRC, f) for f in ("gen_basis.cpp", "host_rules.cpp", "mfx_internal.h")]
    if os.path.exists(hdr) and os.path.getmtime(hdr) >= max(os.path.getmtime(d) for d in deps):
        return hdr
    exe = os.path.join(OUT, "gen_basis")
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", cuda_inc, deps[0], deps[1], "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"basis generator build failed: {' '.join(cmd)}\n{r.stderr}")
    subprocess.check_call([exe, hdr + ".tmp"])
    os.replace(hdr + ".tmp", hdr)
    return hdr


def _headers():
    return glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        [os.path.join(HERE, "..", "include", "mfx.h")]


def _compile(src, nvcc, cuda_inc):
    obj = os.path.join(OUT, os.path.basename(src) + ".o")
    newest_dep = max(os.path.getmtime(h) for h in _headers() + [src, os.path.join(OUT, "basis_tables.h")])
    if os.path.exists(obj) and os.path.getmtime(obj) >= newest_dep:
        return obj
    if src.endswith(".cu"):
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-I", OUT, "-Xcompiler", "-fPIC",
               "-Xcompiler", "-ffp-contract=off", "--expt-relaxed-constexpr", "-c", src, "-o", obj]
    else:
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-I", cuda_inc, "-I", OUT, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj


def build(force=False, verbose=False):
    nvcc = _nvcc()
    cuda_home = os.path.dirname(os.path.dirname(nvcc))
    cuda_inc = os.path.join(cuda_home, "include")
    os.makedirs(OUT, exist_ok=True)
    if force:
        for o in glob.glob(os.path.join(OUT, "*.o")):
            os.remove(o)
    _gen_basis_header(cuda_inc)
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, nvcc, cuda_inc), srcs))
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(o) for o in objs):
        return LIB
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", LIB + ".tmp", *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(LIB + ".tmp", LIB)
    if verbose:
        print(LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
