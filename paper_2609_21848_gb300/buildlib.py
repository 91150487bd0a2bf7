"""Compile the CUDA library ``libdbbc.so`` for sm_103a, in-tree.

Each ``csrc/*.cu`` translation unit is compiled in parallel with nvcc
(``-gencode arch=compute_103a,code=sm_103a``), then linked into
``_build/libdbbc.so`` next to this file. The CUDA runtime is linked
statically, so the library needs only the driver at load time.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libdbbc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
              "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdbbc.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        [os.path.join(os.path.dirname(HERE), "include", "dbbc.h")]


# The bounds-checked debug build (-DDBBC_CHECKED=1): kernels test every index
# they derive from graph data and record a flag instead of accessing out of
# bounds (see dbbc_checked_flags in include/dbbc.h).
CHECKED_DIR = os.path.join(OUT_DIR, "checked")
CHECKED_FLAGS = ["-DDBBC_CHECKED=1"]


def _stamp(lib_path: str) -> str:
    return lib_path + ".flags"


def up_to_date(lib_path: str = LIB, extra_flags: list[str] | None = None) -> bool:
    """The library at lib_path exists, is newer than every source and was
    built with the same extra flags."""
    if not os.path.exists(lib_path):
        return False
    want = " ".join(extra_flags or [])
    have = open(_stamp(lib_path)).read() if os.path.exists(_stamp(lib_path)) else ""
    if have != want:
        return False
    t = os.path.getmtime(lib_path)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None,
          out_dir: str | None = None) -> str:
    """Build the library (into ``out_dir`` instead of ``_build/`` when given,
    e.g. for a variant with -D overrides)."""
    lib_path = os.path.join(out_dir, "libdbbc.so") if out_dir else LIB
    if not force and up_to_date(lib_path, extra_flags):
        return lib_path
    obj_dir = out_dir or OUT_DIR
    os.makedirs(obj_dir, exist_ok=True)
    cc = nvcc()
    flags = NVCC_FLAGS + (extra_flags or [])

    def compile_one(src):
        obj = os.path.join(obj_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *ARCH, *flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, len(_sources()))) as ex:
        objs = list(ex.map(compile_one, _sources()))
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", *objs, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    with open(_stamp(lib_path), "w") as f:
        f.write(" ".join(extra_flags or []))
    os.replace(tmp, lib_path)
    return lib_path


def build_checked(force: bool = False) -> str:
    """Build the bounds-checked library into ``_build/checked/``."""
    return build(force=force, extra_flags=CHECKED_FLAGS, out_dir=CHECKED_DIR)


if __name__ == "__main__":
    print(build(force=True, verbose=True))
