"""Build of the CUDA shared library ``liblbm_mix.so`` (sm_103a only).

Each ``csrc/*.cu`` is compiled to an object in parallel with nvcc, then the
objects are linked into a shared library next to this file.  Rebuilds are
skipped when neither the sources nor the flags changed.
"""

from __future__ import annotations

import hashlib
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
INCLUDE = PKG.parent / "include"
BUILD = PKG.parent / "_build"
LIB = PKG / "liblbm_mix.so"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -prec-div=false: FP32 divisions as the approximate reciprocal-based form
# (within 2 ulp) instead of the IEEE sequence; the FP32 collide has a few
# dozen per node and is half issue-bound (measured on GB300, 128^3 acoustic
# pulse: 3905 against 3791 MLUPS).  FP64 arithmetic is unaffected.
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr", "-prec-div=false",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden"] + ARCH


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _sources():
    return sorted(CSRC.glob("*.cu"))


def _digest(extra_flags) -> str:
    h = hashlib.sha256()
    for p in sorted(list(CSRC.glob("*")) + list(INCLUDE.glob("*.h"))):
        h.update(p.name.encode())
        h.update(p.read_bytes())
    h.update(" ".join(NVCC_FLAGS + list(extra_flags)).encode())
    return h.hexdigest()


def build(verbose: bool = False, force: bool = False, extra_flags=()) -> Path:
    """Compile and link ``liblbm_mix.so``; returns its path.  Additional nvcc
    flags (tuning macros such as -DLBM_COLLIDE_MINB=3) may also come from the
    environment variable LBM_NVCC_EXTRA."""
    extra_flags = list(extra_flags) + os.environ.get("LBM_NVCC_EXTRA", "").split()
    BUILD.mkdir(exist_ok=True)
    stamp = BUILD / "liblbm_mix.stamp"
    digest = _digest(extra_flags)
    if not force and LIB.exists() and stamp.exists() and stamp.read_text() == digest:
        return LIB
    nvcc = _nvcc()
    objs = []

    def compile_one(src: Path):
        obj = BUILD / (src.stem + ".o")
        cmd = [nvcc, "-c", str(src), "-o", str(obj), "-I", str(INCLUDE), "-I", str(CSRC)] \
            + NVCC_FLAGS + list(extra_flags)
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src.name}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, flush=True)
        return obj

    srcs = _sources()
    workers = max(1, min(len(srcs), os.cpu_count() or 4))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB.with_suffix(".so.tmp")
    cmd = [nvcc, "-shared", "-o", str(tmp)] + [str(o) for o in objs] + ARCH + ["-cudart", "static"]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    stamp.write_text(digest)
    return LIB


if __name__ == "__main__":
    out = build(verbose="-v" in sys.argv, force="-f" in sys.argv)
    print(out)
