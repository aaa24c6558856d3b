"""Build the CE search library libgce.so in-tree with nvcc for sm_103a.

Each .cu file under csrc/ is compiled in parallel into an object file, then
linked into paper_2006_06866_gb300/_lib/libgce.so (CUDA runtime linked
statically).  Run ``python -m paper_2006_06866_gb300.build`` or call
``build()``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libgce.so")
CHECKED_MARK = os.path.join(OUT_DIR, "CHECKED")  # present while LIB is a checked build
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              *ARCH]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [
        os.path.join(HERE, "..", "include", "gce.h"), __file__]


def up_to_date() -> bool:
    if not os.path.exists(LIB) or os.path.exists(CHECKED_MARK):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False,
          checked: bool = False) -> str:
    """checked: compile the counter-slot bounds check into the hot loop (every
    increment's slot tested against the trial's kept range; a miss is reported
    by gce_stream_status and the access skipped).  For verification runs only:
    it costs a few instructions per point-trial."""
    if not force and not checked and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tool = nvcc()
    objs = []
    extra = (["-Xptxas", "-v"] if ptxas_info else []) + (["-DGCE_CHECK_SLOTS"] if checked else [])

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + ".o")
        cmd = [tool, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        for obj, log in ex.map(compile_one, _sources()):
            objs.append(obj)
            if (verbose or ptxas_info) and log:
                sys.stderr.write(log)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [tool, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    for o in objs:
        os.remove(o)
    if checked:
        open(CHECKED_MARK, "w").close()
    elif os.path.exists(CHECKED_MARK):
        os.remove(CHECKED_MARK)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv,
                checked="--checked" in sys.argv))
