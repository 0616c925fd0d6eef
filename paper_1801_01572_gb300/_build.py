"""Build of the CUDA library (liblsr.so) in-tree with nvcc for sm_103a.

Each translation unit under csrc/ is compiled in parallel, then linked into
one shared library with the CUDA runtime linked statically. Objects are rebuilt
when a source, a header or the flags change.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "liblsr.so")
CHECKED_LIB = os.path.join(OUT, "liblsr_checked.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
FLAGS = [ARCH, "-O3", "-lineinfo", "-std=c++17", "--expt-extended-lambda", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-fvisibility=hidden", f"-I{os.path.join(ROOT, 'include')}"]


def _nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblsr")
    return exe


def _digest(paths, extra) -> str:
    h = hashlib.sha256(" ".join(extra).encode())
    for p in sorted(paths):
        with open(p, "rb") as f:
            h.update(p.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile csrc/*.cu for sm_103a and link _lib/liblsr.so; returns its path.
    checked=True builds _lib/liblsr_checked.so instead: the same sources with
    LSR_CHECKED defined (device bounds checks that report instead of trapping)."""
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    flags = FLAGS + (["-DLSR_CHECKED"] if checked else [])
    lib = CHECKED_LIB if checked else LIB
    suffix = ".chk" if checked else ""
    headers = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    objs, jobs = [], []
    for src in sources:
        tag = _digest([src] + headers, flags)
        obj = os.path.join(OUT, os.path.basename(src)[:-3] + f"{suffix}.{tag}.o")
        objs.append(obj)
        if force or not os.path.exists(obj):
            jobs.append([nvcc, *flags, "-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stderr}")
        if verbose and r.stderr.strip():
            print(r.stderr)

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(run, jobs))
    link_tag = _digest(objs, flags)
    stamp = lib + ".stamp"
    if force or not os.path.exists(lib) or not os.path.exists(stamp) or open(stamp).read() != link_tag:
        tmp = lib + f".tmp{os.getpid()}"
        run([nvcc, ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs])
        os.replace(tmp, lib)
        with open(stamp, "w") as f:
            f.write(link_tag)
    # drop objects of older source versions of this build
    keep = set(objs)
    for o in glob.glob(os.path.join(OUT, "*.o")):
        if o not in keep and (o.split(".")[-3] == "chk") == checked:
            os.remove(o)
    return lib


if __name__ == "__main__":
    print(build(verbose=True))
