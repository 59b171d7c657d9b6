"""Compile the CUDA sources of this package into an in-tree shared library.

Each translation unit is compiled for sm_103a by its own nvcc process (in parallel),
then linked into ``_build/libmvp.so``. The library is rebuilt when a source or
header changes (content hash in the file name).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
ROOT = os.path.dirname(HERE)
HEADER = os.path.join(ROOT, "include", "mvp.h")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xcompiler", "-fvisibility=hidden"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _digest() -> str:
    h = hashlib.sha1()
    files = _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [HEADER]
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(ARCH + NVCC_FLAGS).encode())
    return h.hexdigest()[:16]


def sources_digest(names: list[str]) -> str:
    """Digest of some of the library's sources (file names relative to csrc/, or the
    header's name) with the compile flags: identifies the build of one kernel."""
    h = hashlib.sha1()
    for name in names:
        f = HEADER if name == os.path.basename(HEADER) else os.path.join(CSRC, name)
        h.update(name.encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(ARCH + NVCC_FLAGS).encode())
    return h.hexdigest()[:16]


def library_path(checked: bool = False) -> str:
    return os.path.join(BUILD, f"libmvp_{_digest()}{'_checked' if checked else ''}.so")


def build(verbose: bool = False, extra_flags: list[str] | None = None, checked: bool = False) -> str:
    """Build (if needed) and return the path of libmvp.so. checked: the variant with
    device-side bounds checks (-DMVP_CHECK_BOUNDS), a library of its own."""
    out = library_path(checked)
    if os.path.exists(out) and not extra_flags:
        return out
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    flags = ARCH + NVCC_FLAGS + (["-DMVP_CHECK_BOUNDS"] if checked else []) + (extra_flags or [])
    objs = []
    jobs = []
    for src in _sources():
        obj = os.path.join(BUILD, os.path.basename(src) + f".{os.getpid()}.o")
        objs.append(obj)
        jobs.append([nvcc, *flags, "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
    for cmd, r in zip(jobs, results):
        if verbose and r.stderr:
            print(r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    tmp = out + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    for o in objs:
        os.remove(o)
    # libraries of earlier sources are stale (a process that loaded one keeps its mapping)
    for old in glob.glob(os.path.join(BUILD, "libmvp_*.so")):
        if old not in (library_path(False), library_path(True)):
            try:
                os.remove(old)
            except OSError:
                pass
    return out


if __name__ == "__main__":
    print(build(verbose=True))
