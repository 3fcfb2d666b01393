"""In-tree build of libdlsh.so (the C-ABI CUDA library) for sm_103a.

Every translation unit under csrc/ is compiled by nvcc in parallel into
_build/<machine>/ and linked into paper_2605_30396_gb300/libdlsh.so.  A stamp
file records the host machine type and a hash of the sources, so a library built
on another architecture or from other sources is rebuilt, never loaded.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import platform
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
SO_PATH = os.path.join(PKG, "libdlsh.so")
STAMP = os.path.join(PKG, "libdlsh.stamp")
SOURCES = ["api.cu", "encode.cu", "enc_one_fp32.cu", "enc_one_lowp.cu", "enc_pair.cu", "enc_split.cu", "decode.cu", "mod.cu", "learn.cu", "noalloc.cu", "mlp.cu", "propose.cu", "learned.cu", "selftest.cu", "splat.cu"]
ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdlsh.so")


def _sources():
    return [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]


def _digest() -> str:
    h = hashlib.sha256()
    h.update(platform.machine().encode())
    h.update(" ".join(ARCH_FLAGS + CFLAGS).encode())
    files = sorted(os.listdir(CSRC)) + ["../../include/dlsh.h"]
    for f in files:
        p = os.path.normpath(os.path.join(CSRC, f))
        if p.endswith((".cu", ".cuh", ".hpp", ".h")) and os.path.isfile(p):
            h.update(f.encode())
            with open(p, "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()


def is_current() -> bool:
    if not (os.path.exists(SO_PATH) and os.path.exists(STAMP)):
        return False
    with open(STAMP) as fh:
        return fh.read().strip() == _digest()


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libdlsh.so; returns its path."""
    if not force and is_current():
        return SO_PATH
    nvcc = _nvcc()
    obj_dir = os.path.join(PKG, "_build", platform.machine())
    os.makedirs(obj_dir, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(obj_dir, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH_FLAGS, *CFLAGS, "-I", INCLUDE, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = SO_PATH + ".tmp"
    cmd = [nvcc, *ARCH_FLAGS, "-shared", "-cudart", "shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, SO_PATH)
    with open(STAMP, "w") as fh:
        fh.write(_digest())
    return SO_PATH


if __name__ == "__main__":
    print(build(force=True, verbose=True))
