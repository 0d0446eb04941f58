"""Build the in-tree shared library libhmm_gb300.so for sm_103a with nvcc.

The translation units are compiled in parallel, then linked with
``nvcc -shared``. Objects go to ``_build/`` next to this file; the library is
written next to this file so that the binding loads it from the source tree.

The rebuild decision is keyed on a SHA-256 of every file under csrc/ and
include/, the compile flags, the nvcc version and the host architecture, stored beside the library in
libhmm_gb300.so.sha256: a library copied in with the tree (built elsewhere, or
for another machine) is rebuilt unless its recorded hash matches this tree and
this compiler. Each call prints one line saying whether it compiled.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhmm_gb300.so")
STAMP = LIB + ".sha256"
SOURCES = ["hmm_api.cu", "macro.cu", "micro_fp64.cu", "micro_fp32.cu", "micro_fp32_2d.cu", "noalloc.cu",
           "res2d_pack.cu", "res2d_cluster_a.cu", "res2d_cluster_b.cu", "res2d_any.cu", "res2d_rk4.cu", "res2d_tr2.cu",
           "res3d.cu", "dns.cu", "fma_rate.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhmm_gb300.so")


def _source_hash(nvcc: str) -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for f in sorted(os.listdir(d)):
            h.update(f.encode())
            with open(os.path.join(d, f), "rb") as fh:
                h.update(fh.read())
    h.update(" ".join(SOURCES + ARCH + FLAGS[:-1]).encode())   # flags without the include path
    ver = subprocess.run([nvcc, "--version"], capture_output=True, text=True).stdout
    h.update(ver.encode())
    h.update(platform.machine().encode())   # a library built on another host architecture never matches
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (unless the recorded source hash matches) and return the path of libhmm_gb300.so.

    Concurrent calls (test workers in parallel processes) are serialised by a lock
    file beside the library: one compiles, the others then find the library current."""
    import fcntl
    with open(LIB + ".lock", "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        try:
            return _build_locked(force, verbose)
        finally:
            fcntl.flock(lock, fcntl.LOCK_UN)


def _build_locked(force: bool, verbose: bool) -> str:
    nvcc = _nvcc()
    digest = _source_hash(nvcc)
    if not force and os.path.exists(LIB) and os.path.exists(STAMP):
        with open(STAMP) as fh:
            if fh.read().strip() == digest:
                print(f"libhmm_gb300.so up to date (sources {digest[:12]})", file=sys.stderr)
                return LIB
    os.makedirs(BUILD, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(STAMP, "w") as fh:
        fh.write(digest + "\n")
    print(f"libhmm_gb300.so compiled from source (sources {digest[:12]})", file=sys.stderr)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
