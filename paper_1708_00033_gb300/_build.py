"""Build of the CUDA library (libhf.so) for sm_103a, in-tree.

Runs the ERI code generator, compiles every translation unit with nvcc in
parallel (one -gencode, -O3 -lineinfo) and links a shared library with the
CUDA runtime linked statically.  Output: paper_1708_00033_gb300/_build/libhf.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
GEN = os.path.join(CSRC, "generated")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libhf.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", CSRC, "-I", INCLUDE]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def sources() -> list[str]:
    sys.path.insert(0, CSRC)
    try:
        import gen_eri  # noqa: E402
    finally:
        sys.path.pop(0)
    gen_eri.main(GEN)
    hand = [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith(".cu")]
    gen = [os.path.join(GEN, f) for f in sorted(os.listdir(GEN)) if f.endswith(".cu")]
    return hand + gen


def _deps_hash(src: str, extra: list[str]) -> str:
    h = hashlib.sha256()
    for path in [src] + extra:
        with open(path, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(ARCH + NVCC_FLAGS).encode())
    return h.hexdigest()[:16]


def build(verbose: bool = False, jobs: int | None = None, ptxas_verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    srcs = sources()
    headers = [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(INCLUDE, "hf.h"))
    exe = nvcc()
    objs = []
    todo = []
    for s in srcs:
        tag = _deps_hash(s, headers)
        obj = os.path.join(OUT, os.path.basename(s)[:-3] + f".{tag}.o")
        objs.append(obj)
        if not os.path.exists(obj):
            todo.append((s, obj))

    def compile_one(item):
        s, obj = item
        cmd = [exe] + ARCH + NVCC_FLAGS + (["-Xptxas", "-v"] if ptxas_verbose else []) + ["-c", s, "-o", obj + ".tmp"]
        t0 = time.time()
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {s}:\n{r.stderr}")
        os.replace(obj + ".tmp", obj)
        return s, time.time() - t0, r.stderr

    if todo:
        n = jobs or max(1, min(len(todo), os.cpu_count() or 4))
        with cf.ThreadPoolExecutor(n) as ex:
            for s, dt, err in ex.map(compile_one, todo):
                if verbose:
                    print(f"  {os.path.basename(s)}: {dt:.1f}s")
                if ptxas_verbose and err:
                    print(err)
    stamp = hashlib.sha256("".join(objs).encode()).hexdigest()[:16]
    stamp_file = LIB + ".stamp"
    if todo or not os.path.exists(LIB) or not os.path.exists(stamp_file) or open(stamp_file).read() != stamp:
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [exe] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
        with open(stamp_file, "w") as fh:
            fh.write(stamp)
    # drop stale objects
    keep = set(objs)
    for f in os.listdir(OUT):
        p = os.path.join(OUT, f)
        if f.endswith(".o") and p not in keep:
            os.remove(p)
    return LIB


if __name__ == "__main__":
    t = time.time()
    print(build(verbose=True, ptxas_verbose="-v" in sys.argv))
    print(f"built in {time.time() - t:.1f}s")
