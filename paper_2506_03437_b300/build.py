"""Compiles the CUDA sources into the in-tree shared library libquake_b300.so.

    python -m paper_2506_03437_b300.build [--force]

Targets sm_103a only (B300).  nvcc cross-compiles, so this runs without a GPU.
Each source compiles to its own object under _build/ (in parallel, and only
when the source, a header or the flags changed); the objects are then linked.
"""

import concurrent.futures
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libquake_b300.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OBJDIR = os.path.join(HERE, "_build")

SEARCH_DIMS = [32, 64, 96, 128, 192, 256, 384, 512, 768, 1024]
SOURCES = (["capi.cu", "search.cu", "kmeans.cu", "arena.cu", "update.cu", "maintain.cu", "quant.cu", "tc_score.cu",
            "noalloc.cu", "batch.cu", "aps_batch.cu", "server.cu", "profile.cu", "checkpoint.cu",
            "views.cu"] + [f"search_d{d}.cu" for d in SEARCH_DIMS])
HEADERS = ["common.cuh", "capvol.cuh", "index.cuh", "trace.h", "search_impl.cuh", "devmem.h", "grouped.cuh", "tc_common.cuh", "aps_prepare.cuh"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMPILE_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]
LINK_FLAGS = ARCH + ["-shared", "-cudart", "shared"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _headers():
    hs = [os.path.join(CSRC, f) for f in HEADERS]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return hs


def _obj(src, tag):
    return os.path.join(OBJDIR, f"{os.path.splitext(src)[0]}.{tag}.o")


def build(force=False, verbose=False, extra=()):
    """Builds the library if a source or header is newer than it; returns its path."""
    extra = list(extra)
    tag = hashlib.sha1(" ".join(COMPILE_FLAGS + extra).encode()).hexdigest()[:10]
    os.makedirs(OBJDIR, exist_ok=True)
    newest_header = max(os.path.getmtime(h) for h in _headers())
    todo = []
    for src in SOURCES:
        o = _obj(src, tag)
        path = os.path.join(CSRC, src)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(path), newest_header):
            todo.append(src)
    objs = [_obj(src, tag) for src in SOURCES]
    if not todo and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(o) for o in objs):
        return LIB

    def compile_one(src):
        o = _obj(src, tag)
        # the object is stamped with the inputs' time taken before compiling, so an
        # edit made while it compiles still counts as newer
        stamp = max(os.path.getmtime(os.path.join(CSRC, src)), newest_header)
        cmd = [_nvcc()] + COMPILE_FLAGS + extra + ["-I", INCLUDE, "-c", os.path.join(CSRC, src), "-o", o + ".tmp"]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)
        os.replace(o + ".tmp", o)
        os.utime(o, (stamp, stamp))

    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as pool:
        for f in [pool.submit(compile_one, s) for s in todo]:
            f.result()
    cmd = [_nvcc()] + LINK_FLAGS + objs + ["-o", LIB + ".tmp"]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    extra = [a for a in sys.argv[1:] if a.startswith("-X")]
    build(force="--force" in sys.argv, verbose=True, extra=extra)
    print(LIB)
