"""Builds libbm.so (the BlockMGARD CUDA library) in-tree for sm_103a.

Each CUDA translation unit is compiled by its own nvcc process (in parallel),
the host plan code by g++ without floating-point contraction, and everything
is linked into ``_lib/libbm.so`` with the static CUDA runtime.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libbm.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

CU_SOURCES = [
    "bm_api.cu",
    "bm_block_f32_b9.cu",
    "bm_block_f32_b17.cu",
    "bm_block_f64_b9.cu",
    "bm_block_f64_b17.cu",
    "bm_adjoint_f32.cu",
    "bm_adjoint_f64.cu",
]
CPP_SOURCES = ["bm_plan.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "--expt-relaxed-constexpr", "-O3", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
              "-I" + INCLUDE]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    srcs = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    srcs.append(os.path.join(INCLUDE, "blockmgard.h"))
    srcs.append(os.path.abspath(__file__))
    return srcs


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, jobs: int | None = None, out: str | None = None,
          defines: tuple = ()) -> str:
    """Compile and link libbm.so (into ``out`` if given, with extra -D
    ``defines``)."""
    lib = out or LIB
    if not force and out is None and not defines and up_to_date():
        return LIB
    out_dir = os.path.dirname(lib)
    os.makedirs(out_dir, exist_ok=True)
    obj_dir = os.path.join(out_dir, "obj")
    os.makedirs(obj_dir, exist_ok=True)
    nvcc = _nvcc()
    cmds = []
    objs = []
    for src in CU_SOURCES:
        obj = os.path.join(obj_dir, src.replace(".cu", ".o"))
        objs.append(obj)
        cmds.append([nvcc, *NVCC_FLAGS, *["-D" + d for d in defines], *ARCH, "-c", os.path.join(CSRC, src), "-o", obj])
    for src in CPP_SOURCES:
        obj = os.path.join(obj_dir, src.replace(".cpp", ".o"))
        objs.append(obj)
        cmds.append(["g++", "-std=c++17", "-O2", "-fPIC", "-ffp-contract=off", "-fno-fast-math", "-c",
                     os.path.join(CSRC, src), "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=jobs or min(len(cmds), os.cpu_count() or 4)) as ex:
        for out in ex.map(run, cmds):
            if verbose and out.strip():
                print(out)
    tmp = lib + ".tmp%d" % os.getpid()
    run([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
