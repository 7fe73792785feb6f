"""Build the CUDA library libbpstereo.so in-tree with nvcc (sm_103a only), and its debug twin
libbpstereo_debug.so (-DBPS_DEBUG_BOUNDS: device-side bounds checks that report through
bps_get_error instead of accessing out of bounds).

Every translation unit (SOURCES) compiles in parallel, then nvcc links them into a shared
library next to this file.  Nothing is installed anywhere else.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libbpstereo.so")
LIB_DEBUG = os.path.join(HERE, "libbpstereo_debug.so")
BUILD_DIR = os.path.join(ROOT, "_build")
SOURCES = ["api.cu", "ncc.cu", "bp.cu", "readout.cu", "persist.cu", "noalloc.cu", "warmnet.cu", "sparse.cu", "sweep_f16.cu", "conv_tc.cu", "ncc_tc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbpstereo.so")
    return path


def _inputs() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    return files + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]


def is_stale(path: str = LIB) -> bool:
    if not os.path.exists(path):
        return True
    t = os.path.getmtime(path)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Build libbpstereo.so if stale (and, with debug, libbpstereo_debug.so too, in the same pool
    of compile jobs); returns the path of libbpstereo.so."""
    targets = [(LIB, [], "release")]
    if debug:
        targets.append((LIB_DEBUG, ["-DBPS_DEBUG_BOUNDS"], "debug"))
    targets = [t for t in targets if force or is_stale(t[0])]
    if not targets:
        return LIB
    cc = nvcc()

    def compile_one(job) -> str:
        src, extra, tag = job
        out_dir = os.path.join(BUILD_DIR, tag)
        os.makedirs(out_dir, exist_ok=True)
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src} ({tag}):\n{res.stderr}")
        if verbose and res.stderr:
            print(res.stderr)
        return obj

    jobs = [(src, extra, tag) for _, extra, tag in targets for src in SOURCES]
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 8)) as ex:
        objs = list(ex.map(compile_one, jobs))
    for k, (lib, _, _) in enumerate(targets):
        tmp = lib + f".{os.getpid()}.tmp"
        mine = objs[k * len(SOURCES):(k + 1) * len(SOURCES)]
        res = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *mine], capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc link failed:\n{res.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True, debug=True))
