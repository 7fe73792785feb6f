"""ctypes binding of the plain C oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; the product path never imports it.  It shares no code
with the CUDA path.  Every function below returns numpy arrays in the layouts documented in
``oracle.h`` (D innermost; messages [4][H][W][D] indexed by the neighbour they come from:
up, down, left, right).
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC"]


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, a second or two); with `openmp`, the
    timing build liboracle_omp.so (same source and results, threads over pixels)."""
    out = _LIB_OMP if openmp else _LIB
    stale = (not os.path.exists(out)) or os.path.getmtime(out) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h")))
    if force or stale:
        tmp = out + f".{os.getpid()}.tmp"
        flags = CFLAGS + (["-fopenmp"] if openmp else [])
        subprocess.check_call(["gcc", *flags, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, out)
    return out


_libs: dict[bool, ctypes.CDLL] = {}
_use_openmp = False


def openmp_available() -> bool:
    """Whether the OpenMP build compiles and loads here."""
    try:
        _load(True)
        return True
    except (OSError, subprocess.CalledProcessError):
        return False


@contextlib.contextmanager
def openmp(threads: int = 0):
    """Inside the block every oracle call runs on the OpenMP build with `threads` threads (0:
    the OpenMP default); yields the thread count in use."""
    global _use_openmp
    n = _load(True).oracle_threads(threads)
    prev, _use_openmp = _use_openmp, True
    try:
        yield n
    finally:
        _use_openmp = prev


def lib() -> ctypes.CDLL:
    return _load(_use_openmp)


def _load(openmp_build: bool) -> ctypes.CDLL:
    if openmp_build not in _libs:
        _lib = ctypes.CDLL(build(openmp=openmp_build))
        P = ctypes.c_void_p
        i, i64, u64, d = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        sig = {
            "oracle_ncc": (i, [P, P, i, i, i, i, P]),
            "oracle_quantise": (i, [P, i64, i, P]),
            "oracle_cost_float": (i, [P, i64, i, P]),
            "oracle_level_dims": (i, [i, i, i, P, P]),
            "oracle_pyramid_i32": (i, [P, i, i, i, i, P]),
            "oracle_pyramid_f64": (i, [P, i, i, i, i, P]),
            "oracle_message_i32": (None, [P, i, i, i, P]),
            "oracle_message_f64": (None, [P, i, d, i, P]),
            "oracle_bp_i32": (i, [P, i, i, i, i, i, i, i, i, P, u64, P, P]),
            "oracle_bp_f64": (i, [P, i, i, i, i, i, d, i, i, P, u64, P, P]),
            "oracle_bp_rule_i32": (i, [P, i, i, i, i, i, i, i, i, i, i, P, u64, P, P]),
            "oracle_bp_rule_f64": (i, [P, i, i, i, i, i, d, i, i, d, i, P, u64, P, P]),
            "oracle_bp_wta_i32": (i, [P, i, i, i, i, i, i, i, i, P, P]),
            "oracle_bp_schedule_i32": (i, [P, i, i, i, i, P, i, i, i, P, P, P]),
            "oracle_bp_wta_f64": (i, [P, i, i, i, i, i, d, i, i, P, P]),
            "oracle_candidates": (i, [P, i, i, i, i, P]),
            "oracle_bp_sparse_i32": (i, [P, i, i, i, i, i, i, i, i, i, P, P, P]),
            "oracle_wta_sparse_i32": (i, [P, P, P, i, i, i, i, P]),
            "oracle_wta_i32": (i, [P, P, i, i, i, P]),
            "oracle_wta_f64": (i, [P, P, i, i, i, P]),
            "oracle_energy_i32": (i64, [P, P, i, i, i, i, i]),
            "oracle_energy_f64": (d, [P, P, i, i, i, d, i]),
            "oracle_threads": (i, [i]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
        _libs[openmp_build] = _lib
    return _libs[openmp_build]


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"{what}: invalid arguments")


def ncc(L: np.ndarray, R: np.ndarray, D: int, window: int) -> np.ndarray:
    L = np.ascontiguousarray(L, dtype=np.uint8)
    R = np.ascontiguousarray(R, dtype=np.uint8)
    H, W = L.shape
    out = np.empty((H, W, D), dtype=np.float64)
    _check(lib().oracle_ncc(_p(L), _p(R), W, H, D, window, _p(out)), "oracle_ncc")
    return out


def quantise(ncc_vol: np.ndarray, trunc_data: int) -> np.ndarray:
    a = np.ascontiguousarray(ncc_vol, dtype=np.float64)
    out = np.empty(a.shape, dtype=np.int32)
    _check(lib().oracle_quantise(_p(a), a.size, trunc_data, _p(out)), "oracle_quantise")
    return out


def cost_float(ncc_vol: np.ndarray, trunc_data: int) -> np.ndarray:
    a = np.ascontiguousarray(ncc_vol, dtype=np.float64)
    out = np.empty(a.shape, dtype=np.float64)
    _check(lib().oracle_cost_float(_p(a), a.size, trunc_data, _p(out)), "oracle_cost_float")
    return out


def level_dims(W: int, H: int, levels: int) -> list[tuple[int, int]]:
    Ws = np.zeros(levels, dtype=np.int32)
    Hs = np.zeros(levels, dtype=np.int32)
    if lib().oracle_level_dims(W, H, levels, _p(Ws), _p(Hs)) < 0:
        raise ValueError("bad dims")
    return [(int(w), int(h)) for w, h in zip(Ws, Hs)]


def pyramid(cost0: np.ndarray, levels: int) -> list[np.ndarray]:
    H, W, D = cost0.shape
    dims = level_dims(W, H, levels)
    total = sum(w * h * D for w, h in dims)
    if cost0.dtype == np.int32:
        a = np.ascontiguousarray(cost0)
        out = np.empty(total, dtype=np.int32)
        _check(lib().oracle_pyramid_i32(_p(a), W, H, D, levels, _p(out)), "oracle_pyramid_i32")
    else:
        a = np.ascontiguousarray(cost0, dtype=np.float64)
        out = np.empty(total, dtype=np.float64)
        _check(lib().oracle_pyramid_f64(_p(a), W, H, D, levels, _p(out)), "oracle_pyramid_f64")
    res, off = [], 0
    for w, h in dims:
        res.append(out[off: off + w * h * D].reshape(h, w, D))
        off += w * h * D
    return res


def message(h: np.ndarray, lam, trunc: int) -> np.ndarray:
    if h.dtype == np.int32:
        a = np.ascontiguousarray(h)
        out = np.empty_like(a)
        lib().oracle_message_i32(_p(a), a.size, int(lam), trunc, _p(out))
    else:
        a = np.ascontiguousarray(h, dtype=np.float64)
        out = np.empty_like(a)
        lib().oracle_message_f64(_p(a), a.size, float(lam), trunc, _p(out))
    return out


def bp(cost0: np.ndarray, levels: int, iters: int, lam, trunc: int, skip: bool = True,
       init_coarsest: np.ndarray | None = None, order_seed: int = 0, eps=0, freeze: bool = False):
    """Hierarchical min-sum BP.  Returns (finest messages [4][H][W][D], trace per half-sweep).
    eps / freeze: the approximate skip rule (0 / False: the exact skip)."""
    H, W, D = cost0.shape
    ntrace = levels * iters * 2
    trace = np.zeros(max(ntrace, 1), dtype=np.int64)
    if cost0.dtype == np.int32:
        a = np.ascontiguousarray(cost0)
        out = np.empty((4, H, W, D), dtype=np.int32)
        init = None if init_coarsest is None else np.ascontiguousarray(init_coarsest, dtype=np.int32)
        rc = lib().oracle_bp_rule_i32(_p(a), W, H, D, levels, iters, int(lam), trunc, int(skip), int(eps),
                                      int(freeze), _p(init), order_seed, _p(out), _p(trace))
    else:
        a = np.ascontiguousarray(cost0, dtype=np.float64)
        out = np.empty((4, H, W, D), dtype=np.float64)
        init = None if init_coarsest is None else np.ascontiguousarray(init_coarsest, dtype=np.float64)
        rc = lib().oracle_bp_rule_f64(_p(a), W, H, D, levels, iters, float(lam), trunc, int(skip), float(eps),
                                      int(freeze), _p(init), order_seed, _p(out), _p(trace))
    _check(rc, "oracle_bp")
    return out, trace[:ntrace]


def bp_schedule(cost0: np.ndarray, iters, lam: int, trunc: int, skip: bool = True,
                init_coarsest: np.ndarray | None = None):
    """Hierarchical BP (integer costs) with iters[l] iterations at scale l (0 = the finest); the
    number of scales is len(iters).  Returns (finest messages [4][H][W][D], trace per half-sweep)."""
    H, W, D = cost0.shape
    its = np.ascontiguousarray(iters, dtype=np.int32)
    levels = len(its)
    ntrace = int(2 * its.sum())
    trace = np.zeros(max(ntrace, 1), dtype=np.int64)
    out = np.empty((4, H, W, D), dtype=np.int32)
    init = None if init_coarsest is None else np.ascontiguousarray(init_coarsest, dtype=np.int32)
    _check(lib().oracle_bp_schedule_i32(_p(np.ascontiguousarray(cost0, dtype=np.int32)), W, H, D, levels, _p(its),
                                        int(lam), trunc, int(skip), _p(init), _p(out), _p(trace)), "oracle_bp_schedule")
    return out, trace[:ntrace]


def bp_wta(cost0: np.ndarray, levels: int, iters: int, lam, trunc: int, skip: bool = True):
    """Hierarchical BP (exact skip, zero start) and the read-out, without the messages: the same
    results as bp() then wta() in half the host memory.  Returns (disparities [H][W], trace)."""
    H, W, D = cost0.shape
    ntrace = levels * iters * 2
    trace = np.zeros(max(ntrace, 1), dtype=np.int64)
    disp = np.empty((H, W), dtype=np.int32)
    if cost0.dtype == np.int32:
        rc = lib().oracle_bp_wta_i32(_p(np.ascontiguousarray(cost0)), W, H, D, levels, iters, int(lam), trunc,
                                     int(skip), _p(disp), _p(trace))
    else:
        rc = lib().oracle_bp_wta_f64(_p(np.ascontiguousarray(cost0, dtype=np.float64)), W, H, D, levels, iters,
                                     float(lam), trunc, int(skip), _p(disp), _p(trace))
    _check(rc, "oracle_bp_wta")
    return disp, trace[:ntrace]


def candidates(cost0: np.ndarray, K: int) -> np.ndarray:
    """The K labels of lowest cost per pixel, in increasing label order, int32 [H][W][K]."""
    H, W, D = cost0.shape
    out = np.empty((H, W, K), dtype=np.int32)
    _check(lib().oracle_candidates(_p(np.ascontiguousarray(cost0, dtype=np.int32)), W, H, D, K, _p(out)),
           "oracle_candidates")
    return out


def bp_sparse(cost0: np.ndarray, levels: int, iters: int, lam: int, trunc: int, K: int, skip: bool = True):
    """Hierarchical BP with K candidates per pixel at the finest scale.  Returns (candidates
    [H][W][K], finest messages [4][H][W][K], trace per half-sweep)."""
    H, W, D = cost0.shape
    ntrace = levels * iters * 2
    trace = np.zeros(max(ntrace, 1), dtype=np.int64)
    cand = np.empty((H, W, K), dtype=np.int32)
    msg = np.empty((4, H, W, K), dtype=np.int32)
    _check(lib().oracle_bp_sparse_i32(_p(np.ascontiguousarray(cost0, dtype=np.int32)), W, H, D, levels, iters,
                                      int(lam), trunc, int(skip), K, _p(cand), _p(msg), _p(trace)), "oracle_bp_sparse")
    return cand, msg, trace[:ntrace]


def wta_sparse(cost0: np.ndarray, cand: np.ndarray, msg: np.ndarray) -> np.ndarray:
    H, W, D = cost0.shape
    K = cand.shape[2]
    out = np.empty((H, W), dtype=np.int32)
    _check(lib().oracle_wta_sparse_i32(_p(np.ascontiguousarray(cost0, dtype=np.int32)),
                                       _p(np.ascontiguousarray(cand, dtype=np.int32)),
                                       _p(np.ascontiguousarray(msg, dtype=np.int32)), W, H, D, K, _p(out)),
           "oracle_wta_sparse")
    return out


def wta(cost0: np.ndarray, msg0: np.ndarray) -> np.ndarray:
    H, W, D = cost0.shape
    out = np.empty((H, W), dtype=np.int32)
    if cost0.dtype == np.int32:
        rc = lib().oracle_wta_i32(_p(np.ascontiguousarray(cost0)),
                                  _p(np.ascontiguousarray(msg0, dtype=np.int32)), W, H, D, _p(out))
    else:
        rc = lib().oracle_wta_f64(_p(np.ascontiguousarray(cost0, dtype=np.float64)),
                                  _p(np.ascontiguousarray(msg0, dtype=np.float64)), W, H, D, _p(out))
    _check(rc, "oracle_wta")
    return out


def energy(cost0: np.ndarray, disp: np.ndarray, lam, trunc: int):
    H, W, D = cost0.shape
    dsp = np.ascontiguousarray(disp, dtype=np.int32)
    if cost0.dtype == np.int32:
        e = lib().oracle_energy_i32(_p(np.ascontiguousarray(cost0)), _p(dsp), W, H, D, int(lam), trunc)
        if e == np.iinfo(np.int64).min:
            raise ValueError("labels out of range")
        return int(e)
    e = lib().oracle_energy_f64(_p(np.ascontiguousarray(cost0, dtype=np.float64)), _p(dsp), W, H, D,
                                float(lam), trunc)
    if np.isnan(e):
        raise ValueError("labels out of range")
    return float(e)


def stereo_int(L: np.ndarray, R: np.ndarray, D: int, window: int, trunc_data: int, levels: int,
               iters: int, lam: int, trunc: int, skip: bool = True):
    """The whole integer path: cost volume, BP, WTA and energy."""
    c = quantise(ncc(L, R, D, window), trunc_data)
    msg, trace = bp(c, levels, iters, lam, trunc, skip)
    d = wta(c, msg)
    return {"cost": c, "msg": msg, "trace": trace, "disp": d, "energy": energy(c, d, lam, trunc)}


def stereo_f64(L: np.ndarray, R: np.ndarray, D: int, window: int, trunc_data: int, levels: int,
               iters: int, lam: float, trunc: int, skip: bool = True):
    """The FP64 reference of the float-message path (no quantisation of the data cost)."""
    c = cost_float(ncc(L, R, D, window), trunc_data)
    msg, trace = bp(c, levels, iters, lam, trunc, skip)
    d = wta(c, msg)
    return {"cost": c, "msg": msg, "trace": trace, "disp": d, "energy": energy(c, d, lam, trunc)}
