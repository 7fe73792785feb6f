"""GB300-native stereo hot path of arXiv 1709.06509: NCC matching-cost volume, 4-scale
coarse-to-fine min-sum loopy BP with a truncated-linear smoothness term and the
fast-converging skip, winner-take-all disparity.

This module is a thin ctypes binding of the C ABI declared in ``include/bpstereo.h``
(library ``libbpstereo.so`` next to this file).  Every step of the path runs in the CUDA
kernels behind that ABI; this file only marshals arguments.  PyTorch is used for device
memory and streams.  If the library is missing, ``lib()`` raises: there is no CPU
fallback.

The ``bps_*`` functions mirror the C entry points one to one (same names, same argument
order, tensors or raw device addresses for pointers, a CUDA stream or None for the
current stream).  ``Stereo`` wraps one context and its workspace tensor.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

LIB_PATH = _build.LIB
LIB_DEBUG_PATH = _build.LIB_DEBUG

BPS_OK = 0
BPS_ERR_ARG = -1
BPS_ERR_UNSUPPORTED = -2
BPS_ERR_CUDA = -3
BPS_ERR_WORKSPACE = -4
BPS_ERR_TIMEOUT = -5
BPS_ERR_STATE = -6
BPS_ERR_INTERNAL = -7

BPS_MSG_INT32 = 0
BPS_MSG_U8 = 1
BPS_MSG_FP16 = 2

BPS_FLAG_FAST_SKIP = 1
BPS_FLAG_WARM_START = 2
BPS_FLAG_GRAPH = 4
BPS_FLAG_PROFILE = 8
BPS_FLAG_PERSISTENT = 16
BPS_FLAG_TEST_TIMEOUT = 32
BPS_FLAG_ASYNC = 64

BPS_MAX_LEVELS = 8
BPS_MAX_D = 512
BPS_MAX_ITERS = 1024
BPS_MAX_CANDIDATES = 32
BPS_MAX_WINDOW = 31
BPS_MAX_BATCH = 256
BPS_VARIANT_GENERAL_DT = 1
BPS_VARIANT_LISTS = 2
BPS_VARIANT_CLUSTER = 4
BPS_VARIANT_EAGER = 8
BPS_VARIANT_DPAR = 16
BPS_VARIANT_DPAR_LISTS = 32
BPS_VARIANT_STAGED = 64
BPS_VARIANT_STAGED_LISTS = 128
BPS_VARIANT_BULK = 256
BPS_VARIANT_BULK_LISTS = 512
BPS_VARIANT_BLOCK2 = 1024
BPS_NCC_DEFAULT = 0
BPS_NCC_ROWS = 1
BPS_NCC_TENSOR = 2
BPS_NOALLOC_MAX_BLOCKS = 16384
BPS_NOALLOC_MAX_PIXELS = BPS_NOALLOC_MAX_BLOCKS * 1024


class BPSError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = f"{what}: {status_string(status)} ({status})"
        if status == BPS_ERR_CUDA:
            code = lib().bps_last_cuda_error()
            msg += f": {lib().bps_cuda_error_string(code).decode()} ({code})"
        super().__init__(msg)


_lib = None

_P, _I, _SZ, _I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_int64
_SIGS = {
    "bps_status_string": (ctypes.c_char_p, [_I]),
    "bps_workspace_bytes": (_SZ, [_I, _I, _I, _I, _I]),
    "bps_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, _I, _I, _P, _SZ]),
    "bps_destroy": (_I, [_P]),
    "bps_build_cost_volume": (_I, [_P, _P, _P, _I, _I, _I, _P, _P]),
    "bps_bp_solve": (_I, [_P, _I, _I, _I, _I, _I, _P, _P]),
    "bps_wta_disparity": (_I, [_P, _P, _P]),
    "bps_energy": (_I, [_P, _P, _I, _I, _P, _P, _P]),
    "bps_stereo": (_I, [_P, _P, _P, _I, _I, _I, _I, _I, _I, _I, _P, _P]),
    "bps_stereo_host": (_I, [_P, _P, _P, _I, _I, _I, _I, _I, _I, _I, _P, _P, _P, _P]),
    "bps_get_trace": (_I, [_P, _P, _I]),
    "bps_export_messages": (_I, [_P, _I, _P, _P]),
    "bps_export_cost": (_I, [_P, _I, _P, _P]),
    "bps_read_profile": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I64)]),
    "bps_read_launch_times": (_I, [_P, _P, _I]),
    "bps_get_error": (_I, [_P]),
    "bps_last_cuda_error": (_I, []),
    "bps_cuda_error_string": (ctypes.c_char_p, [_I]),
    "bps_energy_noalloc": (_I, [_P, _P, _I, _I, _I, _I, _I, _P, _P]),
    "bps_test_fail_resources": (_I, [_I]),
    "bps_bp_solve_schedule": (_I, [_P, _I, _P, _I, _I, _I, _P, _P]),
    "bps_warmnet_get_error": (_I, []),
    "bps_measure_sync_costs": (_I, [_I, _I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "bps_batch_create": (_I, [ctypes.POINTER(_P), _P, _I]),
    "bps_batch_destroy": (_I, [_P]),
    "bps_batch_stereo": (_I, [_P, _P, _P, _P, _P, _I, _I, _I, _I, _I, _P, _P]),
    "bps_batch_get_error": (_I, [_P]),
    "bps_batch_stereo_host": (_I, [_P, _P, _P, _P, _P, _I, _I, _I, _I, _I, _P, _P, _P]),
    "bps_set_sweep_variant": (_I, [_P, _I, _I]),
    "bps_get_sweep_variant": (_I, [_P, _I]),
    "bps_set_skip_rule": (_I, [_P, _I, _I]),
    "bps_set_candidates": (_I, [_P, _I]),
    "bps_export_sparse": (_I, [_P, _P, _P, _P]),
    "bps_set_ncc_shape": (_I, [_P, _I, _I]),
    "bps_set_ncc_kernel": (_I, [_P, _I, _I]),
    "bps_peek_error_code": (_I, [_P]),
    "bps_get_ncc_kernel": (_I, [_P, _I, _I]),
    "bps_warmnet_conv3x3": (_I, [_P, _I, _I, _I, _I, _I, _P, _P, _I, _I, _P, _I, _P]),
    "bps_warmnet_conv3x3_backward": (_I, [_P, _P, _P, _I, _I, _I, _I, _I, _P, _I, _P, _P, _P, _P]),
    "bps_warmnet_mse": (_I, [_P, _P, _P, _I64, _P, _P, _I, _P]),
    "bps_warmnet_adam": (_I, [_P, _P, _P, _P, _I64, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                              _I, _P, _P]),
    "bps_warmnet_features": (_I, [_P, _I, _I, _I, ctypes.c_float, _P, _P]),
    "bps_warmnet_messages": (_I, [_P, _I, _I, _I, _I, _P, _P]),
}


def lib() -> ctypes.CDLL:
    """Load libbpstereo.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1709_06509_gb300._build.build()")
        _lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


_lib_debug = None


def lib_debug() -> ctypes.CDLL:
    """Load libbpstereo_debug.so, the same library built with -DBPS_DEBUG_BOUNDS: its kernels check
    list entries, list appends, cost stores and read-out pixels against their buffers and report a
    failed check through bps_get_error (BPS_ERR_INTERNAL) instead of accessing out of bounds.  For
    tests; raises if it has not been built (_build.build(debug=True))."""
    global _lib_debug
    if _lib_debug is None:
        if not os.path.exists(LIB_DEBUG_PATH):
            raise RuntimeError(f"{LIB_DEBUG_PATH} is missing: build it with paper_1709_06509_gb300._build.build(debug=True)")
        _lib_debug = ctypes.CDLL(LIB_DEBUG_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(_lib_debug, name)
            f.restype = res
            f.argtypes = args
    return _lib_debug


def status_string(status: int) -> str:
    return lib().bps_status_string(status).decode()


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise BPSError(rc, what)
    return rc


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------------ one-to-one entry points

def bps_workspace_bytes(W: int, H: int, D: int, levels: int, msg_type: int) -> int:
    return lib().bps_workspace_bytes(W, H, D, levels, msg_type)


def bps_create(W: int, H: int, D: int, levels: int, msg_type: int, workspace=None) -> int:
    ctx = _P()
    nbytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(lib().bps_create(ctypes.byref(ctx), W, H, D, levels, msg_type, _ptr(workspace), nbytes), "bps_create")
    return ctx.value


def bps_destroy(ctx: int) -> None:
    _check(lib().bps_destroy(ctx), "bps_destroy")


def bps_build_cost_volume(ctx, left, right, pitch, window, trunc_data, ncc_out=None, stream=None):
    _check(lib().bps_build_cost_volume(ctx, _ptr(left), _ptr(right), pitch, window, trunc_data, _ptr(ncc_out),
                                       _stream(stream)), "bps_build_cost_volume")


def bps_bp_solve(ctx, levels, iters, lam, trunc, flags, init_msgs=None, stream=None):
    _check(lib().bps_bp_solve(ctx, levels, iters, lam, trunc, flags, _ptr(init_msgs), _stream(stream)),
           "bps_bp_solve")


def bps_bp_solve_schedule(ctx, iters_per_scale, lam, trunc, flags, init_msgs=None, stream=None):
    """iters_per_scale[l] iterations at scale l (0 = the finest); len() scales."""
    n = len(iters_per_scale)
    arr = (_I * n)(*[int(v) for v in iters_per_scale])
    _check(lib().bps_bp_solve_schedule(ctx, n, arr, lam, trunc, flags, _ptr(init_msgs), _stream(stream)),
           "bps_bp_solve_schedule")


def bps_wta_disparity(ctx, disp, stream=None):
    _check(lib().bps_wta_disparity(ctx, _ptr(disp), _stream(stream)), "bps_wta_disparity")


def bps_energy(ctx, disp, lam, trunc, energy_i64=None, energy_f64=None, stream=None):
    _check(lib().bps_energy(ctx, _ptr(disp), lam, trunc, _ptr(energy_i64), _ptr(energy_f64), _stream(stream)),
           "bps_energy")


def bps_stereo(ctx, left, right, pitch, window, trunc_data, iters, lam, trunc, flags, disp, stream=None):
    _check(lib().bps_stereo(ctx, _ptr(left), _ptr(right), pitch, window, trunc_data, iters, lam, trunc, flags,
                            _ptr(disp), _stream(stream)), "bps_stereo")


def bps_stereo_host(ctx, h_left, h_right, pitch, window, trunc_data, iters, lam, trunc, flags, h_disp,
                    h_energy_i64=None, h_energy_f64=None, stream=None):
    _check(lib().bps_stereo_host(ctx, _ptr(h_left), _ptr(h_right), pitch, window, trunc_data, iters, lam, trunc,
                                 flags, _ptr(h_disp), _ptr(h_energy_i64), _ptr(h_energy_f64), _stream(stream)),
           "bps_stereo_host")


def bps_get_trace(ctx, h_counts, cap: int) -> int:
    return _check(lib().bps_get_trace(ctx, _ptr(h_counts), cap), "bps_get_trace")


def bps_export_messages(ctx, level, out, stream=None):
    _check(lib().bps_export_messages(ctx, level, _ptr(out), _stream(stream)), "bps_export_messages")


def bps_export_cost(ctx, level, out, stream=None):
    _check(lib().bps_export_cost(ctx, level, _ptr(out), _stream(stream)), "bps_export_cost")


def bps_read_profile(ctx):
    n, ms, px = _I(), ctypes.c_double(), _I64()
    _check(lib().bps_read_profile(ctx, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(px)), "bps_read_profile")
    return n.value, ms.value, px.value


def bps_energy_noalloc(cost, disp, W, H, D, lam, trunc, energy, stream=None):
    """Energy of `disp` over the natural-layout int32 cost volume `cost`, into the int64
    device tensor `energy`, with no memory allocated (scratch is a fixed device array)."""
    _check(lib().bps_energy_noalloc(_ptr(cost), _ptr(disp), W, H, D, lam, trunc, _ptr(energy), _stream(stream)),
           "bps_energy_noalloc")


def bps_test_fail_resources(n: int) -> None:
    """Plan a failure of the (n+1)-th resource acquisition of bps_create / bps_batch_create (n < 0: none)."""
    _check(lib().bps_test_fail_resources(n), "bps_test_fail_resources")


def bps_measure_sync_costs(ctas: int, phases: int = 2000) -> tuple[float, float]:
    """(us per grid barrier in one cooperative launch, us per PDL-chained kernel boundary in a graph)."""
    b, k = ctypes.c_double(), ctypes.c_double()
    _check(lib().bps_measure_sync_costs(ctas, phases, ctypes.byref(b), ctypes.byref(k)), "bps_measure_sync_costs")
    return b.value, k.value


def bps_batch_create(ctxs) -> int:
    arr = (_P * len(ctxs))(*ctxs)
    out = _P()
    _check(lib().bps_batch_create(ctypes.byref(out), arr, len(ctxs)), "bps_batch_create")
    return out.value


def bps_batch_destroy(batch: int) -> None:
    _check(lib().bps_batch_destroy(batch), "bps_batch_destroy")


def bps_batch_stereo(batch, lefts, rights, pitches, windows, trunc_data, iters, lam, trunc, flags, disps,
                     stream=None):
    n = len(lefts)
    P = (_P * n)(*[_ptr(t) for t in lefts])
    Q = (_P * n)(*[_ptr(t) for t in rights])
    pi = (_I * n)(*pitches)
    wi = (_I * n)(*windows)
    D = (_P * n)(*[_ptr(t) for t in disps])
    _check(lib().bps_batch_stereo(batch, P, Q, pi, wi, trunc_data, iters, lam, trunc, flags, D, _stream(stream)),
           "bps_batch_stereo")


def bps_batch_stereo_host(batch, h_lefts, h_rights, pitches, windows, trunc_data, iters, lam, trunc, flags, h_disps,
                          h_energies=None, stream=None):
    n = len(h_lefts)
    P = (_P * n)(*[_ptr(t) for t in h_lefts])
    Q = (_P * n)(*[_ptr(t) for t in h_rights])
    pi = (_I * n)(*pitches)
    wi = (_I * n)(*windows)
    D = (_P * n)(*[_ptr(t) for t in h_disps])
    _check(lib().bps_batch_stereo_host(batch, P, Q, pi, wi, trunc_data, iters, lam, trunc, flags, D, _ptr(h_energies),
                                       _stream(stream)), "bps_batch_stereo_host")


def bps_batch_get_error(batch) -> int:
    rc = lib().bps_batch_get_error(batch)
    if rc not in (BPS_OK, BPS_ERR_TIMEOUT):
        raise BPSError(rc, "bps_batch_get_error")
    return rc


def bps_set_sweep_variant(ctx, level: int, variant: int) -> None:
    _check(lib().bps_set_sweep_variant(ctx, level, variant), "bps_set_sweep_variant")


def bps_set_ncc_shape(ctx, column_groups: int, rows: int) -> None:
    _check(lib().bps_set_ncc_shape(ctx, column_groups, rows), "bps_set_ncc_shape")


def bps_peek_error_code(ctx) -> int:
    """The raw error word of the device-side checks, not cleared (see include/bpstereo.h)."""
    return _check(lib().bps_peek_error_code(ctx), "bps_peek_error_code")


def bps_set_ncc_kernel(ctx, kernel: int, rows: int = 0) -> None:
    _check(lib().bps_set_ncc_kernel(ctx, kernel, rows), "bps_set_ncc_kernel")


def bps_get_ncc_kernel(ctx, window: int, trunc_data: int) -> int:
    return _check(lib().bps_get_ncc_kernel(ctx, window, trunc_data), "bps_get_ncc_kernel")


def bps_get_sweep_variant(ctx, level: int) -> int:
    return _check(lib().bps_get_sweep_variant(ctx, level), "bps_get_sweep_variant")


def bps_set_skip_rule(ctx, eps: int, freeze: bool) -> None:
    _check(lib().bps_set_skip_rule(ctx, int(eps), int(freeze)), "bps_set_skip_rule")


def bps_set_candidates(ctx, K: int) -> None:
    _check(lib().bps_set_candidates(ctx, int(K)), "bps_set_candidates")


def bps_export_sparse(ctx, d_cand, d_msgs, stream=None) -> None:
    _check(lib().bps_export_sparse(ctx, _ptr(d_cand), _ptr(d_msgs), _stream(stream)), "bps_export_sparse")


def bps_warmnet_conv3x3(x, x_bf16, B, Cin, H, W, w, bias, Cout, relu, out, out_bf16, stream=None):
    _check(lib().bps_warmnet_conv3x3(_ptr(x), int(x_bf16), B, Cin, H, W, _ptr(w), _ptr(bias), Cout, int(relu), _ptr(out),
                                     int(out_bf16), _stream(stream)), "bps_warmnet_conv3x3")


def bps_warmnet_get_error() -> int:
    """BPS_OK, or BPS_ERR_TIMEOUT when a tensor-core convolution's bounded wait gave up (cleared)."""
    rc = lib().bps_warmnet_get_error()
    if rc not in (BPS_OK, BPS_ERR_TIMEOUT):
        raise BPSError(rc, "bps_warmnet_get_error")
    return rc


def bps_warmnet_conv3x3_backward(gout, relu_out, x, x_bf16, B, Cin, H, W, w, Cout, gin, gw, gb, stream=None):
    _check(lib().bps_warmnet_conv3x3_backward(_ptr(gout), _ptr(relu_out), _ptr(x), int(x_bf16), B, Cin, H, W, _ptr(w),
                                              Cout, _ptr(gin), _ptr(gw), _ptr(gb), _stream(stream)),
           "bps_warmnet_conv3x3_backward")


def bps_warmnet_mse(pred, target, mask, n, grad, loss_parts, nparts, stream=None):
    _check(lib().bps_warmnet_mse(_ptr(pred), _ptr(target), _ptr(mask), n, _ptr(grad), _ptr(loss_parts), nparts,
                                 _stream(stream)), "bps_warmnet_mse")


def bps_warmnet_adam(w, m, v, g, n, lr, beta1, beta2, eps, step, w_bf16=None, stream=None):
    _check(lib().bps_warmnet_adam(_ptr(w), _ptr(m), _ptr(v), _ptr(g), n, lr, beta1, beta2, eps, step, _ptr(w_bf16),
                                  _stream(stream)), "bps_warmnet_adam")


def bps_warmnet_features(cost, H, W, D, scale, feat, stream=None):
    _check(lib().bps_warmnet_features(_ptr(cost), H, W, D, scale, _ptr(feat), _stream(stream)), "bps_warmnet_features")


def bps_warmnet_messages(pred, H, W, D, cap, init, stream=None):
    _check(lib().bps_warmnet_messages(_ptr(pred), H, W, D, cap, _ptr(init), _stream(stream)), "bps_warmnet_messages")


def bps_last_cuda_error() -> int:
    return lib().bps_last_cuda_error()


def bps_cuda_error_string(code: int) -> str:
    return lib().bps_cuda_error_string(code).decode()


def bps_get_error(ctx) -> int:
    """BPS_OK, BPS_ERR_TIMEOUT or BPS_ERR_INTERNAL from the context's device-side checks (returned, not
    raised; see include/bpstereo.h)."""
    rc = lib().bps_get_error(ctx)
    if rc not in (BPS_OK, BPS_ERR_TIMEOUT, BPS_ERR_INTERNAL):
        raise BPSError(rc, "bps_get_error")
    return rc


def bps_read_launch_times(ctx, h_ms, cap: int) -> int:
    return _check(lib().bps_read_launch_times(ctx, _ptr(h_ms), cap), "bps_read_launch_times")


# ------------------------------------------------------------------ convenience wrapper

def level_dims(W: int, H: int, levels: int) -> list[tuple[int, int]]:
    dims = [(W, H)]
    for _ in range(1, levels):
        w, h = dims[-1]
        dims.append(((w + 1) // 2, (h + 1) // 2))
    return dims


class Stereo:
    """One context (W x H images, D labels, `levels` scales, numerical form `msg_type`) with
    its workspace held in a torch uint8 tensor on `device`."""

    def __init__(self, W: int, H: int, D: int, levels: int = 4, msg_type: int = BPS_MSG_U8, device="cuda"):
        import torch

        self.W, self.H, self.D, self.levels, self.msg_type = W, H, D, levels, msg_type
        nbytes = bps_workspace_bytes(W, H, D, levels, msg_type)
        if nbytes == 0:
            raise BPSError(BPS_ERR_ARG, "bps_workspace_bytes")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.ctx = bps_create(W, H, D, levels, msg_type, self.workspace)
        self.device = self.workspace.device

    def close(self):
        if getattr(self, "ctx", None):
            bps_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def msg_dtype(self):
        import torch

        return torch.float32 if self.msg_type == BPS_MSG_FP16 else torch.int32

    def build_cost_volume(self, left, right, window: int, trunc_data: int, want_ncc: bool = False, stream=None):
        import torch

        ncc = torch.empty((self.H, self.W, self.D), dtype=torch.float32, device=self.device) if want_ncc else None
        bps_build_cost_volume(self.ctx, left, right, left.stride(0), window, trunc_data, ncc, stream)
        return ncc

    def bp_solve(self, iters: int, lam: int, trunc: int, levels: int | None = None, skip: bool = True,
                 init_msgs=None, profile: bool = False, persistent: bool = False, test_timeout: bool = False,
                 graph: bool = False, stream=None):
        flags = (BPS_FLAG_FAST_SKIP if skip else 0) | (BPS_FLAG_WARM_START if init_msgs is not None else 0)
        flags |= (BPS_FLAG_PROFILE if profile else 0) | (BPS_FLAG_PERSISTENT if persistent else 0)
        flags |= (BPS_FLAG_TEST_TIMEOUT if test_timeout else 0) | (BPS_FLAG_GRAPH if graph else 0)
        bps_bp_solve(self.ctx, levels or self.levels, iters, lam, trunc, flags, init_msgs, stream)

    def bp_solve_schedule(self, iters_per_scale, lam: int, trunc: int, skip: bool = True, init_msgs=None,
                          graph: bool = False, stream=None):
        """The solve with iters_per_scale[l] iterations at scale l (0 = the finest)."""
        flags = (BPS_FLAG_FAST_SKIP if skip else 0) | (BPS_FLAG_WARM_START if init_msgs is not None else 0)
        flags |= BPS_FLAG_GRAPH if graph else 0
        bps_bp_solve_schedule(self.ctx, iters_per_scale, lam, trunc, flags, init_msgs, stream)

    def wta_disparity(self, out=None, stream=None):
        import torch

        out = out if out is not None else torch.empty((self.H, self.W), dtype=torch.int32, device=self.device)
        bps_wta_disparity(self.ctx, out, stream)
        return out

    def energy(self, disp, lam: int, trunc: int, stream=None):
        import torch

        ei = torch.zeros(1, dtype=torch.int64, device=self.device)
        ef = torch.zeros(1, dtype=torch.float64, device=self.device)
        bps_energy(self.ctx, disp, lam, trunc, ei, ef, stream)
        return ei, ef

    def stereo(self, left, right, window, trunc_data, iters, lam, trunc, skip=True, graph=False, out=None,
               persistent=False, stream=None):
        import torch

        out = out if out is not None else torch.empty((self.H, self.W), dtype=torch.int32, device=self.device)
        flags = (BPS_FLAG_FAST_SKIP if skip else 0) | (BPS_FLAG_GRAPH if graph else 0)
        flags |= BPS_FLAG_PERSISTENT if persistent else 0
        bps_stereo(self.ctx, left, right, left.stride(0), window, trunc_data, iters, lam, trunc, flags, out, stream)
        return out

    def stereo_host(self, h_left, h_right, window, trunc_data, iters, lam, trunc, skip=True, graph=True,
                    h_disp=None, stream=None):
        """Host tensors in, host disparity and energy out (synchronous)."""
        import torch

        pin = h_left.is_pinned()
        own = h_disp is None
        if pin:
            # page-locked buffers kept across calls: the call replays as one recorded graph
            # while its buffers stay the same
            if getattr(self, "_host_bufs", None) is None:
                self._host_bufs = (torch.empty((self.H, self.W), dtype=torch.int32).pin_memory(),
                                   torch.zeros(1, dtype=torch.int64).pin_memory(),
                                   torch.zeros(1, dtype=torch.float64).pin_memory())
            d0, ei, ef = self._host_bufs
            h_disp = d0 if own else h_disp
        else:
            h_disp = torch.empty((self.H, self.W), dtype=torch.int32) if own else h_disp
            ei = torch.zeros(1, dtype=torch.int64)
            ef = torch.zeros(1, dtype=torch.float64)
        flags = (BPS_FLAG_FAST_SKIP if skip else 0) | (BPS_FLAG_GRAPH if graph else 0)
        bps_stereo_host(self.ctx, h_left, h_right, h_left.stride(0), window, trunc_data, iters, lam, trunc, flags,
                        h_disp, ei if self.msg_type != BPS_MSG_FP16 else None, ef, stream)
        energy = int(ei.item()) if self.msg_type != BPS_MSG_FP16 else float(ef.item())
        return (h_disp.clone() if own and pin else h_disp), energy

    def get_trace(self):
        import numpy as np

        buf = np.zeros(self.levels * BPS_MAX_ITERS * 2, dtype=np.int64)
        n = bps_get_trace(self.ctx, buf.ctypes.data, buf.size)
        return buf[:n]

    def export_messages(self, level: int = 0, stream=None):
        import torch

        w, h = level_dims(self.W, self.H, self.levels)[level]
        out = torch.empty((4, h, w, self.D), dtype=self.msg_dtype, device=self.device)
        bps_export_messages(self.ctx, level, out, stream)
        return out

    def export_cost(self, level: int = 0, stream=None):
        import torch

        w, h = level_dims(self.W, self.H, self.levels)[level]
        out = torch.empty((h, w, self.D), dtype=self.msg_dtype, device=self.device)
        bps_export_cost(self.ctx, level, out, stream)
        return out

    def read_profile(self):
        return bps_read_profile(self.ctx)

    def get_error(self) -> int:
        return bps_get_error(self.ctx)

    def set_variant(self, level: int, variant: int) -> None:
        bps_set_sweep_variant(self.ctx, level, variant)

    def set_skip_rule(self, eps: int = 0, freeze: bool = False) -> None:
        """Approximate fast-converging skip: eps threshold on message changes, permanent freeze."""
        bps_set_skip_rule(self.ctx, eps, freeze)

    def set_candidates(self, K: int) -> None:
        """K sparse candidate labels per pixel at the finest scale (0: the dense solve)."""
        bps_set_candidates(self.ctx, K)
        self.K = K

    def export_sparse(self, stream=None):
        """Finest-scale candidates int32 [H][W][K] and messages int32 [4][H][W][K] of a sparse solve."""
        import torch

        K = getattr(self, "K", 0)
        cand = torch.empty((self.H, self.W, K), dtype=torch.int32, device=self.device)
        msgs = torch.empty((4, self.H, self.W, K), dtype=torch.int32, device=self.device)
        bps_export_sparse(self.ctx, cand, msgs, stream)
        return cand, msgs

    def set_ncc_shape(self, column_groups: int, rows: int) -> None:
        bps_set_ncc_shape(self.ctx, column_groups, rows)

    def set_ncc_kernel(self, kernel: int, rows: int = 0) -> None:
        bps_set_ncc_kernel(self.ctx, kernel, rows)

    def ncc_kernel(self, window: int, trunc_data: int) -> int:
        return bps_get_ncc_kernel(self.ctx, window, trunc_data)

    def variants(self) -> list[int]:
        return [bps_get_sweep_variant(self.ctx, l) for l in range(self.levels)]

    def read_launch_times(self):
        import numpy as np

        buf = np.zeros(self.levels * BPS_MAX_ITERS * 2, dtype=np.float64)
        n = bps_read_launch_times(self.ctx, buf.ctypes.data, buf.size)
        return buf[:n]


class Batch:
    """Several Stereo contexts solved together (concurrent chains, or one persistent launch)."""

    def __init__(self, stereos):
        self.stereos = list(stereos)
        self.handle = bps_batch_create([st.ctx for st in self.stereos])

    def close(self):
        if getattr(self, "handle", None):
            bps_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def stereo(self, lefts, rights, windows, trunc_data, iters, lam, trunc, skip=True, graph=True,
               persistent=False, outs=None, stream=None):
        import torch

        if outs is None:
            outs = [torch.empty((st.H, st.W), dtype=torch.int32, device=st.device) for st in self.stereos]
        flags = (BPS_FLAG_FAST_SKIP if skip else 0) | (BPS_FLAG_GRAPH if graph else 0)
        flags |= BPS_FLAG_PERSISTENT if persistent else 0
        bps_batch_stereo(self.handle, lefts, rights, [t.stride(0) for t in lefts], windows, trunc_data, iters, lam,
                         trunc, flags, outs, stream)
        return outs

    def get_error(self) -> int:
        return bps_batch_get_error(self.handle)

    def stereo_host(self, h_lefts, h_rights, windows, trunc_data, iters, lam, trunc, skip=True, graph=True,
                    persistent=False, h_disps=None, stream=None, sync=True):
        """Host tensors in; host disparities and int64 energies out.  sync=False: return once the
        work is queued (copies included); the outputs are valid after the stream is synchronised."""
        import torch

        # page-locked buffers kept across calls: the call replays as one recorded graph while
        # its buffers stay the same
        if getattr(self, "_host_bufs", None) is None:
            self._host_bufs = ([torch.empty((st.H, st.W), dtype=torch.int32).pin_memory() for st in self.stereos],
                               torch.zeros(len(self.stereos), dtype=torch.int64).pin_memory())
        own = h_disps is None
        h_disps = self._host_bufs[0] if own else h_disps
        energies = self._host_bufs[1]
        flags = (BPS_FLAG_FAST_SKIP if skip else 0) | (BPS_FLAG_GRAPH if graph else 0)
        flags |= (BPS_FLAG_PERSISTENT if persistent else 0) | (0 if sync else BPS_FLAG_ASYNC)
        bps_batch_stereo_host(self.handle, h_lefts, h_rights, [t.stride(0) for t in h_lefts], windows, trunc_data,
                              iters, lam, trunc, flags, h_disps, energies, stream)
        if not sync:
            return h_disps, energies  # valid after the stream is synchronised
        return ([d.clone() for d in h_disps] if own else h_disps), energies.clone()
