"""Autotuner: the NCC kernel's CTA shape and the red-black sweep's kernel variant of every
scale, picked by measurement.

Every variant computes the same messages (bit for bit); they differ in how fast they run at a
given scale size and label count (see bps_set_sweep_variant in include/bpstereo.h):
  0                          stencil form where trunc <= 2, dense launch over all pixels
  LISTS                      ... with active lists after the scale's first iteration
  GENERAL_DT                 distance-transform form, dense launch
  GENERAL_DT | LISTS         distance-transform form with active lists
For one context and one representative input, tune() runs the whole solve once per
candidate with CUDA events around every half-sweep launch (BPS_FLAG_PROFILE), sums the
launch times of each scale, and keeps each scale's fastest candidate.  Scales do not
interact, so one solve per candidate times every scale at once.  Choices can be cached in
a JSON file keyed by GPU, scale size, padded label count, numerical form, truncation class
and skip, so later contexts of the same shapes skip the measurement.
"""
from __future__ import annotations

import json
import os

from . import BPS_VARIANT_GENERAL_DT, BPS_VARIANT_LISTS, level_dims

CANDIDATES = (0, BPS_VARIANT_LISTS, BPS_VARIANT_GENERAL_DT, BPS_VARIANT_GENERAL_DT | BPS_VARIANT_LISTS)


def _key(gpu: str, w: int, h: int, D: int, msg_type: int, trunc: int, skip: bool) -> str:
    tclass = trunc if trunc <= 2 else 3  # the stencil forms exist for trunc 0, 1, 2 only
    Dp = (D + 15) // 16 * 16
    return f"{gpu}|{w}x{h}|Dp{Dp}|form{msg_type}|T{tclass}|skip{int(skip)}"


def _load(path: str | None) -> dict:
    if path and os.path.exists(path):
        with open(path) as fh:
            return json.load(fh)
    return {}


def tune(st, left, right, window: int, trunc_data: int, iters: int, lam: int, trunc: int, skip: bool = True,
         reps: int = 3, cache: str | None = None) -> list[int]:
    """Pick and set the variant of every scale of `st` (a Stereo); returns them per scale."""
    import torch

    gpu = torch.cuda.get_device_name(st.device)
    dims = level_dims(st.W, st.H, st.levels)
    keys = [_key(gpu, w, h, st.D, st.msg_type, trunc, skip) for w, h in dims]
    table = _load(cache)
    if all(k in table for k in keys):
        chosen = [int(table[k]) for k in keys]
    else:
        per = 2 * iters
        times = {v: [0.0] * st.levels for v in CANDIDATES}
        st.build_cost_volume(left, right, window, trunc_data)
        for v in CANDIDATES:
            for lvl in range(st.levels):
                st.set_variant(lvl, v)
            st.bp_solve(iters, lam, trunc, skip=skip, profile=True)  # warm-up of this variant
            for _ in range(reps):
                st.bp_solve(iters, lam, trunc, skip=skip, profile=True)
                t = st.read_launch_times()
                # launch order is coarsest scale first
                for k in range(st.levels):
                    times[v][st.levels - 1 - k] += float(t[k * per:(k + 1) * per].sum())
        chosen = [min(CANDIDATES, key=lambda v: times[v][lvl]) for lvl in range(st.levels)]
        if cache:
            table.update({k: v for k, v in zip(keys, chosen)})
            os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
            with open(cache, "w") as fh:
                json.dump(table, fh, indent=1, sort_keys=True)
    for lvl, v in enumerate(chosen):
        st.set_variant(lvl, v)
    return chosen


def tune_ncc(st, left, right, window: int, trunc_data: int, reps: int = 5, cache: str | None = None):
    """Pick and set the NCC CTA shape (column groups per CTA, rows per strip) of `st` for
    windows up to 15; returns it.  Every shape computes the same costs."""
    import torch

    if window > 15:
        return (0, 0)
    gpu = torch.cuda.get_device_name(st.device)
    Dp = (st.D + 15) // 16 * 16
    key = f"{gpu}|ncc|{st.W}x{st.H}|Dp{Dp}|w{window}|form{st.msg_type}"
    table = _load(cache)
    if key in table:
        best = tuple(table[key])
    else:
        xs_max = 1 if Dp >= 256 else 256 // Dp
        cands = [(0, 0)]
        xs = xs_max
        while xs >= 1:
            if 32 <= xs * Dp <= 512:
                cands += [(xs, r) for r in (2, 4, 8, 16, 32, 64) if r <= max(2, st.H)]
            xs //= 2
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        timed = {}
        for c in cands:
            st.set_ncc_shape(*c)
            st.build_cost_volume(left, right, window, trunc_data)
            e0.record()
            for _ in range(reps):
                st.build_cost_volume(left, right, window, trunc_data)
            e1.record()
            torch.cuda.synchronize()
            timed[c] = e0.elapsed_time(e1)
        best = min(timed, key=timed.get)
        if cache:
            table[key] = list(best)
            os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
            with open(cache, "w") as fh:
                json.dump(table, fh, indent=1, sort_keys=True)
    st.set_ncc_shape(*best)
    return best
