"""Autotuner: the NCC kernel's CTA shape and the red-black sweep's kernel variant of every
scale, picked by measurement.

Every variant computes the same messages (bit for bit); they differ in how fast they run at a
given scale size and label count (see bps_set_sweep_variant in include/bpstereo.h):
  0                  stencil form where trunc <= 2, dense launch over all pixels, the dirty
                     flag read before the inputs
  GENERAL_DT         distance-transform form instead of the stencil
  LISTS              active lists after the scale's first iteration (large scales)
  EAGER              every load of a half-sweep issued at once (small scales)
  CLUSTER            every iteration of the scale in one thread-block-cluster launch
  DPAR               one lane group per (pixel, direction): the four messages side by side
  DPAR_LISTS         ... on the list launches only
  STAGED             dense launches prefetch the next block's inputs into shared memory (large scales)
  STAGED_LISTS       ... list launches
  BULK               dense launches fed by a copy warp's bulk copies of whole records (large scales)
  BULK_LISTS         ... list launches
and their combinations.  For one context and one representative input, tune() replays the
whole pipeline from its CUDA graph (the way the variants run in production: consecutive
launches overlap, which per-launch events would hide) and descends one scale at a time,
coarsest first, keeping each scale's fastest candidate with the others fixed.  Choices can
be cached in a JSON file keyed by GPU, scale size, padded label count, numerical form,
truncation class and skip, so later contexts of the same shapes skip the measurement.
"""
from __future__ import annotations

import json
import os

from . import (BPS_ERR_UNSUPPORTED, BPS_VARIANT_BLOCK2, BPS_VARIANT_BULK, BPS_VARIANT_BULK_LISTS, BPS_VARIANT_CLUSTER,
               BPS_VARIANT_DPAR,
               BPS_VARIANT_DPAR_LISTS, BPS_VARIANT_EAGER, BPS_VARIANT_GENERAL_DT, BPS_VARIANT_LISTS,
               BPS_VARIANT_STAGED, BPS_VARIANT_STAGED_LISTS, BPSError, level_dims)

_G, _L, _E, _C, _P, _PL, _S, _SL = (BPS_VARIANT_GENERAL_DT, BPS_VARIANT_LISTS, BPS_VARIANT_EAGER, BPS_VARIANT_CLUSTER,
                                    BPS_VARIANT_DPAR, BPS_VARIANT_DPAR_LISTS, BPS_VARIANT_STAGED,
                                    BPS_VARIANT_STAGED_LISTS)
_B, _BL = BPS_VARIANT_BULK, BPS_VARIANT_BULK_LISTS
_K = BPS_VARIANT_BLOCK2  # blocking depth 2 for a scale's first iteration (depth 1 without it)
# a cluster launch is only a candidate for scales of at most this many lanes (pixels x lanes per pixel)
CLUSTER_MAX_LANES = 16 * 16 * 512
SMALL_CANDIDATES = (0, _G, _E, _E | _G, _C, _C | _E, _C | _E | _G, _P, _P | _G, _P | _E, _P | _E | _G)
LARGE_CANDIDATES = (0, _G, _L, _G | _L, _E, _E | _G, _E | _L, _E | _G | _L, _P, _P | _E, _P | _L, _P | _E | _L,
                    _L | _PL, _E | _L | _PL, _G | _L | _PL, _E | _G | _L | _PL, _S, _S | _G, _S | _L, _S | _G | _L,
                    _S | _L | _PL, _S | _G | _L | _PL, _L | _SL, _G | _L | _SL, _E | _L | _SL, _E | _G | _L | _SL,
                    _S | _L | _SL, _S | _G | _L | _SL, _B, _B | _L, _L | _BL, _B | _L | _BL, _B | _G | _L | _BL,
                    _B | _L | _SL, _S | _L | _BL, _E | _L | _BL)
# the blocking-depth axis: depth 2 (a scale's first iteration in one tiled launch) is offered only
# when asked for (tune(depths=(1, 2))); it measured slower on every workload tried (the half-sweeps
# are bound by instruction issue, and depth 2 recomputes the even pixels around each tile), so by
# default the tuner does not spend its time on it nor risk picking it on noise
BLOCKED_CANDIDATES = (_K, _K | _L, _K | _E | _L, _K | _L | _SL)
CANDIDATES = tuple(sorted(set(SMALL_CANDIDATES) | set(LARGE_CANDIDATES) | set(BLOCKED_CANDIDATES)))
DPAR_MAX_LANES_PER_PIXEL = 8  # direction-parallel lanes exist up to 128 labels
# the list and staged candidates are tried on every scale of at least this many lanes (a scale
# small enough for the cluster launch may still have enough pixels for active lists to pay)
LIST_MIN_LANES = 8 * 1024


def _candidates(lanes: int, Gp: int, depths: tuple = (1,)) -> list[int]:
    """The variants tried on a scale of `lanes` lanes (pixels of a colour x lanes a pixel), at the
    blocking depths `depths` of a scale's first iteration (1, or 1 and 2)."""
    cands = list(SMALL_CANDIDATES) if lanes <= CLUSTER_MAX_LANES else []
    if lanes > CLUSTER_MAX_LANES or lanes >= LIST_MIN_LANES:
        cands += [v for v in LARGE_CANDIDATES if v not in cands]
        if 2 in depths:
            cands += [v for v in BLOCKED_CANDIDATES if v not in cands]
    return [v for v in cands if not (v & (_P | _PL) and Gp > DPAR_MAX_LANES_PER_PIXEL)]


def _key(gpu: str, w: int, h: int, D: int, msg_type: int, trunc: int, skip: bool) -> str:
    tclass = trunc if trunc <= 2 else 3  # the stencil forms exist for trunc 0, 1, 2 only
    Dp = (D + 15) // 16 * 16
    return f"{gpu}|{w}x{h}|Dp{Dp}|form{msg_type}|T{tclass}|skip{int(skip)}|v6"


def _load(path: str | None) -> dict:
    if path and os.path.exists(path):
        with open(path) as fh:
            return json.load(fh)
    return {}


def _lanes_per_pixel(D: int) -> int:
    Gp = 1
    while Gp * 16 < (D + 15) // 16 * 16:
        Gp *= 2
    return Gp


def tune(st, left, right, window: int, trunc_data: int, iters: int, lam: int, trunc: int, skip: bool = True,
         reps: int = 3, cache: str | None = None, target_ms: float = 10.0, depths: tuple = (1,)) -> list[int]:
    """Pick and set the variant of every scale of `st` (a Stereo); returns them per scale.
    depths: the blocking depths of a scale's first iteration to consider, (1,) or (1, 2)."""
    import torch

    gpu = torch.cuda.get_device_name(st.device)
    dims = level_dims(st.W, st.H, st.levels)
    keys = [_key(gpu, w, h, st.D, st.msg_type, trunc, skip) + ("|depth2" if 2 in depths else "") for w, h in dims]
    table = _load(cache)
    if all(k in table for k in keys):
        chosen = [int(table[k]) for k in keys]
    else:
        Gp = _lanes_per_pixel(st.D)
        lanes = [h * ((w + 1) // 2) * Gp for w, h in dims]
        out = torch.empty((st.H, st.W), dtype=torch.int32, device=st.device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        def run():
            st.stereo(left, right, window, trunc_data, iters, lam, trunc, graph=True, skip=skip, out=out)

        def step_ms(vs) -> float:
            for lvl, v in enumerate(vs):
                st.set_variant(lvl, v)
            run()  # records the graph
            run()
            e0.record()
            run()
            e1.record()
            e1.synchronize()
            n = max(2, min(200, int(target_ms / max(e0.elapsed_time(e1), 1e-3))))
            best = float("inf")
            for _ in range(reps):
                e0.record()
                for _ in range(n):
                    run()
                e1.record()
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1) / n)
            return best

        current = st.variants()
        for lvl in reversed(range(st.levels)):
            times = {}
            for v in _candidates(lanes[lvl], Gp, depths):
                trial = list(current)
                trial[lvl] = v
                try:
                    times[v] = step_ms(trial)
                except BPSError as e:
                    if e.status == BPS_ERR_UNSUPPORTED:  # no room for the cluster on this GPU
                        continue
                    raise
            current[lvl] = min(times, key=times.get)
        chosen = current
        if cache:
            table.update({k: v for k, v in zip(keys, chosen)})
            os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
            with open(cache, "w") as fh:
                json.dump(table, fh, indent=1, sort_keys=True)
    for lvl, v in enumerate(chosen):
        st.set_variant(lvl, v)
    return chosen


def _set_ncc(st, choice) -> None:
    """Apply an NCC choice: (-1, rows) is the tensor-core kernel with `rows` rows per strip,
    (column_groups, rows) the row kernel's CTA shape."""
    import paper_1709_06509_gb300 as bps

    xs, rows = choice
    if xs < 0:
        st.set_ncc_kernel(bps.BPS_NCC_TENSOR, rows)
    else:
        st.set_ncc_kernel(bps.BPS_NCC_ROWS)
        st.set_ncc_shape(xs, rows)


def tune_ncc(st, left, right, window: int, trunc_data: int, reps: int = 5, cache: str | None = None):
    """Pick and set the NCC kernel of `st` for windows up to 15 and return the choice: the
    tensor-core kernel as (-1, rows per strip) where it applies, or the row kernel's CTA shape
    (column groups per CTA, rows per strip).  Every choice computes the same costs."""
    import torch

    import paper_1709_06509_gb300 as bps

    if window > 15:
        return (0, 0)
    gpu = torch.cuda.get_device_name(st.device)
    Dp = (st.D + 15) // 16 * 16
    key = f"{gpu}|ncc|{st.W}x{st.H}|Dp{Dp}|w{window}|t{trunc_data}|form{st.msg_type}|v3"
    table = _load(cache)
    if key in table:
        best = tuple(table[key])
    else:
        xs_max = max(1, 512 // Dp)  # CTAs of up to 512 threads
        cands = [(0, 0)]
        xs = xs_max
        while xs >= 1:
            if 32 <= xs * Dp <= 512:
                cands += [(xs, r) for r in (2, 4, 8, 16, 32, 64) if r <= max(2, st.H)]
            xs //= 2
        st.set_ncc_kernel(bps.BPS_NCC_DEFAULT)
        if st.ncc_kernel(window, trunc_data) == bps.BPS_NCC_TENSOR:
            cands += [(-1, 0)] + [(-1, r) for r in (8, 16, 32, 64, 128, 256) if r < st.H]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        timed = {}
        for c in cands:
            _set_ncc(st, c)
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
    _set_ncc(st, best)
    return best


def tune_batch(batch, sts, lefts, rights, windows, trunc_data: int, iters: int, lam: int, trunc: int,
               skip: bool = True, reps: int = 3, cache: str | None = None, target_ms: float = 20.0,
               margin: float = 0.005) -> list[list[int]]:
    """Refine the sweep variants of every member of a batch jointly and set them; returns them.

    The members' launch chains run side by side on one GPU, so the variant that is fastest for a
    member alone may take SMs from another member's critical path.  Starting from the current
    choices (normally each member's own tuning), one pass of coordinate descent over (member,
    scale) times the whole batch graph; a candidate replaces the current choice only when it
    makes the batch faster by more than `margin`.  Cached under the members' keys together."""
    import torch

    gpu = torch.cuda.get_device_name(sts[0].device)
    member_keys = []
    for st in sts:
        dims = level_dims(st.W, st.H, st.levels)
        member_keys.append([_key(gpu, w, h, st.D, st.msg_type, trunc, skip) for w, h in dims])
    key = "batch[" + ";".join(",".join(k) for k in member_keys) + "]"
    table = _load(cache)
    if key in table:
        chosen = [list(map(int, v)) for v in table[key]]
        for st, vs in zip(sts, chosen):
            for lvl, v in enumerate(vs):
                st.set_variant(lvl, v)
        return chosen
    outs = [torch.empty((st.H, st.W), dtype=torch.int32, device=st.device) for st in sts]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def run():
        batch.stereo(lefts, rights, windows, trunc_data, iters, lam, trunc, skip=skip, graph=True, outs=outs)

    def step_ms() -> float:
        run()  # records the graph
        run()
        e0.record()
        run()
        e1.record()
        e1.synchronize()
        n = max(2, min(400, int(target_ms / max(e0.elapsed_time(e1), 1e-3))))
        best = float("inf")
        for _ in range(reps):
            e0.record()
            for _ in range(n):
                run()
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / n)
        return best

    base = step_ms()
    for st in sts:
        Gp = _lanes_per_pixel(st.D)
        dims = level_dims(st.W, st.H, st.levels)
        for lvl in reversed(range(st.levels)):
            w, h = dims[lvl]
            current = st.variants()[lvl]
            best_v, best_t = current, base
            for v in _candidates(h * ((w + 1) // 2) * Gp, Gp):
                if v == current:
                    continue
                try:
                    st.set_variant(lvl, v)
                except BPSError as e:
                    if e.status == BPS_ERR_UNSUPPORTED:
                        continue
                    raise
                t = step_ms()
                if t < best_t * (1.0 - margin):
                    best_v, best_t = v, t
            st.set_variant(lvl, best_v)
            base = best_t
    chosen = [st.variants() for st in sts]
    if cache:
        table[key] = chosen
        os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
        with open(cache, "w") as fh:
            json.dump(table, fh, indent=1, sort_keys=True)
    return chosen
