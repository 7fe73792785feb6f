"""Throughput of the stereo hot path (NCC cost volume + 4-scale min-sum BP with the
fast-converging skip + WTA) in Mpix*disp/s, one JSON line on stdout.

Workload (per GPU): the full-HD configuration, one seeded synthetic 1920x1080 pair with
D = 256 labels, 9x9 NCC window, data costs quantised with trunc 20, 4 scales, 10 iterations
per scale, lambda = 10, trunc = 2, the exact fast-converging skip, integer messages in uint8
storage (bit-exact with the int32 method).  One step = one bps_stereo graph replay of the
whole path (cost volume, solve, read-out).  Its working set (4.3 GB) is far above L2; a
256 MiB buffer is also written between timed steps.

Beside the headline the line carries:
  roofline       the red-black half-sweeps (every sweep launch of a solve), algorithmic bytes
                 from the live skip trace over the graph-timed solve;
  fp16           the fp16-message form on the same pair, with its energy gap and label
                 disagreement against the FP64 oracle's result (tests/golden);
  c2             the 384x288 D16 + 450x375 D64 pairs as one batch graph, checked against the
                 oracle;
  e2e            bps_stereo_host from pinned host buffers, copies inside the timed region;
  cpu_baseline   the C oracle on a bounded crop of the same pair, which the GPU must match.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own replica (different seeds, weak scaling); the
per-rank device time is max-reduced and rank 0 prints.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpix·disp/s (cost vol + BP) at equal energy; plain int32 vs FP16/learned/batched"
UNIT = "Mpix·disp/s"
HEADLINE = "hd_1920x1080_d256"
C2_PAIRS = ["tsukuba_384x288_d16", "teddy_450x375_d64"]
TRUNC_DATA, LEVELS, ITERS, LAM, TRUNC = 20, 4, 10, 10, 2
FLUSH_BYTES = 256 << 20
# the bounded CPU sample: a central 384x216 crop of the full-HD pair (1/25 of its pixels), all
# 256 labels, the same window and solve parameters
CROP = (768, 432, 384, 216)  # x0, y0, width, height
GOLDEN = os.path.join(ROOT, "tests", "golden", HEADLINE + ".json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="headline only: no fp16 and c2 keys")
    ap.add_argument("--tune-cache", default=None,
                    help="JSON file of autotuned choices: read if present, else measured and written")
    ap.add_argument("--warmstart-report", action="store_true",
                    help="instead of the benchmark line: train the learned warm start on seeded 450x375 D64 "
                         "pairs and report energy and throughput against the plain solve, one JSON line")
    ap.add_argument("--train-pairs", type=int, default=None, help="default 2000 (450x375) or 48 (1920x1080)")
    ap.add_argument("--eval-pairs", type=int, default=None, help="default 200 (450x375) or 8 (1920x1080)")
    ap.add_argument("--warmstart-workload", choices=["teddy", "hd"], default="teddy",
                    help="with --warmstart-report: 450x375 D64 pairs (7x7) or 1920x1080 D256 pairs (9x9)")
    ap.add_argument("--batch-report", type=int, default=0, metavar="N",
                    help="instead of the benchmark line: throughput of a batch of N mixed pairs (320-1280 x "
                         "240-720, D in {32,64,96,128}) in every batch mode, one JSON line")
    ap.add_argument("--approx-report", action="store_true",
                    help="instead of the benchmark line: the approximate skip rules (eps threshold, permanent "
                         "freeze) on the benchmark pairs and the 960x540 D256 pair: time, work and energy gap "
                         "against the exact skip, one JSON line")
    ap.add_argument("--sparse-report", action="store_true",
                    help="instead of the benchmark line: the finest scale over K sparse candidates against the "
                         "dense solve on the benchmark pairs and the 1920x1080 D256 pair: throughput, energy gap, "
                         "bad pixels, one JSON line")
    ap.add_argument("--forms-report", action="store_true",
                    help="instead of the benchmark line: every message form (int32, u8, fp16) on the benchmark "
                         "pairs and the 1920x1080 D256 pair: throughput, energy, fp16 energy gap against the FP64 "
                         "oracle and bad-pixel rates, one JSON line")
    ap.add_argument("--launch-report", action="store_true",
                    help="instead of the benchmark line: per-launch times (profile mode) and recomputed pixels of "
                         "every sweep launch of the headline pair, one JSON line")
    ap.add_argument("--trace-jsonl", default=None, metavar="PATH",
                    help="also write, after the timed region, one JSON line per iteration count k = 1..10 of "
                         "the headline pair: the energy after k iterations per scale and, per half-sweep of the "
                         "finest scale, the pixels recomputed and the converged fraction")
    ap.add_argument("--blocking-report", action="store_true",
                    help="temporal blocking of a scale's first iteration: depth 1 (two launches) against depth 2 "
                         "(BPS_VARIANT_BLOCK2) on the 1280x720 D64 pair and the full-HD pair")
    ap.add_argument("--sync-report", action="store_true",
                    help="instead of the benchmark line: the cost of a grid barrier inside one cooperative launch "
                         "against a programmatically chained kernel boundary in a graph, for grids of 1 to 3 CTAs "
                         "a SM, one JSON line")
    ap.add_argument("--batch-form", choices=["u8", "fp16"], default="u8",
                    help="message form of --batch-report")
    ap.add_argument("--ncu-case", action="store_true",
                    help="only run warm-up + steps of the workload (no timing, no JSON): the command to profile")
    ap.add_argument("--form", choices=["u8", "fp16"], default="u8", help="with --ncu-case: the message form")
    ap.add_argument("--workload", default=None,
                    help="with --ncu-case: one named pair of paper_1709_06509_gb300.synth.WORKLOADS instead of "
                         "the full-HD pair")
    ap.add_argument("--ncc-kernel", choices=["tensor", "rows"], default=None,
                    help="with --ncu-case: the NCC kernel instead of the tuned one")
    ap.add_argument("--variants", default=None, metavar="V0,V1,V2,V3",
                    help="with --ncu-case: the sweep variant of each scale (finest first) instead of the tuned ones")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def work_units(pairs) -> int:
    return sum(p.left.shape[0] * p.left.shape[1] * p.D for p, _ in pairs)


def crop_pair(pair):
    """The bounded CPU sample of the full-HD pair (a StereoPair of the crop)."""
    from paper_1709_06509_gb300 import synth

    x0, y0, w, h = CROP
    sl = (slice(y0, y0 + h), slice(x0, x0 + w))
    return synth.StereoPair(pair.left[sl].copy(), pair.right[sl].copy(), pair.disparity[sl].copy(),
                            pair.occluded[sl].copy(), pair.D, pair.seed)


def golden() -> dict | None:
    try:
        with open(GOLDEN) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return None


def sha(a) -> str:
    import numpy as np

    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


# ------------------------------------------------------------------ CPU oracle (baseline)

def oracle_run(pair, window):
    """The whole integer path through the oracle: disparities, energy and trace."""
    import oracle

    c = oracle.quantise(oracle.ncc(pair.left, pair.right, pair.D, window), TRUNC_DATA)
    d, tr = oracle.bp_wta(c, LEVELS, ITERS, LAM, TRUNC, skip=True)
    return {"disp": d, "trace": tr, "energy": oracle.energy(c, d, LAM, TRUNC)}


def timed_oracle_run(pair, window):
    t0 = time.perf_counter()
    r = oracle_run(pair, window)
    return r, time.perf_counter() - t0


def cpu_baselines(crop, window) -> tuple[dict, dict | None, dict]:
    """The oracle as it stands on the crop: single-threaded, and its OpenMP build over every host
    core (same bits).  Returns (cpu_baseline, cpu_baseline_parallel or None, oracle result)."""
    import oracle

    from paper_1709_06509_gb300 import synth

    tiny, w = synth.workload_pair("tiny_96x72_d16")
    oracle_run(tiny, w)  # load / build the library outside the timing
    units = crop.left.size * crop.D
    ref, t = timed_oracle_run(crop, window)
    what = (f"a central {CROP[2]}x{CROP[3]} crop of the 1920x1080 D256 pair (1/25 of its pixels, all 256 labels, "
            "9x9 window, 4 scales, 10 iterations, skip on) through the C oracle")
    base = {"value": units / t / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{what}, single-threaded, {t:.1f} s"}
    par = None
    if oracle.openmp_available():
        with oracle.openmp(os.cpu_count() or 1) as n:
            r2, t2 = timed_oracle_run(crop, window)
        if not (r2["disp"] == ref["disp"]).all() or r2["energy"] != ref["energy"]:
            raise RuntimeError("the OpenMP build of the oracle disagrees with the serial build")
        par = {"value": units / t2 / 1e6, "unit": UNIT, "cores": n, "kind": "oracle (OpenMP build)",
               "sample": f"{what}, {n} threads, {t2:.1f} s"}
    return base, par, ref


def run_reference(args):
    """The reference arm: the oracle as it stands (OpenMP build, every host core) on the bounded
    crop of the headline pair, one crop per step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle

    from paper_1709_06509_gb300 import synth

    pair, window = synth.workload_pair(HEADLINE)
    crop = crop_pair(pair)
    units = crop.left.size * crop.D
    cores = 1
    ctx = oracle.openmp(os.cpu_count() or 1) if oracle.openmp_available() else None
    if ctx:
        cores = ctx.__enter__()
    try:
        for _ in range(args.warmup):
            oracle_run(crop, window)
        times = [timed_oracle_run(crop, window)[1] for _ in range(args.steps)]
    finally:
        if ctx:
            ctx.__exit__(None, None, None)
    total = sum(times)
    value = units * args.steps / total / 1e6
    sample = (f"a central {CROP[2]}x{CROP[3]} crop of the 1920x1080 D256 pair per step (1/25 of its pixels, all "
              f"256 labels), the C oracle's OpenMP build on {cores} host threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": "1920x1080 D256 pair (bounded sample: a central crop per step)", "window": 9,
                   "trunc_data": TRUNC_DATA, "levels": LEVELS, "iters": ITERS, "lambda": LAM, "trunc": TRUNC,
                   "fast_skip": True, "crop": list(CROP)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------------------ GPU arm

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("bp.cu", "sweep_body.cuh", "bps_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1709_06509_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(profile_name: str):
    """DRAM bytes per sweep launch recorded by ncu for this kernel source, else None."""
    path = os.path.join(ROOT, "profiles", profile_name)
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def pixel_labels_recomputed(st, trace) -> float:
    """Sum over the half-sweeps of a solve of (recomputed pixels) x Dp (labels a pixel moves)."""
    Dp = (st.D + 15) // 16 * 16
    return float(trace.sum()) * Dp


def torch_from(a, dev):
    import torch

    return torch.from_numpy(a).to(dev)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def time_region(fn, steps, flush, stream, flush_value=1) -> list[float]:
    """CUDA-event time (ms) of each of `steps` calls of fn on `stream`; L2 flushed before each,
    outside the events."""
    import torch

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_((flush_value + k) & 0xFF)
        ev[k][0].record(stream)
        fn()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def pair_launches(bps, st, window: int) -> int:
    """Kernels one bps_stereo call of a context launches: the NCC kernel (scale 1 fused; the
    tensor-core kernel adds its FP64 follow-up), the pyramid kernels of scales 2.. (two scales a
    launch), the solve-start kernel, one copy kernel per scale that does not start from its parent's
    records itself, 2 * ITERS half-sweeps per scale (one launch for a cluster scale), and the
    read-out."""
    if st.msg_type == bps.BPS_MSG_FP16:
        # float costs: scale 1 is not fused into the NCC kernel; every finer scale's start is copied
        return 1 + LEVELS // 2 + 1 + (LEVELS - 1) + 2 * ITERS * LEVELS + 1
    ncc = 2 if st.ncc_kernel(window, TRUNC_DATA) == bps.BPS_NCC_TENSOR else 1
    vs = st.variants()
    cluster_scales = [lvl for lvl in range(LEVELS) if vs[lvl] & bps.BPS_VARIANT_CLUSTER]
    sweeps = sum(1 if lvl in cluster_scales else 2 * ITERS for lvl in range(LEVELS))
    copies = sum(1 for lvl in cluster_scales if lvl < LEVELS - 1)
    return ncc + (max(0, LEVELS - 2) + 1) // 2 + 1 + copies + sweeps + 1


def batch_report(args):
    """Aggregate Mpix*disp/s of one batch of mixed pairs: a per-pair loop of bps_stereo graphs
    against one bps_batch_stereo call (concurrent chains, or one persistent launch), each as a
    CUDA graph, K timed repetitions after W warm-ups, L2 flushed between repetitions."""
    import torch

    import paper_1709_06509_gb300 as bps
    from paper_1709_06509_gb300 import autotune, synth

    dev = torch.device("cuda", 0)
    specs = synth.batch_specs(args.batch_report)
    pairs = [synth.make_pair(seed, W, H, D, 8, 3.0) for seed, W, H, D in specs]
    form = bps.BPS_MSG_FP16 if args.batch_form == "fp16" else bps.BPS_MSG_U8
    sts = [bps.Stereo(p.left.shape[1], p.left.shape[0], p.D, LEVELS, form, device=dev) for p in pairs]
    Ls = [torch.from_numpy(p.left).to(dev) for p in pairs]
    Rs = [torch.from_numpy(p.right).to(dev) for p in pairs]
    outs = [torch.empty(p.left.shape, dtype=torch.int32, device=dev) for p in pairs]
    windows = [7] * len(pairs)
    for st, L, R in zip(sts, Ls, Rs):
        if form == bps.BPS_MSG_U8:  # the NCC shapes are tuned on the u8 form's int16 costs
            autotune.tune_ncc(st, L, R, 7, TRUNC_DATA, reps=2)
        autotune.tune(st, L, R, 7, TRUNC_DATA, ITERS, LAM, TRUNC, reps=1)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    units = sum(p.left.size * p.D for p in pairs)
    batch = bps.Batch(sts)
    modes = {
        "per_pair_loop": lambda: [st.stereo(L, R, 7, TRUNC_DATA, ITERS, LAM, TRUNC, graph=True, out=o)
                                  for st, L, R, o in zip(sts, Ls, Rs, outs)],
        "batch_concurrent_chains": lambda: batch.stereo(Ls, Rs, windows, TRUNC_DATA, ITERS, LAM, TRUNC, outs=outs),
        "batch_persistent": lambda: batch.stereo(Ls, Rs, windows, TRUNC_DATA, ITERS, LAM, TRUNC, persistent=True,
                                                 outs=outs),
    }
    res = {}
    for name, fn in modes.items():
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        total = 0.0
        for _ in range(args.steps):
            flush.fill_(3)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            total += a.elapsed_time(b)
        res[name] = {"value": units * args.steps / (total / 1e3) / 1e6, "ms_per_batch": total / args.steps}
    batch.close()
    for st in sts:
        st.close()
    print(json.dumps({"metric": METRIC, "unit": UNIT, "workload": f"batch of {len(pairs)} mixed pairs", "form": args.batch_form,
                      "pixels_x_labels": units, "steps": args.steps, "modes": res}))


def warmstart_report(args):
    """The learned warm start: trained on converged-BP labels of seeded 450x375 D64 pairs
    (seeds 10000..), evaluated on held-out seeds (20000..) for the iterations it saves at equal
    final energy, and timed against the plain solve at that energy."""
    import torch

    import paper_1709_06509_gb300 as bps
    from paper_1709_06509_gb300 import warmstart

    hd = args.warmstart_workload == "hd"
    W, H, D, window = (1920, 1080, 256, 9) if hd else (450, 375, 64, 7)
    n_train = args.train_pairs or (48 if hd else 2000)
    n_eval = args.eval_pairs or (8 if hd else 200)
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    train_imgs = warmstart.generate_pairs(range(10000, 10000 + n_train), W, H, D)
    eval_imgs = warmstart.generate_pairs(range(20000, 20000 + n_eval), W, H, D)
    t_gen = time.perf_counter() - t0
    feats, targets = warmstart.make_dataset(None, W, H, D, window, TRUNC_DATA, LAM, TRUNC, label_iters=40,
                                            device=dev, images=train_imgs)
    net = warmstart.WarmNet(D, seed=0, device=dev)
    t1 = time.perf_counter()
    losses = warmstart.train(net, feats, targets, epochs=15, batch=8 if hd else 32, lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    del feats, targets
    res = warmstart.evaluate(net, None, W, H, D, window, TRUNC_DATA, LAM, TRUNC, iters_list=(1, 2, 3, 4, 5, 6, 8, 10),
                             device=dev, images=eval_imgs)
    eq = warmstart.iterations_at_equal_energy(res, ITERS)
    # the warm start acts on the coarse scales: fewer iterations there, the finest scale's fixed
    sched = warmstart.evaluate_schedules(net, eval_imgs, W, H, D, window, TRUNC_DATA, LAM, TRUNC,
                                         finest_iters=ITERS, device=dev)
    # the network's own cost at this size (tensor-core forward convolutions)
    with bps.Stereo(W, H, D, LEVELS, bps.BPS_MSG_U8, device=dev) as st:
        st.build_cost_volume(torch.from_numpy(eval_imgs[0][0]).to(dev), torch.from_numpy(eval_imgs[0][1]).to(dev),
                             window, TRUNC_DATA)
        for _ in range(3):
            net.predict_messages(st, LAM, TRUNC)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(10):
            net.predict_messages(st, LAM, TRUNC)
        b.record()
        torch.cuda.synchronize()
        net_ms = a.elapsed_time(b) / 10
    # throughput at equal energy: plain solve with ITERS iterations against the warm-started
    # solve (network included) with the fewest iterations reaching the same total energy
    units = W * H * D
    timing = {}
    with bps.Stereo(W, H, D, LEVELS, bps.BPS_MSG_U8, device=dev) as st:
        Ls = [torch.from_numpy(l).to(dev) for l, _ in eval_imgs[:20]]
        Rs = [torch.from_numpy(r).to(dev) for _, r in eval_imgs[:20]]
        out = torch.empty((H, W), dtype=torch.int32, device=dev)
        for form, k in (("plain", ITERS), ("warm", eq["warm"])):
            if k is None:
                continue
            def run():
                for L, R in zip(Ls, Rs):
                    st.build_cost_volume(L, R, window, TRUNC_DATA)
                    init = net.predict_messages(st, LAM, TRUNC) if form == "warm" else None
                    st.bp_solve(k, LAM, TRUNC, init_msgs=init)
                    st.wta_disparity(out)
            run()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            run()
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / len(Ls)
            timing[form] = {"iters": k, "ms_per_pair": ms, "value": units / ms / 1e3}
    print(json.dumps({"metric": METRIC, "unit": UNIT,
                      "workload": f"learned warm start, {W}x{H} D{D} pairs ({window}x{window} window)",
                      "train_pairs": n_train, "eval_pairs": n_eval, "label_iters": 40,
                      "loss_per_epoch": losses, "energy_sum_by_iters": res, "iters_at_equal_energy": eq,
                      "coarse_schedules": sched, "network_ms_per_pair": net_ms,
                      "timing_at_equal_energy": timing, "seconds": {"generate": t_gen, "train": t_train}}))


def approx_report(args):
    """The approximate fast-converging rules against the exact skip: per rule, the benchmark step
    (both pairs, one batch graph, L2 flushed between repetitions) and a 960x540 D256 pair (one
    graph), with the recomputed pixels (trace) and the read-out energy of each pair."""
    import torch

    import paper_1709_06509_gb300 as bps
    from paper_1709_06509_gb300 import autotune, synth

    dev = torch.device("cuda", 0)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    rules = [(0, False), (1, False), (2, False), (4, False), (0, True), (1, True), (2, True)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def measure(sts, run, units):
        for _ in range(max(3, args.warmup)):
            run()
        torch.cuda.synchronize()
        total = 0.0
        for _ in range(args.steps):
            flush.fill_(5)
            e0.record()
            run()
            e1.record()
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
        return units * args.steps / (total / 1e3) / 1e6, total / args.steps

    out = {"metric": METRIC, "unit": UNIT, "report": "approximate skip rules", "rules": []}
    groups = {"benchmark_pairs": [synth.workload_pair(n) for n in ("tsukuba_384x288_d16", "teddy_450x375_d64")],
              "qhd_960x540_d256": [synth.workload_pair("qhd_960x540_d256")]}
    ctx = {}
    for gname, prs in groups.items():
        sts = [bps.Stereo(p.left.shape[1], p.left.shape[0], p.D, LEVELS, bps.BPS_MSG_U8, device=dev) for p, _ in prs]
        Ls = [torch.from_numpy(p.left).to(dev) for p, _ in prs]
        Rs = [torch.from_numpy(p.right).to(dev) for p, _ in prs]
        outs = [torch.empty(p.left.shape, dtype=torch.int32, device=dev) for p, _ in prs]
        ws = [w for _, w in prs]
        for st, L, R, w in zip(sts, Ls, Rs, ws):
            autotune.tune_ncc(st, L, R, w, TRUNC_DATA, reps=2)
            autotune.tune(st, L, R, w, TRUNC_DATA, ITERS, LAM, TRUNC, reps=1)
        ctx[gname] = (prs, sts, Ls, Rs, outs, ws, bps.Batch(sts))
    for eps, freeze in rules:
        row = {"eps": eps, "freeze": freeze}
        for gname, (prs, sts, Ls, Rs, outs, ws, batch) in ctx.items():
            for st in sts:
                st.set_skip_rule(eps, freeze)
            units = work_units(prs)
            value, ms = measure(sts, lambda: batch.stereo(Ls, Rs, ws, TRUNC_DATA, ITERS, LAM, TRUNC, outs=outs), units)
            energies, work = [], []
            for st, L, R, w in zip(sts, Ls, Rs, ws):
                st.build_cost_volume(L, R, w, TRUNC_DATA)
                st.bp_solve(ITERS, LAM, TRUNC, skip=True)
                energies.append(int(st.energy(st.wta_disparity(), LAM, TRUNC)[0].item()))
                work.append(int(st.get_trace().sum()))
            row[gname] = {"value": value, "ms": ms, "energy": energies, "recomputed_pixels": work}
        out["rules"].append(row)
    base = out["rules"][0]
    for row in out["rules"]:
        for gname in groups:
            r, b = row[gname], base[gname]
            r["energy_gap_rel"] = [(e - e0_) / e0_ for e, e0_ in zip(r["energy"], b["energy"])]
            r["speedup"] = r["value"] / b["value"]
            r["work_ratio"] = sum(r["recomputed_pixels"]) / sum(b["recomputed_pixels"])
    print(json.dumps(out))


def bad_pixel_rate(disp, pair) -> float:
    """Share of visible (non-occluded) pixels whose disparity is off the generator's truth by more than 1."""
    import numpy as np

    vis = ~pair.occluded
    return float((np.abs(disp.astype(np.int64) - pair.disparity)[vis] > 1).mean())


def forms_report(args):
    """The message forms side by side: int32 messages, u8 messages (the same integer method, bit-exact),
    fp16 messages on the unquantised float cost (judged by its energy gap against the FP64 oracle of
    the float form, scored by the oracle's own energy).  One graph per pair, L2 flushed between
    repetitions; the 1920x1080 pair has no oracle run (hours on one core)."""
    import numpy as np
    import torch

    import oracle
    import paper_1709_06509_gb300 as bps
    from paper_1709_06509_gb300 import autotune, synth

    dev = torch.device("cuda", 0)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    forms = {"int32": bps.BPS_MSG_INT32, "u8": bps.BPS_MSG_U8, "fp16": bps.BPS_MSG_FP16}
    out = {"metric": METRIC, "unit": UNIT, "report": "message forms", "pairs": {}}
    for name in ("tsukuba_384x288_d16", "teddy_450x375_d64", "hd_1920x1080_d256"):
        pair, window = synth.workload_pair(name)
        H, W = pair.left.shape
        L = torch.from_numpy(pair.left).to(dev)
        R = torch.from_numpy(pair.right).to(dev)
        disp = torch.empty((H, W), dtype=torch.int32, device=dev)
        row = {}
        ref = None
        if not name.startswith("hd"):
            ref = oracle.stereo_f64(pair.left, pair.right, pair.D, window, TRUNC_DATA, LEVELS, ITERS, float(LAM), TRUNC)
        for fname, form in forms.items():
            with bps.Stereo(W, H, pair.D, LEVELS, form, device=dev) as st:
                if form == bps.BPS_MSG_U8:
                    autotune.tune_ncc(st, L, R, window, TRUNC_DATA, reps=2)
                if form != bps.BPS_MSG_INT32:  # the int32 form has the generic kernel only
                    autotune.tune(st, L, R, window, TRUNC_DATA, ITERS, LAM, TRUNC, reps=1)
                steps = max(3, args.steps if not name.startswith("hd") else min(args.steps, 10))
                for _ in range(3):
                    st.stereo(L, R, window, TRUNC_DATA, ITERS, LAM, TRUNC, graph=True, out=disp)
                torch.cuda.synchronize()
                total = 0.0
                for _ in range(steps):
                    flush.fill_(7)
                    e0.record()
                    st.stereo(L, R, window, TRUNC_DATA, ITERS, LAM, TRUNC, graph=True, out=disp)
                    e1.record()
                    torch.cuda.synchronize()
                    total += e0.elapsed_time(e1)
                ei, ef = st.energy(disp, LAM, TRUNC)
                d = disp.cpu().numpy()
                r = {"value": W * H * pair.D * steps / (total / 1e3) / 1e6, "ms": total / steps,
                     "bad_pixel_rate": bad_pixel_rate(d, pair)}
                if form == bps.BPS_MSG_FP16:
                    r["energy_fp64_gpu"] = float(ef.item())
                    if ref is not None:
                        e_gpu = oracle.energy(ref["cost"], d, float(LAM), TRUNC)  # GPU labels, oracle's scoring
                        r["energy_gap_rel"] = (e_gpu - ref["energy"]) / ref["energy"]
                        r["label_disagreement"] = float((d != ref["disp"]).mean())
                        r["oracle_bad_pixel_rate"] = bad_pixel_rate(ref["disp"], pair)
                else:
                    r["energy_int64"] = int(ei.item())
                row[fname] = r
        row["fp16_vs_int32"] = row["fp16"]["value"] / row["int32"]["value"]
        row["u8_vs_int32"] = row["u8"]["value"] / row["int32"]["value"]
        out["pairs"][name] = row
    print(json.dumps(out))


def sparse_report(args):
    """The finest scale over K candidate labels per pixel (the abstract's sparse set of NCC matches)
    against the exact dense solve: one graph per pair, L2 flushed between repetitions; the energy
    gap is relative to the dense solve's energy on the same integer cost."""
    import torch

    import paper_1709_06509_gb300 as bps
    from paper_1709_06509_gb300 import autotune, synth

    dev = torch.device("cuda", 0)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"metric": METRIC, "unit": UNIT, "report": "sparse candidates", "pairs": {}}
    for name, ks in (("tsukuba_384x288_d16", (2, 4, 8)), ("teddy_450x375_d64", (4, 8, 16, 32)),
                     ("hd_1920x1080_d256", (4, 8, 16, 32))):
        pair, window = synth.workload_pair(name)
        H, W = pair.left.shape
        L = torch.from_numpy(pair.left).to(dev)
        R = torch.from_numpy(pair.right).to(dev)
        disp = torch.empty((H, W), dtype=torch.int32, device=dev)
        rows = {}
        with bps.Stereo(W, H, pair.D, LEVELS, bps.BPS_MSG_U8, device=dev) as st:
            autotune.tune_ncc(st, L, R, window, TRUNC_DATA, reps=2)
            autotune.tune(st, L, R, window, TRUNC_DATA, ITERS, LAM, TRUNC, reps=1)
            steps = max(3, args.steps if not name.startswith("hd") else min(args.steps, 10))
            for K in (0,) + ks:
                st.set_candidates(K)
                for _ in range(3):
                    st.stereo(L, R, window, TRUNC_DATA, ITERS, LAM, TRUNC, graph=True, out=disp)
                torch.cuda.synchronize()
                total = 0.0
                for _ in range(steps):
                    flush.fill_(9)
                    e0.record()
                    st.stereo(L, R, window, TRUNC_DATA, ITERS, LAM, TRUNC, graph=True, out=disp)
                    e1.record()
                    torch.cuda.synchronize()
                    total += e0.elapsed_time(e1)
                e = int(st.energy(disp, LAM, TRUNC)[0].item())
                rows["dense" if K == 0 else f"K{K}"] = {
                    "value": W * H * pair.D * steps / (total / 1e3) / 1e6, "ms": total / steps, "energy": e,
                    "bad_pixel_rate": bad_pixel_rate(disp.cpu().numpy(), pair)}
            st.set_candidates(0)
        base = rows["dense"]
        for r in rows.values():
            r["speedup"] = r["value"] / base["value"]
            r["energy_gap_rel"] = (r["energy"] - base["energy"]) / base["energy"]
        out["pairs"][name] = rows
    print(json.dumps(out))


def setup_ctx(bps, autotune, pair, window, form, dev, tune_cache):
    """A context for `pair` in message form `form`, its kernel choices autotuned (untimed)."""
    H, W = pair.left.shape
    st = bps.Stereo(W, H, pair.D, LEVELS, form, device=dev)
    L, R = torch_from(pair.left, dev), torch_from(pair.right, dev)
    tuned = {}
    if form == bps.BPS_MSG_U8:  # the NCC shapes are tuned on the u8 form's int16 costs
        shape = list(autotune.tune_ncc(st, L, R, window, TRUNC_DATA, cache=tune_cache))
        tuned["ncc_kernel"] = "tensor-core" if shape[0] < 0 else "rows"
        tuned["ncc_shape"] = shape
    tuned["sweep_variants"] = autotune.tune(st, L, R, window, TRUNC_DATA, ITERS, LAM, TRUNC, reps=3, cache=tune_cache)
    return st, L, R, tuned


def solve_roofline(st, L, R, window, steps, flush, stream, per_label: int, per_label_change: int) -> dict:
    """The red-black half-sweeps of one solve as the dominant kernel: every sweep launch of the
    4 scales.  Time: graph replays of bps_bp_solve (CUDA events on the launching stream, L2
    flushed before each).  Bytes: (8s + c) per recomputed pixel-label from the live trace."""
    st.build_cost_volume(L, R, window, TRUNC_DATA)
    solve = lambda: st.bp_solve(ITERS, LAM, TRUNC, skip=True, graph=True)
    for _ in range(3):
        solve()
    ms = time_region(solve, steps, flush, stream, flush_value=11)
    trace = st.get_trace()
    launches = 2 * ITERS * LEVELS
    solve_ms = statistics.median(ms)
    pl = pixel_labels_recomputed(st, trace)
    hbm, kind = peaks()
    achieved = pl * per_label / (solve_ms / 1e3) / 1e9
    return {"achieved": achieved, "peak": hbm, "frac": achieved / hbm, "peak_kind": kind,
            "solve_ms": solve_ms, "launches_per_solve": launches, "avg_launch_us": 1e3 * solve_ms / launches,
            "algorithmic_bytes_per_launch": pl * per_label / launches,
            "pixel_labels_recomputed_per_solve": pl,
            "frac_with_change_test": pl * per_label_change / (solve_ms / 1e3) / 1e9 / hbm}


def stage_times(st, L, R, window, disp, flush, stream, reps=10) -> dict:
    """Median CUDA-event time of the cost-volume stage (NCC + pyramid launches)."""
    cost = time_region(lambda: st.build_cost_volume(L, R, window, TRUNC_DATA), reps, flush, stream, 21)
    return {"cost_volume_ms": statistics.median(cost)}


def check_headline(st, disp, gold) -> dict:
    """The timed pair's results against the oracle's (tests/golden, written by a script that calls
    only the oracle): disparity digest, int64 energy, skip trace.  Raises on a mismatch."""
    import numpy as np

    d = disp.cpu().numpy().astype("<i4")
    e = int(st.energy(disp, LAM, TRUNC)[0].item())
    tr = st.get_trace()
    g = gold["int"]
    ok = sha(d) == g["disp_sha256"] and e == g["energy"] and [int(v) for v in tr] == g["trace"]
    if not ok:
        raise RuntimeError(f"full-HD results differ from the oracle's: energy {e} vs {g['energy']}, "
                           f"digest {sha(d)[:16]} vs {g['disp_sha256'][:16]}")
    return {"disp_sha256": sha(d), "energy": e, "oracle_energy": g["energy"], "trace_equal": True,
            "source": "tests/golden/" + HEADLINE + ".json"}


def fp16_key(bps, autotune, pair, window, dev, args, flush, stream, gold) -> dict:
    """The fp16-message form on the headline pair: throughput, and its energy gap and label
    disagreement against the FP64 oracle's result."""
    import numpy as np
    import torch

    st, L, R, tuned = setup_ctx(bps, autotune, pair, window, bps.BPS_MSG_FP16, dev, args.tune_cache)
    disp = torch.empty(pair.left.shape, dtype=torch.int32, device=dev)
    step = lambda: st.stereo(L, R, window, TRUNC_DATA, ITERS, LAM, TRUNC, graph=True, out=disp)
    for _ in range(args.warmup):
        step()
    ms = time_region(step, args.steps, flush, stream, flush_value=41)
    total = sum(ms)
    units = pair.left.size * pair.D
    _, ef = st.energy(disp, LAM, TRUNC)
    e = float(ef.item())
    d = disp.cpu().numpy()
    out = {"value": units * len(ms) / (total / 1e3) / 1e6, "unit": UNIT, "ms_per_step": total / len(ms),
           "dtype": "fp16 messages, fp32 costs and arithmetic, FP64 energy", "energy_fp64": e,
           "autotuned": tuned}
    if gold:
        g = gold["f64"]
        ref = float.fromhex(g["energy_hex"])
        out["energy_gap_rel"] = (e - ref) / ref
        path = os.path.join(ROOT, "tests", "golden", g["disp_file"])
        if os.path.exists(path):
            ref_d = np.load(path)["disp"].astype(np.int32)
            out["label_disagreement"] = float((d != ref_d).mean())
        out["oracle"] = "FP64 oracle of the float-message form (tests/golden/" + HEADLINE + ".json)"
    roof = solve_roofline(st, L, R, window, max(3, min(args.steps, 20)), flush, stream, 2 * 8 + 4, 2 * 12 + 4)
    out["roofline"] = {"bound": "hbm", "achieved": roof["achieved"], "peak": roof["peak"], "unit": "GB/s",
                       "frac": roof["frac"], "bytes_model": "(8s + c) = 20 B per recomputed pixel-label "
                       "(s = 2 B fp16 message, c = 4 B fp32 cost)", "solve_ms": roof["solve_ms"]}
    out["gpu_launches_per_step"] = pair_launches(bps, st, window)
    st.close()
    return out


def c2_key(bps, autotune, dev, args, flush, stream, rank) -> dict:
    """The 384x288 D16 + 450x375 D64 pairs as one batch graph (concurrent chains), L2 flushed
    between steps, results checked against the oracle."""
    import numpy as np
    import torch

    from paper_1709_06509_gb300 import shard, synth

    pairs = [synth.workload_pair(n, shard.seed_offset(rank)) for n in C2_PAIRS]
    ctxs, tuned = [], {}
    for pair, window in pairs:
        st, L, R, t = setup_ctx(bps, autotune, pair, window, bps.BPS_MSG_U8, dev, args.tune_cache)
        ctxs.append((st, L, R, window))
        tuned[f"{st.W}x{st.H}_D{st.D}"] = t
    sts = [c[0] for c in ctxs]
    Ls, Rs, ws = [c[1] for c in ctxs], [c[2] for c in ctxs], [c[3] for c in ctxs]
    outs = [torch.empty(p.left.shape, dtype=torch.int32, device=dev) for p, _ in pairs]
    batch = bps.Batch(sts)
    joint = autotune.tune_batch(batch, sts, Ls, Rs, ws, TRUNC_DATA, ITERS, LAM, TRUNC, cache=args.tune_cache)
    for st, vs in zip(sts, joint):
        tuned[f"{st.W}x{st.H}_D{st.D}"]["sweep_variants"] = vs
    step = lambda: batch.stereo(Ls, Rs, ws, TRUNC_DATA, ITERS, LAM, TRUNC, skip=True, graph=True, outs=outs)
    for _ in range(args.warmup):
        step()
    steps = max(args.steps, 20)
    ms = time_region(step, steps, flush, stream, flush_value=51)
    total = sum(ms)
    units = work_units(pairs)
    res = {"workload": "384x288 D16 + 450x375 D64 pairs (7x7 window; one step = both, one batch graph)",
           "value": units * steps / (total / 1e3) / 1e6, "unit": UNIT, "ms_per_step": total / steps,
           "l2": "flushed between timed steps (256 MiB write)", "autotuned": tuned}
    if rank == 0:
        import oracle

        ctx = oracle.openmp(os.cpu_count() or 1) if oracle.openmp_available() else None
        if ctx:
            ctx.__enter__()
        try:
            for (pair, window), (st, _, _, _), o in zip(pairs, ctxs, outs):
                ref = oracle_run(pair, window)
                e = int(st.energy(o, LAM, TRUNC)[0].item())
                if not np.array_equal(o.cpu().numpy(), ref["disp"]) or e != ref["energy"] or \
                        not np.array_equal(st.get_trace(), ref["trace"]):
                    raise RuntimeError(f"{st.W}x{st.H} D{st.D}: the timed batch's results differ from the oracle's")
        finally:
            if ctx:
                ctx.__exit__(None, None, None)
        res["oracle_match"] = "disparities, int64 energies and skip traces equal to the oracle's"
    batch.close()
    for st in sts:
        st.close()
    return res


def write_trace_jsonl(path, st, L, R, window, pair):
    """Per iteration count k (every scale runs k iterations): the read-out's energy and, per
    half-sweep of the finest scale, the pixels recomputed and the fraction of that colour's pixels
    left alone (converged, in the fast-converging sense of the skip)."""
    H, W = pair.left.shape
    even = (W * H + 1) // 2
    with open(path, "w") as fh:
        for k in range(1, ITERS + 1):
            disp = st.stereo(L, R, window, TRUNC_DATA, k, LAM, TRUNC, graph=False)
            e = int(st.energy(disp, LAM, TRUNC)[0].item())
            tr = [int(v) for v in st.get_trace()]
            finest = tr[-2 * k:]
            conv = [1.0 - n / (even if t % 2 == 0 else W * H - even) for t, n in enumerate(finest)]
            fh.write(json.dumps({"workload": HEADLINE, "iters": k, "energy": e, "finest_recomputed": finest,
                                 "finest_converged_frac": conv, "trace": tr}) + "\n")


def blocking_report(args):
    """Blocking depth 1 against 2 for a scale's first iteration (BPS_VARIANT_BLOCK2 cleared or set
    on every scale below the coarsest, the other variant bits as tuned): the graph-replayed solve
    time (median, L2 flushed) and the first iteration's profile-mode launch time per scale; both
    depths must give the same disparities, energy and trace."""
    import numpy as np
    import torch

    import paper_1709_06509_gb300 as bps
    from paper_1709_06509_gb300 import autotune, synth

    dev = torch.device("cuda", 0)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    K = bps.BPS_VARIANT_BLOCK2
    out = {"report": "temporal blocking of a scale's first iteration", "pairs": {}}
    for name in ("c3_1280x720_d64", HEADLINE):
        pair, window = synth.workload_pair(name)
        st, L, R, tuned = setup_ctx(bps, autotune, pair, window, bps.BPS_MSG_U8, dev, args.tune_cache)
        base = st.variants()
        rows, ref = {}, None
        for depth in (1, 2):
            vs = [(v | K) if depth == 2 and lvl < LEVELS - 1 else (v & ~K) for lvl, v in enumerate(base)]
            for lvl, v in enumerate(vs):
                st.set_variant(lvl, v)
            st.build_cost_volume(L, R, window, TRUNC_DATA)
            solve = lambda: st.bp_solve(ITERS, LAM, TRUNC, skip=True, graph=True)
            for _ in range(3):
                solve()
            ms = statistics.median(time_region(solve, max(5, args.steps), flush, stream, flush_value=13))
            firsts = []
            for _ in range(3):
                flush.fill_(5)
                st.build_cost_volume(L, R, window, TRUNC_DATA)
                st.bp_solve(ITERS, LAM, TRUNC, skip=True, profile=True)
                t = st.read_launch_times()
                firsts.append([t[2 * ITERS * (LEVELS - 1 - lvl)] + t[2 * ITERS * (LEVELS - 1 - lvl) + 1]
                               for lvl in range(LEVELS)])
            disp = st.wta_disparity()
            res = (np.asarray(disp.cpu()).tobytes(), int(st.energy(disp, LAM, TRUNC)[0].item()),
                   [int(v) for v in st.get_trace()])
            if ref is None:
                ref = res
            elif res != ref:
                raise RuntimeError(f"{name}: blocking depth 2 changed the result")
            rows[f"depth{depth}"] = {"sweep_variants": vs, "solve_ms": ms,
                                     "first_iteration_ms_per_scale": [min(f[l] for f in firsts) for l in range(LEVELS)]}
        out["pairs"][name] = {"tuned": tuned, **rows, "same_result": True}
        st.close()
    print(json.dumps(out))


def sync_report(args):
    """bps_measure_sync_costs for grids of 1, 2 and 3 CTAs a SM: the phase separation the persistent
    form pays (a grid barrier) against the chained form's (a PDL kernel boundary in a graph)."""
    import torch

    import paper_1709_06509_gb300 as bps

    dev = torch.device("cuda", 0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    rows = {}
    for per_sm in (1, 2, 3):
        barrier_us, boundary_us = bps.bps_measure_sync_costs(sms * per_sm, 2000)
        rows[f"{per_sm * sms}_ctas"] = {"grid_barrier_us": barrier_us, "pdl_kernel_boundary_us": boundary_us}
    print(json.dumps({"report": "phase separation costs", "phases": 2000, "sms": sms, "costs": rows}))


def launch_report(args):
    """Per-launch CUDA-event times (profile mode) of every sweep launch of the headline pair, with
    the pixels each recomputed."""
    import torch

    import paper_1709_06509_gb300 as bps
    from paper_1709_06509_gb300 import autotune, synth

    dev = torch.device("cuda", 0)
    name = args.workload or HEADLINE
    pair, window = synth.workload_pair(name)
    form = bps.BPS_MSG_FP16 if args.form == "fp16" else bps.BPS_MSG_U8
    st, L, R, tuned = setup_ctx(bps, autotune, pair, window, form, dev, args.tune_cache)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    runs = []
    for _ in range(3):
        flush.fill_(3)
        st.build_cost_volume(L, R, window, TRUNC_DATA)
        st.bp_solve(ITERS, LAM, TRUNC, skip=True, profile=True)
        runs.append(st.read_launch_times())
    t = [min(r[k] for r in runs) for k in range(len(runs[0]))]
    print(json.dumps({"workload": name, "form": args.form, "autotuned": tuned, "trace": [int(v) for v in st.get_trace()],
                      "launch_ms": t, "total_ms": sum(t)}))
    st.close()


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.sparse_report:
        return sparse_report(args)
    if args.batch_report:
        return batch_report(args)
    if args.forms_report:
        return forms_report(args)
    if args.approx_report:
        return approx_report(args)
    if args.warmstart_report:
        return warmstart_report(args)
    if args.launch_report:
        return launch_report(args)
    if args.sync_report:
        return sync_report(args)
    if args.blocking_report:
        return blocking_report(args)
    args.warmup = max(3, args.warmup)  # at least three untimed warm-up steps
    rank, world, local = dist_env()
    import torch

    import paper_1709_06509_gb300 as bps
    from paper_1709_06509_gb300 import _build, autotune, shard, synth

    if not os.path.exists(bps.LIB_PATH) or _build.is_stale():
        if rank == 0 or world == 1:
            _build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        dist.barrier()
        _build.build()  # no-op once rank 0 has built

    name = args.workload if (args.ncu_case and args.workload) else HEADLINE
    pair, window = synth.workload_pair(name, shard.seed_offset(rank))
    form = bps.BPS_MSG_FP16 if (args.ncu_case and args.form == "fp16") else bps.BPS_MSG_U8
    st, L, R, tuned = setup_ctx(bps, autotune, pair, window, form, dev, args.tune_cache)
    if args.ncu_case and args.ncc_kernel:
        st.set_ncc_kernel(bps.BPS_NCC_TENSOR if args.ncc_kernel == "tensor" else bps.BPS_NCC_ROWS)
    if args.ncu_case and args.variants:
        for lvl, v in enumerate(int(x) for x in args.variants.split(",")):
            st.set_variant(lvl, v)
    disp = torch.empty(pair.left.shape, dtype=torch.int32, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        st.stereo(L, R, window, TRUNC_DATA, ITERS, LAM, TRUNC, skip=True, graph=True, out=disp)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if args.ncu_case:
        for _ in range(args.steps):
            step()
        torch.cuda.synchronize()
        return
    props = torch.cuda.get_device_properties(dev)
    uuid = str(getattr(props, "uuid", "") or "")
    sampler = ClockSampler(("GPU-" + uuid if uuid and not uuid.startswith("GPU-") else uuid) or str(local))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.2)
    ms = time_region(step, args.steps, flush, stream)
    clocks = sampler.stop()
    if world > 1:
        torch.distributed.barrier()
    total_ms = sum(ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    units = pair.left.size * pair.D * world
    value = units * args.steps / (total_ms / 1e3) / 1e6

    # the timed step's results: against the oracle's (rank 0 holds the golden pair's seeds)
    gold = golden() if rank == 0 else None
    verified = check_headline(st, disp, gold) if gold else {"oracle_match": "no golden file"}

    # dominant kernel: the red-black half-sweeps of the solve, graph-timed, algorithmic bytes
    # (8s + c) = 10 B per recomputed pixel-label of the u8 form (1 B messages, 2 B costs); the
    # change test of the skip reads the 4 old outgoing messages too: (12s + c) = 14 B
    roof = solve_roofline(st, L, R, window, max(3, min(args.steps, 20)), flush, stream, 10, 14)
    stages = stage_times(st, L, R, window, disp, flush, stream)
    traffic = ncu_traffic(f"sweep_u8_{HEADLINE}.txt")
    ncc_bytes = pair.left.size * ((pair.D + 15) // 16 * 16) * 2 * 1.25  # int16 costs of scale 0, plus scale 1

    # end to end through the public API from pinned host buffers: every step copies the images in
    # and the disparities and energy out (bps_stereo_host, one recorded graph per call)
    hL = torch.from_numpy(pair.left).pin_memory()
    hR = torch.from_numpy(pair.right).pin_memory()
    hD = torch.empty(pair.left.shape, dtype=torch.int32).pin_memory()
    hE = torch.zeros(1, dtype=torch.int64).pin_memory()
    flags = bps.BPS_FLAG_FAST_SKIP | bps.BPS_FLAG_GRAPH
    host = lambda f: bps.bps_stereo_host(st.ctx, hL, hR, pair.left.shape[1], window, TRUNC_DATA, ITERS, LAM, TRUNC,
                                         f, hD, hE, None, stream)
    for _ in range(3):
        host(flags)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        host(flags)
    e2e_sync_s = time.perf_counter() - t0
    hD.fill_(-1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        host(flags | bps.BPS_FLAG_ASYNC)
    stream.synchronize()
    e2e_s = time.perf_counter() - t0
    if not torch.equal(hD, disp.cpu()):
        raise RuntimeError("host-entry disparities differ from the device entry's")
    if world > 1:
        t = torch.tensor([e2e_s, e2e_sync_s], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s, e2e_sync_s = (float(v) for v in t.tolist())
    h2d = 2 * pair.left.size
    d2h = 4 * pair.left.size + 8
    launches_per_step = pair_launches(bps, st, window)
    if args.trace_jsonl and rank == 0:
        write_trace_jsonl(args.trace_jsonl, st, L, R, window, pair)
    extras = {}
    if not args.no_extras:
        extras["fp16"] = fp16_key(bps, autotune, pair, window, dev, args, flush, stream, gold)
        extras["c2"] = c2_key(bps, autotune, dev, args, flush, stream, rank)
    if rank == 0:
        hbm, kind = roof["peak"], roof["peak_kind"]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "1920x1080 D256 pair (one step = one pair)", "window": window,
                       "trunc_data": TRUNC_DATA, "levels": LEVELS, "iters": ITERS, "lambda": LAM, "trunc": TRUNC,
                       "fast_skip": True, "message_storage": "uint8 (exact: 0 <= m <= lambda*trunc)",
                       "cost_storage": "int16", "cuda_graph": True, "autotuned": tuned,
                       "l2": "working set 4.3 GB, far above L2; a 256 MiB buffer is also written between timed "
                             "steps", "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": roof["achieved"], "peak": hbm, "unit": "GB/s",
                         "frac": roof["frac"], "traffic": traffic,
                         "kernel": "red-black half-sweep (sweep_u8_* kernels, every launch of the 4 scales)",
                         "bytes_model": "(8s + c) = 10 B per recomputed pixel-label (s = 1 B uint8 message, "
                                        "c = 2 B int16 cost), pixels from the live skip trace",
                         "timing": "graph replays of bps_bp_solve, CUDA events on the launching stream, median",
                         "peak_kind": kind, **{k: roof[k] for k in ("solve_ms", "launches_per_solve", "avg_launch_us",
                                                                    "algorithmic_bytes_per_launch",
                                                                    "frac_with_change_test")}},
            "roofline_ncc": {"bound": "hbm", "achieved": ncc_bytes / (stages["cost_volume_ms"] / 1e3) / 1e9,
                             "peak": hbm, "unit": "GB/s",
                             "frac": ncc_bytes / (stages["cost_volume_ms"] / 1e3) / 1e9 / hbm,
                             "bytes_model": "int16 data costs written: scale 0 plus the fused scale 1 (x1.25)",
                             **stages},
            "e2e": {"value": units * args.steps / e2e_s / 1e6, "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "mode": "bps_stereo_host once per step from pinned host buffers, queued on one stream "
                            "(BPS_FLAG_ASYNC), one synchronisation after the last step",
                    "value_synchronous": units * args.steps / e2e_sync_s / 1e6},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
            "verified": verified,
            **extras,
        }
        if world == 1 and not args.no_cpu_baseline:
            crop = crop_pair(pair)
            base, par, ref = cpu_baselines(crop, window)
            with bps.Stereo(CROP[2], CROP[3], pair.D, LEVELS, bps.BPS_MSG_U8, device=dev) as sc:
                cd = sc.stereo(torch_from(crop.left, dev), torch_from(crop.right, dev), window, TRUNC_DATA, ITERS,
                               LAM, TRUNC, graph=True)
                ce = int(sc.energy(cd, LAM, TRUNC)[0].item())
                import numpy as np

                if not np.array_equal(cd.cpu().numpy(), ref["disp"]) or ce != ref["energy"] or \
                        not np.array_equal(sc.get_trace(), ref["trace"]):
                    raise RuntimeError("GPU results on the CPU sample differ from the oracle's")
            base["gpu_match"] = "the GPU's disparities, energy and trace on the sample equal the oracle's"
            line["cpu_baseline"] = base
            if par:
                line["cpu_baseline_parallel"] = par
        print(json.dumps(line))
    st.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
