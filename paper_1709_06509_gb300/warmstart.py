"""Learned warm start of the hierarchical BP.

A 4-layer 3x3 convolutional network (32 channels, BF16 weights and activations, FP32
accumulation) maps the coarsest scale's cost volume, min-pooled to ceil(D/8) channels, to the
four directional messages of the coarsest scale (4 * D channels).  Its prediction, rounded
and min-normalised, becomes the start messages of the solve (BPS_FLAG_WARM_START), which
otherwise starts from zero.  Labels for training are the coarsest-scale messages of BP run
to convergence on seeded synthetic pairs.  Every kernel is in csrc/warmnet.cu behind the C
ABI; this module holds the weights (device tensors), sequences the kernels and runs the
training loop.  The BP energy judges the result: evaluate() compares the final energy of the
warm-started and the plain solve for every iteration count, and the warm start is only
worth using where it reaches the plain solve's energy in fewer iterations.
"""
from __future__ import annotations

import math

import numpy as np

from . import (BPS_MSG_U8, Stereo, bps_warmnet_adam, bps_warmnet_conv3x3, bps_warmnet_conv3x3_backward,
               bps_warmnet_features, bps_warmnet_messages, bps_warmnet_mse, level_dims)
from . import synth

FEATURE_SCALE = 1.0 / 64.0


class WarmNet:
    """The network: conv(Cin->C) ReLU, conv(C->C) ReLU, conv(C->C) ReLU, conv(C->4D)."""

    def __init__(self, D: int, channels: int = 32, seed: int = 0, device="cuda"):
        import torch

        self.D, self.C = D, channels
        self.cin = (D + 7) // 8
        self.shapes = [(self.cin, channels), (channels, channels), (channels, channels), (channels, 4 * D)]
        self.device = torch.device(device)
        rng = np.random.default_rng(seed)
        self.w32, self.b, self.w16 = [], [], []
        for cin, cout in self.shapes:
            bound = math.sqrt(6.0 / (cin * 9))  # He-uniform for the ReLU layers
            w = rng.uniform(-bound, bound, (cout, cin, 3, 3)).astype(np.float32)
            self.w32.append(torch.from_numpy(w).to(self.device))
            self.b.append(torch.zeros(cout, dtype=torch.float32, device=self.device))
            self.w16.append(self.w32[-1].to(torch.bfloat16))
        self.b[-1].fill_(0.0)
        self.adam_m = [torch.zeros_like(t) for t in self.w32 + self.b]
        self.adam_v = [torch.zeros_like(t) for t in self.w32 + self.b]
        self.step_count = 0
        self.acts = None

    def forward(self, feat, H: int, W: int):
        """feat: BF16 [B][cin][H][W] -> FP32 [B][4D][H][W]; keeps the activations for backward."""
        import torch

        B = feat.shape[0]
        acts = [feat]
        x = feat
        for k, (cin, cout) in enumerate(self.shapes):
            last = k == len(self.shapes) - 1
            out = torch.empty((B, cout, H, W), dtype=torch.float32 if last else torch.bfloat16, device=self.device)
            bps_warmnet_conv3x3(x, x.dtype == torch.bfloat16, B, cin, H, W, self.w16[k], self.b[k], cout, not last,
                                out, not last)
            acts.append(out)
            x = out
        self.acts = acts
        return x

    def backward(self, gout, H: int, W: int):
        """Gradients of the last forward pass from gout (FP32, like the output)."""
        import torch

        B = gout.shape[0]
        gw = [None] * len(self.shapes)
        gb = [None] * len(self.shapes)
        g = gout
        for k in range(len(self.shapes) - 1, -1, -1):
            cin, cout = self.shapes[k]
            relu_out = None if k == len(self.shapes) - 1 else self.acts[k + 1]
            gw[k] = torch.empty_like(self.w32[k])
            gb[k] = torch.empty_like(self.b[k])
            gin = torch.empty((B, cin, H, W), dtype=torch.float32, device=self.device) if k > 0 else None
            x = self.acts[k]
            bps_warmnet_conv3x3_backward(g, relu_out, x, x.dtype == torch.bfloat16, B, cin, H, W, self.w16[k], cout,
                                         gin, gw[k], gb[k])
            g = gin
        return gw, gb

    def adam(self, gw, gb, lr: float = 2e-3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        self.step_count += 1
        params = self.w32 + self.b
        grads = gw + gb
        for i, (p, g) in enumerate(zip(params, grads)):
            w16 = self.w16[i] if i < len(self.w32) else None
            bps_warmnet_adam(p, self.adam_m[i], self.adam_v[i], g, p.numel(), lr, beta1, beta2, eps,
                             self.step_count, w16)

    def predict_messages(self, st: Stereo, lam: int, trunc: int):
        """Start messages of the coarsest scale of `st` (its cost volume must be built):
        int32 [4][H_c][W_c][D] on the device."""
        import torch

        feat = coarse_features(st)
        wc, hc = level_dims(st.W, st.H, st.levels)[-1]
        pred = self.forward(feat[None], hc, wc)
        init = torch.empty((4, hc, wc, st.D), dtype=torch.int32, device=self.device)
        bps_warmnet_messages(pred, hc, wc, st.D, lam * trunc, init)
        return init


def coarse_features(st: Stereo):
    """Network input (BF16 [ceil(D/8)][H_c][W_c]) from the coarsest cost volume of `st`."""
    import torch

    wc, hc = level_dims(st.W, st.H, st.levels)[-1]
    cost = st.export_cost(st.levels - 1)
    feat = torch.empty(((st.D + 7) // 8, hc, wc), dtype=torch.bfloat16, device=st.device)
    bps_warmnet_features(cost, hc, wc, st.D, FEATURE_SCALE, feat)
    return feat


def message_mask(hc: int, wc: int, D: int, device):
    """1 for the channels of existing neighbours, [4 * D][H_c][W_c]."""
    import torch

    m = torch.ones((4, D, hc, wc), dtype=torch.float32, device=device)
    m[0, :, 0, :] = 0
    m[1, :, -1, :] = 0
    m[2, :, :, 0] = 0
    m[3, :, :, -1] = 0
    return m.reshape(4 * D, hc, wc)


def _pair_images(args):
    seed, W, H, D, planes, sigma = args
    p = synth.make_pair(seed, W, H, D, planes, sigma)
    return p.left, p.right


def generate_pairs(seeds, W: int, H: int, D: int, planes: int = 8, sigma: float = 3.0, workers: int = 0):
    """(left, right) images of every seed, drawn in a pool of spawned processes."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os

    jobs = [(int(s), W, H, D, planes, sigma) for s in seeds]
    workers = workers or max(1, min(len(jobs), os.cpu_count() or 1))
    if workers == 1:
        return [_pair_images(j) for j in jobs]
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_pair_images, jobs, chunksize=8))


def make_dataset(seeds, W: int, H: int, D: int, window: int, trunc_data: int, lam: int, trunc: int,
                 label_iters: int, levels: int = 4, planes: int = 8, sigma: float = 3.0, device="cuda",
                 images=None):
    """(features BF16 [N][cin][H_c][W_c], targets FP32 [N][4D][H_c][W_c]): the coarsest-scale
    messages after label_iters iterations of BP from zero messages, per seed."""
    import torch

    wc, hc = level_dims(W, H, levels)[-1]
    if images is None:
        images = [_pair_images((int(s), W, H, D, planes, sigma)) for s in seeds]
    feats, targets = [], []
    with Stereo(W, H, D, levels, BPS_MSG_U8, device=device) as st:
        for left, right in images:
            pair = synth.StereoPair(left, right, None, None, D, 0)
            st.build_cost_volume(torch.from_numpy(pair.left).to(device), torch.from_numpy(pair.right).to(device),
                                 window, trunc_data)
            feats.append(coarse_features(st))
            st.bp_solve(label_iters, lam, trunc, levels=levels, skip=True)
            msg = st.export_messages(levels - 1)  # [4][hc][wc][D]
            targets.append(msg.permute(0, 3, 1, 2).reshape(4 * D, hc, wc).to(torch.float32))
    return torch.stack(feats), torch.stack(targets)


def train(net: WarmNet, feats, targets, epochs: int = 15, batch: int = 32, lr: float = 2e-3, seed: int = 0,
          log=None):
    """Adam on the masked mean squared error of the messages; returns the loss per epoch."""
    import torch

    N, _, hc, wc = feats.shape
    mask = message_mask(hc, wc, net.D, net.device)
    rng = np.random.default_rng(seed)
    losses = []
    nparts = 256
    parts = torch.zeros(nparts, dtype=torch.float32, device=net.device)
    for ep in range(epochs):
        order = rng.permutation(N)
        total, count = 0.0, 0
        for k in range(0, N - batch + 1, batch):
            idx = torch.from_numpy(order[k:k + batch]).to(net.device)
            x = feats.index_select(0, idx).contiguous()
            t = targets.index_select(0, idx).contiguous()
            pred = net.forward(x, hc, wc)
            m = mask.expand(batch, -1, -1, -1).contiguous()
            grad = torch.empty_like(pred)
            bps_warmnet_mse(pred, t, m, pred.numel(), grad, parts, nparts)
            gw, gb = net.backward(grad, hc, wc)
            net.adam(gw, gb, lr=lr)
            total += float(parts.sum().item())
            count += 1
        losses.append(total / max(count, 1))
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.4f}")
    return losses


def evaluate(net: WarmNet, seeds, W: int, H: int, D: int, window: int, trunc_data: int, lam: int, trunc: int,
             iters_list=(2, 3, 4, 5, 6, 8, 10), levels: int = 4, planes: int = 8, sigma: float = 3.0,
             device="cuda", images=None):
    """Final BP energy (int64, summed over the seeds) of the plain and the warm-started solve
    for each iteration count, and the per-pair energies for the fallback judgement."""
    import torch

    plain = {k: 0 for k in iters_list}
    warm = {k: 0 for k in iters_list}
    better = {k: 0 for k in iters_list}
    if images is None:
        images = [_pair_images((int(s), W, H, D, planes, sigma)) for s in seeds]
    with Stereo(W, H, D, levels, BPS_MSG_U8, device=device) as st:
        for left, right in images:
            pair = synth.StereoPair(left, right, None, None, D, 0)
            st.build_cost_volume(torch.from_numpy(pair.left).to(device), torch.from_numpy(pair.right).to(device),
                                 window, trunc_data)
            init = net.predict_messages(st, lam, trunc)
            for k in iters_list:
                st.bp_solve(k, lam, trunc, skip=True)
                ep = int(st.energy(st.wta_disparity(), lam, trunc)[0].item())
                st.bp_solve(k, lam, trunc, skip=True, init_msgs=init)
                ew = int(st.energy(st.wta_disparity(), lam, trunc)[0].item())
                plain[k] += ep
                warm[k] += ew
                better[k] += int(ew <= ep)
    return {"plain": plain, "warm": warm, "warm_not_worse_pairs": better, "pairs": len(images)}


def evaluate_schedules(net: WarmNet, images, W: int, H: int, D: int, window: int, trunc_data: int, lam: int,
                       trunc: int, coarse_iters=(0, 1, 2, 3, 4, 6, 10), finest_iters: int = 10, levels: int = 4,
                       device="cuda"):
    """Iterations the warm start saves at the coarse scales, the finest scale's count fixed: for
    each scale l >= 1 alone (the others at finest_iters) and for all coarse scales together, the
    final energy (int64, summed over the pairs) of the plain and the warm-started solve per coarse
    iteration count (bps_bp_solve_schedule)."""
    import torch

    groups = {f"scale_{l}": [l] for l in range(1, levels)}
    groups["all_coarse"] = list(range(1, levels))
    out = {g: {"plain": {k: 0 for k in coarse_iters}, "warm": {k: 0 for k in coarse_iters}} for g in groups}
    with Stereo(W, H, D, levels, BPS_MSG_U8, device=device) as st:
        for left, right in images:
            st.build_cost_volume(torch.from_numpy(left).to(device), torch.from_numpy(right).to(device), window,
                                 trunc_data)
            init = net.predict_messages(st, lam, trunc)
            for g, scales in groups.items():
                for k in coarse_iters:
                    sched = [finest_iters] * levels
                    for l in scales:
                        sched[l] = k
                    for form, start in (("plain", None), ("warm", init)):
                        st.bp_solve_schedule(sched, lam, trunc, init_msgs=start)
                        out[g][form][k] += int(st.energy(st.wta_disparity(), lam, trunc)[0].item())
    for g in groups:
        ref = out[g]["plain"][max(coarse_iters)]
        for form in ("plain", "warm"):
            ks = [k for k in sorted(coarse_iters) if out[g][form][k] <= ref]
            out[g][f"{form}_iters_at_equal_energy"] = ks[0] if ks else None
        p, w = out[g]["plain_iters_at_equal_energy"], out[g]["warm_iters_at_equal_energy"]
        out[g]["iterations_saved"] = (p - w) if (p is not None and w is not None) else None
    return out


def iterations_at_equal_energy(result, reference_iters: int = 10):
    """Smallest iteration count whose total energy is at most the plain solve's at
    reference_iters, for the plain and the warm-started solve (None if never)."""
    target = result["plain"][reference_iters]
    out = {}
    for form in ("plain", "warm"):
        ks = [k for k in sorted(result[form]) if result[form][k] <= target]
        out[form] = ks[0] if ks else None
    return out
