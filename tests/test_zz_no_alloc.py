"""bps_energy_noalloc: the energy entry point for callers that cannot allocate device memory
(inside a graph capture, in an allocation-free real-time loop, behind a foreign allocator).

It must agree with the context-based bps_energy, exactly (int64), on two calls in a row
that reuse its shared scratch array.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import paper_1709_06509_gb300 as bps
from paper_1709_06509_gb300 import synth


@pytest.mark.gpu
def test_noalloc_energy_matches_bps_energy_twice():
    from paper_1709_06509_gb300 import _build

    _build.build()
    dev = torch.device("cuda:0")
    W, H, D, lam, T = 130, 77, 24, 10, 2
    pair = synth.make_pair(77, W, H, D, 4, 2.0)
    with bps.Stereo(W, H, D, 3, bps.BPS_MSG_U8, device=dev) as st:
        st.build_cost_volume(torch.from_numpy(pair.left).to(dev), torch.from_numpy(pair.right).to(dev), 5, 20)
        st.bp_solve(6, lam, T)
        disp_bp = st.wta_disparity()
        cost = st.export_cost(0).contiguous()
        rng = np.random.default_rng(5)
        disp_rand = torch.from_numpy(rng.integers(0, D, (H, W)).astype(np.int32)).to(dev)
        for disp in (disp_bp, disp_rand):  # two calls in a row on the shared scratch
            want, _ = st.energy(disp, lam, T)
            got = torch.full((1,), -1, dtype=torch.int64, device=dev)
            bps.bps_energy_noalloc(cost, disp, W, H, D, lam, T, got)
            torch.cuda.synchronize()
            assert int(got.item()) == int(want.item())


def test_noalloc_rejects_oversized_images_before_launching():
    lib = bps.lib()
    side = 1 << 13  # 8192 x 8192 > BPS_NOALLOC_MAX_PIXELS
    assert side * side > bps.BPS_NOALLOC_MAX_PIXELS
    rc = lib.bps_energy_noalloc(256, 256, side, side, 4, 1, 1, 256, None)
    assert rc == bps.BPS_ERR_UNSUPPORTED
    assert lib.bps_energy_noalloc(None, 256, 4, 4, 4, 1, 1, 256, None) == bps.BPS_ERR_ARG
