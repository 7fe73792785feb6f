"""bps_energy_noalloc: the energy entry point for callers that cannot allocate device memory
(real-time loops that may not wait on an allocator, programs whose device memory belongs to an
allocator this library cannot reach, code under a fixed memory budget).

Its exact int64 energy must equal the CPU oracle's energy of the same labelling on the same
cost volume, on two calls in a row that reuse its shared scratch array, and the context-based
bps_energy's.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
import paper_1709_06509_gb300 as bps
from paper_1709_06509_gb300 import _build, synth


@pytest.mark.gpu
def test_noalloc_energy_matches_the_oracle_twice():
    import torch

    _build.build()
    dev = torch.device("cuda:0")
    W, H, D, lam, T = 130, 77, 24, 10, 2
    pair = synth.make_pair(77, W, H, D, 4, 2.0)
    with bps.Stereo(W, H, D, 3, bps.BPS_MSG_U8, device=dev) as st:
        st.build_cost_volume(torch.from_numpy(pair.left).to(dev), torch.from_numpy(pair.right).to(dev), 5, 20)
        st.bp_solve(6, lam, T)
        disp_bp = st.wta_disparity()
        cost = st.export_cost(0).contiguous()
        c0 = oracle.quantise(oracle.ncc(pair.left, pair.right, D, 5), 20)
        assert np.array_equal(cost.cpu().numpy(), c0)  # the volume the call reads is the oracle's
        rng = np.random.default_rng(5)
        disp_rand = torch.from_numpy(rng.integers(0, D, (H, W)).astype(np.int32)).to(dev)
        for disp in (disp_bp, disp_rand):  # two calls in a row on the shared scratch
            got = torch.full((1,), -1, dtype=torch.int64, device=dev)
            bps.bps_energy_noalloc(cost, disp, W, H, D, lam, T, got)
            torch.cuda.synchronize()
            want = oracle.energy(c0, disp.cpu().numpy(), lam, T)
            assert int(got.item()) == want
            assert int(st.energy(disp, lam, T)[0].item()) == want


def test_noalloc_rejects_oversized_images_before_launching():
    _build.build()
    lib = bps.lib()
    side = 1 << 13  # 8192 x 8192 > BPS_NOALLOC_MAX_PIXELS
    assert side * side > bps.BPS_NOALLOC_MAX_PIXELS
    rc = lib.bps_energy_noalloc(256, 256, side, side, 4, 1, 1, 256, None)
    assert rc == bps.BPS_ERR_UNSUPPORTED
    assert lib.bps_energy_noalloc(None, 256, 4, 4, 4, 1, 1, 256, None) == bps.BPS_ERR_ARG
