"""The full-HD configuration (1920x1080, D = 256, 9x9 window, 4 scales, 10 iterations, lambda 10,
trunc 2, the exact fast-converging skip) against the oracle's results stored in
tests/golden/hd_1920x1080_d256.json (written by tests/golden/make_hd_golden.py, which calls only
the CPU oracle: the oracle needs about 20 minutes of 8 cores for this pair, too long for a test).

Integer forms: the int32 cost volume, the disparities (SHA-256 of the int32 bytes), the int64
energy and the skip trace must equal the oracle's, in the launch configuration the benchmark
times (bps_stereo recorded as a CUDA graph) and under every sweep variant the autotuner can pick
at these sizes.  The fp16-message form: relative energy gap to the FP64 oracle within 0.5%,
under 2% of labels different from the FP64 oracle's.
"""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_1709_06509_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
NAME = "hd_1920x1080_d256"
GOLD_PATH = os.path.join(HERE, "golden", NAME + ".json")
WINDOW, TRUNC_DATA, LEVELS, ITERS, LAM, TRUNC = 9, 20, 4, 10, 10, 2


def sha(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


@pytest.fixture(scope="module")
def gold():
    with open(GOLD_PATH) as fh:
        return json.load(fh)


@pytest.fixture(scope="module")
def pair():
    p, window = synth.workload_pair(NAME)
    assert window == WINDOW
    return p


def test_golden_file_describes_these_inputs(gold, pair):
    # the stored results belong to the generator's current bytes and the configuration above
    assert gold["left_sha256"] == sha(pair.left) and gold["right_sha256"] == sha(pair.right)
    assert (gold["W"], gold["H"], gold["D"], gold["window"]) == (1920, 1080, 256, WINDOW)
    assert (gold["trunc_data"], gold["levels"], gold["iters"], gold["lambda"], gold["trunc"]) == \
        (TRUNC_DATA, LEVELS, ITERS, LAM, TRUNC)
    for form in ("int", "f64"):
        tr = gold[form]["trace"]
        assert len(tr) == 2 * LEVELS * ITERS
        # each scale's first iteration recomputes every pixel of each colour
        dims = [(1920, 1080), (960, 540), (480, 270), (240, 135)][::-1]
        for k, (w, h) in enumerate(dims):
            even = (w * h + 1) // 2
            assert tr[2 * ITERS * k] == even and tr[2 * ITERS * k + 1] == w * h - even
    ref = np.load(os.path.join(HERE, "golden", gold["f64"]["disp_file"]))["disp"]
    assert ref.shape == (1080, 1920) and sha(ref.astype("<i4")) == gold["f64"]["disp_sha256"]


def _gpu():
    import torch

    import paper_1709_06509_gb300 as bps

    return torch, bps, torch.device("cuda:0")


@pytest.fixture(scope="module")
def built():
    import __graft_entry__

    __graft_entry__.build()


# variants forced on every scale: the defaults, and every candidate the autotuner offers at these
# sizes (lanes a pixel 16: no direction-parallel forms)
HD_VARIANTS = [-1, 0, 1, 2, 3, 8, 9, 10, 11, 64, 65, 66, 67, 130, 131, 138, 139, 194, 195, 256, 258, 386, 514, 522,
               578, 770, 771, 1024, 1026, 1034, 1154]


@pytest.mark.gpu
@pytest.mark.slow
def test_hd_u8_cost_volume_and_graph_solve_match_the_oracle(built, gold, pair):
    torch, bps, dev = _gpu()
    H, W = pair.left.shape
    with bps.Stereo(W, H, pair.D, LEVELS, bps.BPS_MSG_U8, device=dev) as st:
        L, R = torch.from_numpy(pair.left).to(dev), torch.from_numpy(pair.right).to(dev)
        # both NCC kernels: the tensor-core one (the default here) and the row kernel
        for kernel in (bps.BPS_NCC_TENSOR, bps.BPS_NCC_ROWS):
            st.set_ncc_kernel(kernel)
            assert st.ncc_kernel(WINDOW, TRUNC_DATA) == kernel
            st.build_cost_volume(L, R, WINDOW, TRUNC_DATA)
            cost = st.export_cost(0)
            assert sha(cost.cpu().numpy().astype("<i4")) == gold["int"]["cost_sha256"], kernel
            del cost
        st.set_ncc_kernel(bps.BPS_NCC_DEFAULT)
        disp = st.stereo(L, R, WINDOW, TRUNC_DATA, ITERS, LAM, TRUNC, graph=True)
        disp = st.stereo(L, R, WINDOW, TRUNC_DATA, ITERS, LAM, TRUNC, graph=True)  # a replay
        ei, _ = st.energy(disp, LAM, TRUNC)
        assert sha(disp.cpu().numpy().astype("<i4")) == gold["int"]["disp_sha256"]
        assert int(ei.item()) == gold["int"]["energy"]
        assert [int(v) for v in st.get_trace()] == gold["int"]["trace"]


@pytest.mark.gpu
@pytest.mark.slow
@pytest.mark.parametrize("variant", HD_VARIANTS)
def test_hd_u8_every_variant_matches_the_oracle(built, gold, pair, variant):
    torch, bps, dev = _gpu()
    H, W = pair.left.shape
    with bps.Stereo(W, H, pair.D, LEVELS, bps.BPS_MSG_U8, device=dev) as st:
        for lvl in range(LEVELS):
            st.set_variant(lvl, variant)
        L, R = torch.from_numpy(pair.left).to(dev), torch.from_numpy(pair.right).to(dev)
        disp = st.stereo(L, R, WINDOW, TRUNC_DATA, ITERS, LAM, TRUNC, graph=True)
        ei, _ = st.energy(disp, LAM, TRUNC)
        assert sha(disp.cpu().numpy().astype("<i4")) == gold["int"]["disp_sha256"]
        assert int(ei.item()) == gold["int"]["energy"]
        assert [int(v) for v in st.get_trace()] == gold["int"]["trace"]


@pytest.mark.gpu
@pytest.mark.slow
def test_hd_u8_autotuned_variants_match_the_oracle(built, gold, pair, tmp_path):
    # exactly what the benchmark times: the autotuner's choices, the pipeline as a graph
    torch, bps, dev = _gpu()
    from paper_1709_06509_gb300 import autotune

    H, W = pair.left.shape
    with bps.Stereo(W, H, pair.D, LEVELS, bps.BPS_MSG_U8, device=dev) as st:
        L, R = torch.from_numpy(pair.left).to(dev), torch.from_numpy(pair.right).to(dev)
        autotune.tune_ncc(st, L, R, WINDOW, TRUNC_DATA, reps=1)
        autotune.tune(st, L, R, WINDOW, TRUNC_DATA, ITERS, LAM, TRUNC, reps=1)
        disp = st.stereo(L, R, WINDOW, TRUNC_DATA, ITERS, LAM, TRUNC, graph=True)
        ei, _ = st.energy(disp, LAM, TRUNC)
        assert sha(disp.cpu().numpy().astype("<i4")) == gold["int"]["disp_sha256"], st.variants()
        assert int(ei.item()) == gold["int"]["energy"]
        assert [int(v) for v in st.get_trace()] == gold["int"]["trace"]


@pytest.mark.gpu
@pytest.mark.slow
def test_hd_int32_messages_match_the_oracle(built, gold, pair):
    torch, bps, dev = _gpu()
    H, W = pair.left.shape
    with bps.Stereo(W, H, pair.D, LEVELS, bps.BPS_MSG_INT32, device=dev) as st:
        L, R = torch.from_numpy(pair.left).to(dev), torch.from_numpy(pair.right).to(dev)
        st.build_cost_volume(L, R, WINDOW, TRUNC_DATA)
        cost = st.export_cost(0)
        assert sha(cost.cpu().numpy().astype("<i4")) == gold["int"]["cost_sha256"]
        del cost
        st.bp_solve(ITERS, LAM, TRUNC, skip=True)
        disp = st.wta_disparity()
        ei, _ = st.energy(disp, LAM, TRUNC)
        assert sha(disp.cpu().numpy().astype("<i4")) == gold["int"]["disp_sha256"]
        assert int(ei.item()) == gold["int"]["energy"]
        assert [int(v) for v in st.get_trace()] == gold["int"]["trace"]


@pytest.mark.gpu
@pytest.mark.slow
@pytest.mark.parametrize("tuned", [False, True], ids=["default", "autotuned"])
def test_hd_fp16_energy_gap_against_the_fp64_oracle(built, gold, pair, tuned):
    torch, bps, dev = _gpu()
    from paper_1709_06509_gb300 import autotune

    H, W = pair.left.shape
    ref_e = float.fromhex(gold["f64"]["energy_hex"])
    ref_d = np.load(os.path.join(HERE, "golden", gold["f64"]["disp_file"]))["disp"].astype(np.int32)
    with bps.Stereo(W, H, pair.D, LEVELS, bps.BPS_MSG_FP16, device=dev) as st:
        L, R = torch.from_numpy(pair.left).to(dev), torch.from_numpy(pair.right).to(dev)
        if tuned:
            autotune.tune(st, L, R, WINDOW, TRUNC_DATA, ITERS, LAM, TRUNC, reps=1)
        disp = st.stereo(L, R, WINDOW, TRUNC_DATA, ITERS, LAM, TRUNC, graph=True)
        _, ef = st.energy(disp, LAM, TRUNC)
        d = disp.cpu().numpy()
    # the GPU's FP64 energy scores its labels on its own fp32 float costs (each within 2e-4 of
    # the oracle's, |ncc error| < 1e-5 times trunc_data): far inside the 0.5% bar
    gap = (float(ef.item()) - ref_e) / ref_e
    assert abs(gap) <= 5e-3, gap
    assert float((d != ref_d).mean()) < 0.02
