"""Failure handling without a GPU fault.

- Resource failures are injected on the host (bps_test_fail_resources): every acquisition of
  bps_create / bps_batch_create in turn is made to fail; the call must return BPS_ERR_CUDA and
  give back every byte of device memory it had taken.
- The debug build of the library (-DBPS_DEBUG_BOUNDS) checks list entries, list appends, cost
  stores and read-out pixels against their buffers in the kernels; on a clean solve under every
  kind of sweep kernel its checks stay quiet (bps_get_error) and its results are the oracle's.
"""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1709_06509_gb300 as bps
from paper_1709_06509_gb300 import _build, synth


def test_failure_hook_is_exported_and_resettable():
    _build.build()
    lib = bps.lib()
    assert lib.bps_test_fail_resources(-1) == bps.BPS_OK
    assert lib.bps_test_fail_resources(3) == bps.BPS_OK
    assert lib.bps_test_fail_resources(-1) == bps.BPS_OK


@pytest.mark.gpu
def test_injected_resource_failures_release_everything():
    import torch

    _build.build()
    W, H, D, levels = 512, 384, 64, 3
    bps.bps_destroy(bps.bps_create(W, H, D, levels, bps.BPS_MSG_U8))  # load every module once
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failed = 0
    try:
        for n in range(4):  # the workspace, the capture stream, then none
            bps.bps_test_fail_resources(n)
            try:
                ctx = bps.bps_create(W, H, D, levels, bps.BPS_MSG_U8)
            except bps.BPSError as e:
                assert e.status == bps.BPS_ERR_CUDA
                failed += 1
            else:
                bps.bps_destroy(ctx)
            bps.bps_test_fail_resources(-1)
        assert failed == 2
        ctxs = [bps.bps_create(200, 100, 32, levels, bps.BPS_MSG_U8) for _ in range(2)]
        try:
            failed = 0
            for n in range(12):  # capture stream, 2 branch streams, 3 events, 3 device buffers
                bps.bps_test_fail_resources(n)
                try:
                    b = bps.bps_batch_create(ctxs)
                except bps.BPSError as e:
                    assert e.status == bps.BPS_ERR_CUDA
                    failed += 1
                else:
                    bps.bps_batch_destroy(b)
                bps.bps_test_fail_resources(-1)
            assert failed == 9
        finally:
            for c in ctxs:
                bps.bps_destroy(c)
    finally:
        bps.bps_test_fail_resources(-1)
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (8 << 20)  # nothing of the ~80 MB workspaces leaked


@pytest.mark.gpu
@pytest.mark.parametrize("variant", [0, 2, 8, 10, 42, 194, 770, 258])
def test_debug_build_checks_stay_quiet_and_results_match(variant):
    import torch

    _build.build(debug=True)
    dlib = bps.lib_debug()
    dev = torch.device("cuda:0")
    W, H, D, window, levels, iters, lam, trunc = 150, 110, 48, 5, 3, 6, 10, 2
    pair = synth.make_pair(880, W, H, D, 4, 2.0)
    ref = oracle.stereo_int(pair.left, pair.right, D, window, 20, levels, iters, lam, trunc)
    ctx = ctypes.c_void_p()
    assert dlib.bps_create(ctypes.byref(ctx), W, H, D, levels, bps.BPS_MSG_U8, None, 0) == bps.BPS_OK
    try:
        for lvl in range(levels):
            assert dlib.bps_set_sweep_variant(ctx, lvl, variant) == bps.BPS_OK
        L = torch.from_numpy(pair.left).to(dev)
        R = torch.from_numpy(pair.right).to(dev)
        disp = torch.empty((H, W), dtype=torch.int32, device=dev)
        stream = torch.cuda.current_stream().cuda_stream
        for _ in range(2):  # recorded as a graph, then replayed
            rc = dlib.bps_stereo(ctx, L.data_ptr(), R.data_ptr(), W, window, 20, iters, lam, trunc,
                                 bps.BPS_FLAG_FAST_SKIP | bps.BPS_FLAG_GRAPH, disp.data_ptr(), stream)
            assert rc == bps.BPS_OK
            torch.cuda.synchronize()
            assert dlib.bps_get_error(ctx) == bps.BPS_OK
            assert np.array_equal(disp.cpu().numpy(), ref["disp"])
    finally:
        dlib.bps_destroy(ctx)
