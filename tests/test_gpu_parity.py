"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer forms (BPS_MSG_INT32 and the narrow-storage BPS_MSG_U8) must match the oracle
bit for bit: data costs at every scale, finest messages, disparities, energy and the
fast-converging trace.  The NCC volume must agree with the FP64 oracle to 1e-5.  The fp16
form is judged against the FP64 oracle by its energy gap.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1709_06509_gb300 as bps
from paper_1709_06509_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
INT_FORMS = [bps.BPS_MSG_INT32, bps.BPS_MSG_U8]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def run_gpu(L, R, D, window, trunc_data, levels, iters, lam, trunc, msg_type, skip=True, init=None,
            persistent=False):
    H, W = L.shape
    with bps.Stereo(W, H, D, levels, msg_type, device=DEV) as st:
        ncc = st.build_cost_volume(to_dev(L), to_dev(R), window, trunc_data, want_ncc=True)
        costs = [st.export_cost(l).cpu().numpy() for l in range(levels)]
        st.bp_solve(iters, lam, trunc, skip=skip, init_msgs=None if init is None else to_dev(init),
                    persistent=persistent)
        assert st.get_error() == bps.BPS_OK
        disp = st.wta_disparity()
        ei, ef = st.energy(disp, lam, trunc)
        msg = st.export_messages(0)
        torch.cuda.synchronize()
        return {"ncc": ncc.cpu().numpy(), "cost": costs, "msg": msg.cpu().numpy(), "disp": disp.cpu().numpy(),
                "energy_i": int(ei.item()), "energy_f": float(ef.item()), "trace": st.get_trace()}


def assert_int_parity(g, L, R, D, window, trunc_data, levels, iters, lam, trunc, skip=True, init=None):
    ncc = oracle.ncc(L, R, D, window)
    assert np.abs(g["ncc"] - ncc).max() < 1e-5
    c0 = oracle.quantise(ncc, trunc_data)
    for lvl, want in enumerate(oracle.pyramid(c0, levels)):
        assert np.array_equal(g["cost"][lvl], want), f"cost level {lvl}"
    msg, trace = oracle.bp(c0, levels, iters, lam, trunc, skip=skip, init_coarsest=init)
    assert np.array_equal(g["msg"], msg), "finest messages"
    disp = oracle.wta(c0, msg)
    assert np.array_equal(g["disp"], disp), "disparity"
    e = oracle.energy(c0, disp, lam, trunc)
    assert g["energy_i"] == e and g["energy_f"] == float(e)
    if skip:
        assert np.array_equal(g["trace"], trace), "fast-converging trace"
    else:
        assert np.array_equal(g["trace"], trace)


# (W, H, D, window, levels, iters, lambda, trunc): tile-spanning, ragged, degenerate shapes
CASES = [
    (96, 72, 16, 5, 4, 10, 10, 2),    # the small published-shape workload
    (45, 19, 33, 7, 3, 4, 7, 3),      # D=33: three lanes of labels, one padded lane
    (130, 9, 64, 9, 4, 3, 10, 2),     # several NCC tiles wide, ragged tail
    (1, 7, 3, 3, 2, 3, 5, 1),         # W = 1
    (7, 1, 5, 1, 3, 4, 4, 5),         # H = 1, 1x1 window, trunc > D
    (1, 1, 4, 3, 4, 2, 10, 2),        # a single pixel
    (33, 13, 17, 31, 2, 2, 3, 4),     # the largest window
    (20, 15, 1, 3, 3, 3, 10, 2),      # one label
    (24, 16, 2, 5, 1, 5, 10, 2),      # two labels, flat BP
    (40, 30, 12, 5, 3, 0, 10, 2),     # zero iterations
    (40, 30, 12, 5, 3, 3, 0, 2),      # lambda = 0
    (40, 30, 12, 5, 3, 3, 10, 0),     # trunc = 0
    (24, 6, 256, 3, 2, 2, 10, 2),     # D = 256: 16 lanes per pixel
    (12, 5, 512, 3, 1, 1, 3, 7),      # D = 512: a full warp per pixel
    (37, 21, 20, 5, 3, 4, 21, 3),     # lambda * trunc = 63: four messages still add up bytewise
    (37, 21, 20, 5, 3, 4, 16, 4),     # lambda * trunc = 64: they do not
    (50, 23, 24, 5, 3, 4, 30, 3),     # lambda * trunc = 90
]


@pytest.mark.parametrize("persistent", [False, True], ids=["chained", "persistent"])
@pytest.mark.parametrize("msg_type", INT_FORMS)
@pytest.mark.parametrize("skip", [True, False])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c)))
def test_int_parity(case, skip, msg_type, persistent):
    W, H, D, window, levels, iters, lam, trunc = case
    if msg_type == bps.BPS_MSG_U8 and lam * trunc > 255:
        pytest.skip("outside the u8 range")
    pair = synth.make_pair(100 + W + H + D, W, H, D, 3, 2.0)
    g = run_gpu(pair.left, pair.right, D, window, 20, levels, iters, lam, trunc, msg_type, skip, persistent=persistent)
    assert_int_parity(g, pair.left, pair.right, D, window, 20, levels, iters, lam, trunc, skip)


def test_barrier_timeout_is_reported_and_the_context_survives():
    # the test hook makes every grid barrier wait for one block more than the grid has: the
    # bounded wait gives up after 2 ms, the kernel returns, and the host reads the status
    pair = synth.make_pair(31, 64, 48, 16, 3, 2.0)
    with bps.Stereo(64, 48, 16, 3, bps.BPS_MSG_U8, device=DEV) as st:
        st.build_cost_volume(to_dev(pair.left), to_dev(pair.right), 5, 20)
        st.bp_solve(4, 10, 2, persistent=True, test_timeout=True)
        torch.cuda.synchronize()
        assert st.get_error() == bps.BPS_ERR_TIMEOUT
        st.bp_solve(4, 10, 2, persistent=True)
        disp = st.wta_disparity()
        torch.cuda.synchronize()
        assert st.get_error() == bps.BPS_OK
        ref = oracle.stereo_int(pair.left, pair.right, 16, 5, 20, 3, 4, 10, 2)
        assert np.array_equal(disp.cpu().numpy(), ref["disp"])


def test_pitched_images_and_random_texture():
    rng = np.random.default_rng(3)
    H, W, D = 23, 37, 9
    big_l = rng.integers(0, 256, (H, W + 11)).astype(np.uint8)
    big_r = rng.integers(0, 256, (H, W + 11)).astype(np.uint8)
    L, R = big_l[:, :W], big_r[:, :W]
    with bps.Stereo(W, H, D, 2, bps.BPS_MSG_U8, device=DEV) as st:
        tl, tr = to_dev(big_l), to_dev(big_r)
        bps.bps_build_cost_volume(st.ctx, tl, tr, W + 11, 5, 20)
        got = st.export_cost(0).cpu().numpy()
    assert np.array_equal(got, oracle.quantise(oracle.ncc(L, R, D, 5), 20))


@pytest.mark.parametrize("msg_type", INT_FORMS)
@pytest.mark.parametrize("kernel", ["tensor", "rows"])
def test_quantiser_rounding_boundaries(kernel, msg_type):
    # windows whose NCC sits on a rounding boundary of the quantiser exercise the FP64 decision
    # (the tensor-core kernel's second pass, which also corrects the scale-1 sums)
    H, W, D = 16, 40, 8
    base = synth.texture(21, 1, W, H)
    L = base
    R = np.clip(base.astype(int) * 3 // 4 + (np.arange(W) % 3)[None, :] * 9, 0, 255).astype(np.uint8)
    for T in (1, 7, 20, 64, 127, 255):
        with bps.Stereo(W, H, D, 2, msg_type, device=DEV) as st:
            st.set_ncc_kernel(bps.BPS_NCC_TENSOR if kernel == "tensor" else bps.BPS_NCC_ROWS)
            st.build_cost_volume(to_dev(L), to_dev(R), 3, T)
            got = [st.export_cost(l).cpu().numpy() for l in range(2)]
        want = oracle.pyramid(oracle.quantise(oracle.ncc(L, R, D, 3), T), 2)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), T


def test_u8_form_equals_int32_form():
    pair = synth.make_pair(7, 70, 50, 24, 4, 3.0)
    a = run_gpu(pair.left, pair.right, 24, 7, 20, 4, 6, 10, 2, bps.BPS_MSG_INT32)
    b = run_gpu(pair.left, pair.right, 24, 7, 20, 4, 6, 10, 2, bps.BPS_MSG_U8)
    for k in ("msg", "disp", "energy_i", "trace"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("msg_type", INT_FORMS)
@pytest.mark.parametrize("init_hi", [21, 256], ids=["normalised", "up_to_255"])
def test_warm_start_matches_oracle(msg_type, init_hi):
    # start messages need not be normalised: up to 255 they still fit the u8 form's bytes, but four
    # of them no longer add up bytewise
    pair = synth.make_pair(9, 50, 40, 10, 3, 2.0)
    dims = oracle.level_dims(50, 40, 3)
    wc, hc = dims[-1]
    init = np.random.default_rng(1).integers(0, init_hi, (4, hc, wc, 10)).astype(np.int32)
    # slots of neighbours outside the image hold 0 (the layout both sides document)
    init[0, 0] = init[1, -1] = 0
    init[2, :, 0] = init[3, :, -1] = 0
    g = run_gpu(pair.left, pair.right, 10, 5, 20, 3, 4, 10, 2, msg_type, True, init)
    assert_int_parity(g, pair.left, pair.right, 10, 5, 20, 3, 4, 10, 2, True, init)


def test_fewer_levels_than_the_context():
    pair = synth.make_pair(12, 60, 44, 16, 3, 2.0)
    with bps.Stereo(60, 44, 16, 4, bps.BPS_MSG_U8, device=DEV) as st:
        st.build_cost_volume(to_dev(pair.left), to_dev(pair.right), 5, 20)
        st.bp_solve(5, 10, 2, levels=2)
        msg = st.export_messages(0).cpu().numpy()
    c0 = oracle.quantise(oracle.ncc(pair.left, pair.right, 16, 5), 20)
    assert np.array_equal(msg, oracle.bp(c0, 2, 5, 10, 2)[0])


def test_graph_replay_and_host_entry():
    pair = synth.make_pair(5, 96, 72, 16, 3, 2.0)
    L, R = to_dev(pair.left), to_dev(pair.right)
    with bps.Stereo(96, 72, 16, 4, bps.BPS_MSG_U8, device=DEV) as st:
        plain = st.stereo(L, R, 5, 20, 10, 10, 2, graph=False).clone()
        sweeps = st.stereo(L, R, 5, 20, 10, 10, 2, graph=True, persistent=True).clone()
        g1 = st.stereo(L, R, 5, 20, 10, 10, 2, graph=True).clone()
        g2 = st.stereo(L, R, 5, 20, 10, 10, 2, graph=True).clone()   # replay
        g3 = st.stereo(L, R, 5, 20, 6, 10, 2, graph=True).clone()    # new arguments: re-capture
        torch.cuda.synchronize()
        hl = torch.from_numpy(pair.left).pin_memory()
        hr = torch.from_numpy(pair.right).pin_memory()
        hd, he = st.stereo_host(hl, hr, 5, 20, 10, 10, 2)
    ref = oracle.stereo_int(pair.left, pair.right, 16, 5, 20, 4, 10, 10, 2)
    assert np.array_equal(plain.cpu().numpy(), ref["disp"])
    assert np.array_equal(sweeps.cpu().numpy(), ref["disp"])
    assert np.array_equal(g1.cpu().numpy(), ref["disp"]) and np.array_equal(g2.cpu().numpy(), ref["disp"])
    ref6 = oracle.stereo_int(pair.left, pair.right, 16, 5, 20, 4, 6, 10, 2)
    assert np.array_equal(g3.cpu().numpy(), ref6["disp"])
    assert np.array_equal(hd.numpy(), ref["disp"]) and he == ref["energy"]


def test_host_entry_graph_reads_current_buffers():
    # the recorded host graph copies from and to the same page-locked buffers every call: new
    # image contents give new results, a new kernel choice records it again, and pageable
    # buffers take the direct path
    p1, p2 = synth.make_pair(8, 96, 72, 16, 3, 2.0), synth.make_pair(9, 96, 72, 16, 3, 2.0)
    refs = [oracle.stereo_int(p.left, p.right, 16, 5, 20, 3, 6, 10, 2) for p in (p1, p2)]
    with bps.Stereo(96, 72, 16, 3, bps.BPS_MSG_U8, device=DEV) as st:
        hl, hr = torch.from_numpy(p1.left).pin_memory(), torch.from_numpy(p1.right).pin_memory()
        hd = torch.empty((72, 96), dtype=torch.int32).pin_memory()
        got = []
        d, e = st.stereo_host(hl, hr, 5, 20, 6, 10, 2, h_disp=hd)
        got.append((d.clone(), e))
        hl.copy_(torch.from_numpy(p2.left))
        hr.copy_(torch.from_numpy(p2.right))
        d, e = st.stereo_host(hl, hr, 5, 20, 6, 10, 2, h_disp=hd)
        got.append((d.clone(), e))
        st.set_variant(0, bps.BPS_VARIANT_GENERAL_DT | bps.BPS_VARIANT_EAGER)
        d, e = st.stereo_host(hl, hr, 5, 20, 6, 10, 2, h_disp=hd)
        got.append((d.clone(), e))
        d, e = st.stereo_host(torch.from_numpy(p1.left), torch.from_numpy(p1.right), 5, 20, 6, 10, 2)
        got.append((d, e))
    for (d, e), ref in zip(got, [refs[0], refs[1], refs[1], refs[0]]):
        assert np.array_equal(d.numpy(), ref["disp"]) and e == ref["energy"]


def test_batch_host_entry_graph_reads_current_buffers():
    shapes = [(70, 40, 16, 5), (45, 33, 64, 7)]
    sets = [[synth.make_pair(70 + 10 * r + k, W, H, D, 3, 2.0) for k, (W, H, D, _) in enumerate(shapes)]
            for r in range(2)]
    windows = [w for *_, w in shapes]
    sts = [bps.Stereo(W, H, D, 3, bps.BPS_MSG_U8, device=DEV) for W, H, D, _ in shapes]
    try:
        with bps.Batch(sts) as batch:
            hl = [torch.from_numpy(p.left).pin_memory() for p in sets[0]]
            hr = [torch.from_numpy(p.right).pin_memory() for p in sets[0]]
            for r in range(2):
                for k, p in enumerate(sets[r]):
                    hl[k].copy_(torch.from_numpy(p.left))
                    hr[k].copy_(torch.from_numpy(p.right))
                for rep in range(2):
                    hd, he = batch.stereo_host(hl, hr, windows, 20, 5, 10, 2)
                    for d, e, p, w in zip(hd, he.tolist(), sets[r], windows):
                        ref = oracle.stereo_int(p.left, p.right, p.D, w, 20, 3, 5, 10, 2)
                        assert np.array_equal(d.numpy(), ref["disp"]) and e == ref["energy"]
    finally:
        for st in sts:
            st.close()


def test_queued_host_calls_give_the_same_results():
    # BPS_FLAG_ASYNC: calls return once queued; after one synchronisation the host outputs of the
    # last call are those of a synchronous call
    shapes = [(70, 40, 16, 5), (45, 33, 64, 7)]
    pairs = [synth.make_pair(150 + k, W, H, D, 3, 2.0) for k, (W, H, D, _) in enumerate(shapes)]
    windows = [w for *_, w in shapes]
    sts = [bps.Stereo(W, H, D, 3, bps.BPS_MSG_U8, device=DEV) for W, H, D, _ in shapes]
    try:
        with bps.Batch(sts) as batch:
            hl = [torch.from_numpy(p.left).pin_memory() for p in pairs]
            hr = [torch.from_numpy(p.right).pin_memory() for p in pairs]
            hd = [torch.full((p.left.shape[0], p.left.shape[1]), -1, dtype=torch.int32).pin_memory() for p in pairs]
            for _ in range(3):
                _, he = batch.stereo_host(hl, hr, windows, 20, 5, 10, 2, h_disps=hd, sync=False)
            torch.cuda.current_stream().synchronize()
            for d, e, p, w in zip(hd, he.tolist(), pairs, windows):
                ref = oracle.stereo_int(p.left, p.right, p.D, w, 20, 3, 5, 10, 2)
                assert np.array_equal(d.numpy(), ref["disp"]) and e == ref["energy"]
    finally:
        for st in sts:
            st.close()


def test_contexts_of_different_shapes_coexist():
    # kernel attributes are process-wide: creating a second context must not break the first
    pairs = [synth.make_pair(40 + k, W, H, D, 3, 2.0) for k, (W, H, D) in enumerate([(80, 40, 16), (60, 30, 64)])]
    ctxs = [bps.Stereo(p.left.shape[1], p.left.shape[0], p.D, 3, bps.BPS_MSG_U8, device=DEV) for p in pairs]
    try:
        for rep in range(2):
            for p, st in zip(pairs, ctxs):
                d = st.stereo(to_dev(p.left), to_dev(p.right), 5, 20, 4, 10, 2, graph=bool(rep))
                ref = oracle.stereo_int(p.left, p.right, p.D, 5, 20, 3, 4, 10, 2)
                assert np.array_equal(d.cpu().numpy(), ref["disp"])
    finally:
        for st in ctxs:
            st.close()


@pytest.mark.parametrize("persistent", [False, True], ids=["chains", "persistent"])
@pytest.mark.parametrize("graph", [False, True])
def test_batch_of_mixed_pairs(persistent, graph):
    shapes = [(70, 40, 16, 5), (45, 33, 64, 7), (96, 20, 33, 3)]
    pairs = [synth.make_pair(60 + k, W, H, D, 3, 2.0) for k, (W, H, D, _) in enumerate(shapes)]
    windows = [w for *_, w in shapes]
    refs = [oracle.stereo_int(p.left, p.right, p.D, w, 20, 3, 5, 10, 2) for p, w in zip(pairs, windows)]
    sts = [bps.Stereo(p.left.shape[1], p.left.shape[0], p.D, 3, bps.BPS_MSG_U8, device=DEV) for p in pairs]
    try:
        with bps.Batch(sts) as batch:
            Ls = [to_dev(p.left) for p in pairs]
            Rs = [to_dev(p.right) for p in pairs]
            for rep in range(3):  # the graph is recorded once, then replayed
                outs = batch.stereo(Ls, Rs, windows, 20, 5, 10, 2, graph=graph, persistent=persistent)
                torch.cuda.synchronize()
                if persistent:
                    assert batch.get_error() == bps.BPS_OK
                for out, ref, st in zip(outs, refs, sts):
                    assert np.array_equal(out.cpu().numpy(), ref["disp"])
                    assert np.array_equal(st.get_trace(), ref["trace"])
            hl = [torch.from_numpy(p.left).pin_memory() for p in pairs]
            hr = [torch.from_numpy(p.right).pin_memory() for p in pairs]
            hd, he = batch.stereo_host(hl, hr, windows, 20, 5, 10, 2, graph=graph, persistent=persistent)
            for d, e, ref in zip(hd, he.tolist(), refs):
                assert np.array_equal(d.numpy(), ref["disp"]) and e == ref["energy"]
    finally:
        for st in sts:
            st.close()


def set_all_variants(st, variant):
    try:
        for lvl in range(st.levels):
            st.set_variant(lvl, variant)
    except bps.BPSError as e:
        if e.status == bps.BPS_ERR_UNSUPPORTED and variant & bps.BPS_VARIANT_CLUSTER:
            pytest.skip("a 16-CTA cluster of the sweep kernel does not fit on this GPU")
        raise
    assert st.variants() == [variant] * st.levels


# every variant the autotuner can pick, and more (tests/test_abi.py checks the tuner's candidates are here)
SWEEP_VARIANTS_TESTED = [0, 1, 2, 3, 4, 6, 8, 9, 10, 11, 12, 13, 16, 17, 18, 24, 25, 26, 27, 34, 35, 42, 43, 64, 65, 66,
                         67, 98, 99, 130, 131, 138, 139, 194, 195, 162, 256, 257, 258, 386, 514, 522, 578, 770, 771,
                         1024, 1026, 1027, 1034, 1154]


@pytest.mark.parametrize("variant", SWEEP_VARIANTS_TESTED)
@pytest.mark.parametrize("case", [(96, 72, 16, 5, 4, 6, 10, 2), (45, 19, 33, 7, 3, 4, 7, 3), (40, 30, 64, 5, 3, 5, 5, 1),
                                  (24, 6, 256, 3, 2, 3, 10, 2), (150, 110, 48, 5, 3, 5, 10, 2)],
                         ids=lambda c: "x".join(map(str, c)))
def test_every_sweep_variant_is_exact(case, variant):
    # every kernel variant (stencil / distance transform, dense / active lists, one cluster
    # launch per scale, eager loads, direction-parallel lanes) forced on every scale, even
    # tiny ones, must give the oracle's messages, trace and disparities
    W, H, D, window, levels, iters, lam, trunc = case
    pair = synth.make_pair(200 + W + D, W, H, D, 3, 2.0)
    with bps.Stereo(W, H, D, levels, bps.BPS_MSG_U8, device=DEV) as st:
        set_all_variants(st, variant)
        st.build_cost_volume(to_dev(pair.left), to_dev(pair.right), window, 20)
        st.bp_solve(iters, lam, trunc, skip=True)
        msg = st.export_messages(0).cpu().numpy()
        trace = st.get_trace()
        disp = st.wta_disparity().cpu().numpy()
    c0 = oracle.quantise(oracle.ncc(pair.left, pair.right, D, window), 20)
    ref_msg, ref_trace = oracle.bp(c0, levels, iters, lam, trunc, skip=True)
    assert np.array_equal(msg, ref_msg) and np.array_equal(trace, ref_trace)
    assert np.array_equal(disp, oracle.wta(c0, ref_msg))


_STAGED_REF = {}


@pytest.mark.parametrize("variant", [64, 66, 130, 194, 256, 258, 514, 770])
@pytest.mark.parametrize("case", [(160, 72, 256, 5, 1, 4, 10, 2), (520, 330, 16, 5, 3, 5, 10, 2), (400, 64, 100, 5, 2, 4, 7, 3)],
                         ids=lambda c: "x".join(map(str, c)))
def test_staged_variants_exact_where_every_cta_loops(case, variant):
    # sizes whose finest scale has more pixel blocks than the staged kernels have resident CTAs
    # (2 a SM), so CTAs stage their next block while they compute the current one (dense and
    # list launches): messages, trace and disparities must be the oracle's
    W, H, D, window, levels, iters, lam, trunc = case
    pair = synth.make_pair(900 + W + D, W, H, D, 4, 2.0)
    with bps.Stereo(W, H, D, levels, bps.BPS_MSG_U8, device=DEV) as st:
        set_all_variants(st, variant)
        st.build_cost_volume(to_dev(pair.left), to_dev(pair.right), window, 20)
        st.bp_solve(iters, lam, trunc, skip=True)
        msg = st.export_messages(0).cpu().numpy()
        trace = st.get_trace()
        disp = st.wta_disparity().cpu().numpy()
        assert st.get_error() == bps.BPS_OK  # no bounded wait gave up
    if case not in _STAGED_REF:
        c0 = oracle.quantise(oracle.ncc(pair.left, pair.right, D, window), 20)
        ref_msg, ref_trace = oracle.bp(c0, levels, iters, lam, trunc, skip=True)
        _STAGED_REF[case] = (ref_msg, ref_trace, oracle.wta(c0, ref_msg))
    ref_msg, ref_trace, ref_disp = _STAGED_REF[case]
    assert np.array_equal(msg, ref_msg) and np.array_equal(trace, ref_trace)
    assert np.array_equal(disp, ref_disp)


@pytest.mark.parametrize("variant", [4, 6, 8, 9, 12, 16, 24, 25, 64, 65, 256, 770])
def test_cluster_and_eager_variants_without_skip_and_in_a_graph(variant):
    # the cluster launch and the eager loads with every pixel recomputed (no skip), then
    # captured in the cached graph of the whole pipeline; the profile shares a cluster
    # launch's time out over its half-sweeps
    W, H, D, window, levels, iters, lam, trunc = 130, 70, 24, 5, 3, 4, 10, 2
    pair = synth.make_pair(61, W, H, D, 3, 2.0)
    with bps.Stereo(W, H, D, levels, bps.BPS_MSG_U8, device=DEV) as st:
        set_all_variants(st, variant)
        st.build_cost_volume(to_dev(pair.left), to_dev(pair.right), window, 20)
        st.bp_solve(iters, lam, trunc, skip=False, profile=True)
        msg = st.export_messages(0).cpu().numpy()
        times = st.read_launch_times()
        assert len(times) == levels * iters * 2 and np.all(times > 0)
        d = st.stereo(to_dev(pair.left), to_dev(pair.right), window, 20, iters, lam, trunc, graph=True)
        d2 = st.stereo(to_dev(pair.left), to_dev(pair.right), window, 20, iters, lam, trunc, graph=True)
    c0 = oracle.quantise(oracle.ncc(pair.left, pair.right, D, window), 20)
    ref_msg, _ = oracle.bp(c0, levels, iters, lam, trunc, skip=False)
    assert np.array_equal(msg, ref_msg)
    ref = oracle.stereo_int(pair.left, pair.right, D, window, 20, levels, iters, lam, trunc)
    assert np.array_equal(d.cpu().numpy(), ref["disp"]) and np.array_equal(d2.cpu().numpy(), ref["disp"])


@pytest.mark.parametrize("shape", [(2, 2), (2, 8), (4, 4), (8, 64), (16, 2), (0, 0)])
def test_ncc_shapes_are_exact(shape):
    pair = synth.make_pair(44, 75, 41, 16, 3, 2.0)
    with bps.Stereo(75, 41, 16, 3, bps.BPS_MSG_U8, device=DEV) as st:
        st.set_ncc_kernel(bps.BPS_NCC_ROWS)  # the CTA shapes of the row kernel
        st.set_ncc_shape(*shape)
        assert st.ncc_kernel(7, 20) == bps.BPS_NCC_ROWS
        st.build_cost_volume(to_dev(pair.left), to_dev(pair.right), 7, 20)
        costs = [st.export_cost(l).cpu().numpy() for l in range(2)]
    want = oracle.pyramid(oracle.quantise(oracle.ncc(pair.left, pair.right, 16, 7), 20), 2)
    assert np.array_equal(costs[0], want[0]) and np.array_equal(costs[1], want[1])


@pytest.mark.parametrize("case", [(70, 37, 256, 9, (1, 2)), (70, 37, 256, 9, (2, 4)), (70, 37, 256, 9, (1, 16)),
                                  (70, 37, 256, 9, (2, 64)), (53, 29, 100, 15, (4, 6)), (53, 29, 100, 15, (1, 2)),
                                  (40, 33, 48, 11, (8, 10)), (31, 9, 16, 3, (32, 2))],
                         ids=lambda c: "x".join(map(str, c[:4])) + f"-shape{c[4][0]}x{c[4][1]}")
def test_ncc_row_pairs_exact_for_every_shape(case):
    # rows are processed in pairs (odd heights end with a single row), one or two column groups
    # of 16 a thread's label; costs of scale 0 and the fused scale 1 must be the oracle's
    W, H, D, window, shape = case
    pair = synth.make_pair(45 + D, W, H, D, 3, 2.0)
    with bps.Stereo(W, H, D, 3, bps.BPS_MSG_U8, device=DEV) as st:
        st.set_ncc_shape(*shape)
        ncc = st.build_cost_volume(to_dev(pair.left), to_dev(pair.right), window, 20, want_ncc=True)
        costs = [st.export_cost(l).cpu().numpy() for l in range(3)]
    ref = oracle.ncc(pair.left, pair.right, D, window)
    assert np.abs(ncc.cpu().numpy() - ref).max() < 1e-5
    want = oracle.pyramid(oracle.quantise(ref, 20), 3)
    for lvl in range(3):
        assert np.array_equal(costs[lvl], want[lvl]), lvl


# (W, H, D, window, trunc_data, levels, rows per strip, form): tiles of 128 pixels with ragged
# tails and images narrower than a tile; label blocks of 128 with a partial last one; odd heights
# (a last row without a partner); strips of 2 rows up to the whole image; every window radius
TC_NCC_CASES = [
    (300, 37, 256, 9, 20, 3, 0, "u8"), (300, 37, 256, 9, 20, 3, 4, "u8"), (300, 38, 256, 9, 20, 3, 2, "u8"),
    (129, 21, 200, 9, 20, 3, 6, "u8"), (97, 31, 48, 7, 20, 3, 0, "u8"), (64, 17, 16, 5, 20, 2, 0, "u8"),
    (257, 19, 100, 3, 20, 3, 8, "u8"), (130, 9, 304, 1, 20, 2, 0, "u8"), (45, 33, 64, 9, 127, 1, 0, "u8"),
    (200, 25, 144, 9, 20, 3, 0, "int32"), (131, 23, 32, 9, 100, 2, 2, "int32"), (17, 5, 16, 3, 20, 3, 0, "int32"),
]


@pytest.mark.parametrize("case", TC_NCC_CASES, ids=lambda c: "x".join(map(str, c[:5])) + f"-L{c[5]}-r{c[6]}-{c[7]}")
def test_tensor_core_ncc_exact(case):
    # the tensor-core kernel: costs of scale 0 and its fused scale 1 (and the pyramid after it)
    # bit-identical to the oracle's quantised NCC and to the row kernel's
    W, H, D, window, td, levels, rows, form = case
    msg = bps.BPS_MSG_U8 if form == "u8" else bps.BPS_MSG_INT32
    pair = synth.make_pair(300 + W + D, W, H, D, 3, 2.0)
    L, R = to_dev(pair.left), to_dev(pair.right)
    with bps.Stereo(W, H, D, levels, msg, device=DEV) as st:
        st.set_ncc_kernel(bps.BPS_NCC_TENSOR, rows)
        assert st.ncc_kernel(window, td) == bps.BPS_NCC_TENSOR
        st.build_cost_volume(L, R, window, td)
        got = [st.export_cost(l).cpu().numpy() for l in range(levels)]
        assert st.get_error() == bps.BPS_OK
        st.set_ncc_kernel(bps.BPS_NCC_ROWS)
        st.build_cost_volume(L, R, window, td)
        rows_k = [st.export_cost(l).cpu().numpy() for l in range(levels)]
    want = oracle.pyramid(oracle.quantise(oracle.ncc(pair.left, pair.right, D, window), td), levels)
    for lvl in range(levels):
        assert np.array_equal(got[lvl], want[lvl]), lvl
        assert np.array_equal(rows_k[lvl], want[lvl]), lvl


def test_tensor_core_ncc_applies_where_documented():
    with bps.Stereo(64, 16, 64, 2, bps.BPS_MSG_U8, device=DEV) as st:
        assert st.ncc_kernel(9, 20) == bps.BPS_NCC_TENSOR  # the default
        assert st.ncc_kernel(11, 20) == bps.BPS_NCC_ROWS   # windows up to 9
        assert st.ncc_kernel(9, 128) == bps.BPS_NCC_ROWS   # trunc_data up to 127
        st.set_ncc_kernel(bps.BPS_NCC_ROWS)
        assert st.ncc_kernel(9, 20) == bps.BPS_NCC_ROWS
        with pytest.raises(bps.BPSError):
            st.set_ncc_kernel(3)
        with pytest.raises(bps.BPSError):
            st.set_ncc_kernel(bps.BPS_NCC_TENSOR, 3)  # odd rows per strip
    with bps.Stereo(64, 16, 64, 2, bps.BPS_MSG_FP16, device=DEV) as st:
        assert st.ncc_kernel(9, 20) == bps.BPS_NCC_ROWS   # the float form keeps the row kernel


def test_autotuner_picks_exact_variants(tmp_path):
    from paper_1709_06509_gb300 import autotune

    pair = synth.make_pair(33, 120, 90, 32, 3, 2.0)
    L, R = to_dev(pair.left), to_dev(pair.right)
    cache = str(tmp_path / "variants.json")
    with bps.Stereo(120, 90, 32, 3, bps.BPS_MSG_U8, device=DEV) as st:
        autotune.tune_ncc(st, L, R, 5, 20, reps=1, cache=cache)
        chosen = autotune.tune(st, L, R, 5, 20, 4, 10, 2, reps=1, cache=cache)
        assert st.variants() == chosen and all(v in autotune.CANDIDATES for v in chosen)
        d = st.stereo(L, R, 5, 20, 4, 10, 2, graph=True)
        again = autotune.tune(st, L, R, 5, 20, 4, 10, 2, cache=cache)  # served from the cache
        assert again == chosen
    ref = oracle.stereo_int(pair.left, pair.right, 32, 5, 20, 3, 4, 10, 2)
    assert np.array_equal(d.cpu().numpy(), ref["disp"])


def test_batch_autotuner_keeps_results_exact(tmp_path):
    from paper_1709_06509_gb300 import autotune

    shapes = [(80, 60, 16, 5), (64, 48, 48, 5)]
    pairs = [synth.make_pair(120 + k, W, H, D, 3, 2.0) for k, (W, H, D, _) in enumerate(shapes)]
    windows = [w for *_, w in shapes]
    sts = [bps.Stereo(W, H, D, 3, bps.BPS_MSG_U8, device=DEV) for W, H, D, _ in shapes]
    cache = str(tmp_path / "joint.json")
    try:
        with bps.Batch(sts) as batch:
            Ls = [to_dev(p.left) for p in pairs]
            Rs = [to_dev(p.right) for p in pairs]
            chosen = autotune.tune_batch(batch, sts, Ls, Rs, windows, 20, 4, 10, 2, reps=1, target_ms=2.0,
                                         cache=cache)
            assert [st.variants() for st in sts] == chosen
            outs = batch.stereo(Ls, Rs, windows, 20, 4, 10, 2)
            torch.cuda.synchronize()
            for out, p, w in zip(outs, pairs, windows):
                ref = oracle.stereo_int(p.left, p.right, p.D, w, 20, 3, 4, 10, 2)
                assert np.array_equal(out.cpu().numpy(), ref["disp"])
            for st in sts:
                for lvl in range(st.levels):
                    st.set_variant(lvl, 0)
            again = autotune.tune_batch(batch, sts, Ls, Rs, windows, 20, 4, 10, 2, cache=cache)  # from the cache
            assert again == chosen and [st.variants() for st in sts] == chosen
    finally:
        for st in sts:
            st.close()


def test_argument_errors_on_a_live_context():
    with bps.Stereo(16, 8, 4, 2, bps.BPS_MSG_U8, device=DEV) as st:
        with pytest.raises(bps.BPSError) as e:
            st.bp_solve(3, 10, 2)  # no cost volume yet
        assert e.value.status == bps.BPS_ERR_STATE
        L = torch.zeros((8, 16), dtype=torch.uint8, device=DEV)
        with pytest.raises(bps.BPSError) as e:
            st.build_cost_volume(L, L, 4, 20)  # even window
        assert e.value.status == bps.BPS_ERR_ARG
        with pytest.raises(bps.BPSError) as e:
            st.build_cost_volume(L, L, 3, 20000)  # coarse costs overflow int16 storage
        assert e.value.status == bps.BPS_ERR_UNSUPPORTED
        st.build_cost_volume(L, L, 3, 20)
        with pytest.raises(bps.BPSError) as e:
            st.bp_solve(3, 100, 3)  # lambda * trunc > 255 in the u8 form
        assert e.value.status == bps.BPS_ERR_UNSUPPORTED
        with pytest.raises(bps.BPSError) as e:
            st.bp_solve(3, 10, 2, levels=3)
        assert e.value.status == bps.BPS_ERR_ARG
        with pytest.raises(bps.BPSError) as e:
            st.bp_solve(bps.BPS_MAX_ITERS + 1, 10, 2)
        assert e.value.status == bps.BPS_ERR_ARG


# ------------------------------------------------------------------ full-size workloads

@pytest.fixture(scope="module")
def teddy():
    pair, window = synth.workload_pair("teddy_450x375_d64")
    return pair, window


@pytest.mark.slow
@pytest.mark.parametrize("name", ["tsukuba_384x288_d16", "teddy_450x375_d64"])
def test_full_size_bit_exact(name):
    """The benchmark's workloads, in the benchmark's launch configuration (u8 form, skip on,
    CUDA graph through bps_stereo), bit-exact against the oracle."""
    pair, window = synth.workload_pair(name)
    H, W = pair.left.shape
    D = pair.D
    ref = oracle.stereo_int(pair.left, pair.right, D, window, 20, 4, 10, 10, 2)
    with bps.Stereo(W, H, D, 4, bps.BPS_MSG_U8, device=DEV) as st:
        L, R = to_dev(pair.left), to_dev(pair.right)
        disp = st.stereo(L, R, window, 20, 10, 10, 2, graph=True)
        disp = st.stereo(L, R, window, 20, 10, 10, 2, graph=True)  # a replay
        ei, _ = st.energy(disp, 10, 2)
        msg = st.export_messages(0)
        torch.cuda.synchronize()
        assert np.array_equal(msg.cpu().numpy(), ref["msg"])
        assert np.array_equal(disp.cpu().numpy(), ref["disp"])
        assert int(ei.item()) == ref["energy"]
        assert np.array_equal(st.get_trace(), ref["trace"])


@pytest.mark.slow
@pytest.mark.parametrize("variant", [42, 34, 35, 98])
def test_full_size_direction_parallel_lists_switch_lane_mapping(teddy, variant):
    # the direction-parallel list launches pick their lane mapping from the list length: one
    # group per (pixel, direction) on short lists, one group per pixel on long ones.  The long
    # lists occur only at full size: 450x375 D64, the variant forced on every scale
    pair, window = teddy
    H, W = pair.left.shape
    ref = oracle.stereo_int(pair.left, pair.right, pair.D, window, 20, 4, 10, 10, 2)
    with bps.Stereo(W, H, pair.D, 4, bps.BPS_MSG_U8, device=DEV) as st:
        set_all_variants(st, variant)
        disp = st.stereo(to_dev(pair.left), to_dev(pair.right), window, 20, 10, 10, 2, graph=True)
        msg = st.export_messages(0)
        torch.cuda.synchronize()
        assert np.array_equal(msg.cpu().numpy(), ref["msg"])
        assert np.array_equal(disp.cpu().numpy(), ref["disp"])
        assert np.array_equal(st.get_trace(), ref["trace"])


@pytest.mark.slow
def test_full_size_pairs_bit_exact_under_the_joint_tuner(tmp_path):
    """The two 384x288 D16 / 450x375 D64 pairs as the benchmark runs them: per-pair tuning, then
    the joint batch tuner, one batch graph; bit-exact against the oracle."""
    from paper_1709_06509_gb300 import autotune

    pairs = [synth.workload_pair(n) for n in ("tsukuba_384x288_d16", "teddy_450x375_d64")]
    sts = [bps.Stereo(p.left.shape[1], p.left.shape[0], p.D, 4, bps.BPS_MSG_U8, device=DEV) for p, _ in pairs]
    try:
        Ls = [to_dev(p.left) for p, _ in pairs]
        Rs = [to_dev(p.right) for p, _ in pairs]
        ws = [w for _, w in pairs]
        for st, L, R, w in zip(sts, Ls, Rs, ws):
            autotune.tune_ncc(st, L, R, w, 20, reps=1)
            autotune.tune(st, L, R, w, 20, 10, 10, 2, reps=1)
        with bps.Batch(sts) as batch:
            autotune.tune_batch(batch, sts, Ls, Rs, ws, 20, 10, 10, 2, reps=1)
            outs = [torch.empty(p.left.shape, dtype=torch.int32, device=DEV) for p, _ in pairs]
            batch.stereo(Ls, Rs, ws, 20, 10, 10, 2, graph=True, outs=outs)
            batch.stereo(Ls, Rs, ws, 20, 10, 10, 2, graph=True, outs=outs)
            torch.cuda.synchronize()
            for (pair, window), st, o in zip(pairs, sts, outs):
                ref = oracle.stereo_int(pair.left, pair.right, pair.D, window, 20, 4, 10, 10, 2)
                assert np.array_equal(o.cpu().numpy(), ref["disp"]), st.variants()
                assert np.array_equal(st.get_trace(), ref["trace"])
                assert np.array_equal(st.export_messages(0).cpu().numpy(), ref["msg"])
    finally:
        for st in sts:
            st.close()


@pytest.mark.parametrize("variant", [0, 2, 194, 770])
@pytest.mark.parametrize("schedule", [[5, 5, 5], [3, 0, 4], [0, 2, 6], [6, 1, 0], [2, 3, 1]],
                         ids=lambda s: "-".join(map(str, s)))
def test_iteration_schedule_matches_the_oracle(schedule, variant):
    # bps_bp_solve_schedule: its own iteration count at every scale (0 = the finest), zero counts
    # included, plain and recorded as a graph, cold and warm-started
    W, H, D, window, lam, trunc = 150, 110, 48, 5, 10, 2
    pair = synth.make_pair(990 + sum(schedule), W, H, D, 4, 2.0)
    c0 = oracle.quantise(oracle.ncc(pair.left, pair.right, D, window), 20)
    rng = np.random.default_rng(3)
    wc, hc = oracle.level_dims(W, H, 3)[-1]
    init = rng.integers(0, lam * trunc + 1, (4, hc, wc, D)).astype(np.int32)
    # slots of neighbours outside the image hold 0 (no sender ever writes them)
    init[0, 0], init[1, -1], init[2, :, 0], init[3, :, -1] = 0, 0, 0, 0
    with bps.Stereo(W, H, D, 3, bps.BPS_MSG_U8, device=DEV) as st:
        set_all_variants(st, variant)
        st.build_cost_volume(to_dev(pair.left), to_dev(pair.right), window, 20)
        for start in (None, init):
            ref_msg, ref_trace = oracle.bp_schedule(c0, schedule, lam, trunc, init_coarsest=start)
            for graph in (False, True, True):
                st.bp_solve_schedule(schedule, lam, trunc, init_msgs=None if start is None else to_dev(start),
                                     graph=graph)
                assert np.array_equal(st.export_messages(0).cpu().numpy(), ref_msg)
                assert np.array_equal(st.get_trace(), ref_trace)
                assert np.array_equal(st.wta_disparity().cpu().numpy(), oracle.wta(c0, ref_msg))


@pytest.mark.gpu
def test_bp_solve_graph_replays_match_eager_solves():
    # bps_bp_solve recorded as a graph and replayed: same messages, trace and labels as the eager
    # solve; an eager solve with other arguments in between, then a replay, restores the trace length
    pair = synth.make_pair(77, 96, 72, 16, 3, 2.0)
    with bps.Stereo(96, 72, 16, 4, bps.BPS_MSG_U8, device=DEV) as st:
        st.build_cost_volume(to_dev(pair.left), to_dev(pair.right), 5, 20)
        st.bp_solve(6, 10, 2, skip=True)
        m0, t0, d0 = st.export_messages(0).clone(), st.get_trace(), st.wta_disparity().clone()
        for _ in range(3):
            st.bp_solve(6, 10, 2, skip=True, graph=True)
            assert torch.equal(st.export_messages(0), m0) and np.array_equal(st.get_trace(), t0)
            assert torch.equal(st.wta_disparity(), d0)
        st.bp_solve(2, 10, 2, skip=True)
        assert len(st.get_trace()) == 4 * 2 * 2
        st.bp_solve(6, 10, 2, skip=True, graph=True)
        assert np.array_equal(st.get_trace(), t0) and torch.equal(st.wta_disparity(), d0)
        st.set_variant(0, 2)  # a kernel choice changes: the graph is recorded again
        st.bp_solve(6, 10, 2, skip=True, graph=True)
        assert torch.equal(st.export_messages(0), m0) and np.array_equal(st.get_trace(), t0)


@pytest.mark.slow
def test_hd_256_properties():
    """1920x1080, D=256, 9x9 window: too large for the oracle, so sampled NCC entries are
    checked one by one and the BP result through properties that hold at any size."""
    pair, window = synth.workload_pair("hd_1920x1080_d256")
    H, W = pair.left.shape
    D, r, lam, T = 256, window // 2, 10, 2
    with bps.Stereo(W, H, D, 4, bps.BPS_MSG_U8, device=DEV) as st:
        L, R = to_dev(pair.left), to_dev(pair.right)
        st.build_cost_volume(L, R, window, 20)
        cost = st.export_cost(0)
        rng = np.random.default_rng(0)
        ys = rng.integers(r, H - r, 40)
        xs = rng.integers(D - 1 + r, W - r, 40)
        for y, x in zip(ys, xs):
            # a crop with no clamped taps gives the same window sums as the full image
            cl = pair.left[y - r: y + r + 1, x - D + 1 - r: x + r + 1]
            cr = pair.right[y - r: y + r + 1, x - D + 1 - r: x + r + 1]
            want = oracle.quantise(oracle.ncc(cl, cr, D, window), 20)[r, D - 1 + r]
            assert np.array_equal(cost[y, x].cpu().numpy(), want)
        st.bp_solve(10, lam, T, skip=True)
        d_skip = st.wta_disparity().clone()
        msg_skip = st.export_messages(0)
        trace = st.get_trace()
        st.bp_solve(10, lam, T, skip=False)
        d_full = st.wta_disparity()
        msg_full = st.export_messages(0)
        assert torch.equal(msg_skip, msg_full) and torch.equal(d_skip, d_full)  # the skip is exact
        interior = msg_full[:, 1:-1, 1:-1]
        assert int(interior.min()) == 0 and int(msg_full.max()) <= lam * T
        assert int(interior.amin(dim=3).max()) == 0  # every message is min-normalised
        ei, _ = st.energy(d_full, lam, T)
        c = cost.to(torch.int64)
        d = d_full.to(torch.int64)
        e = c.gather(2, d[..., None]).sum()
        e += lam * ((d[:, 1:] - d[:, :-1]).abs().clamp(max=T).sum() + (d[1:] - d[:-1]).abs().clamp(max=T).sum())
        assert int(ei.item()) == int(e.item())
        n0 = W * H
        assert trace[-20:].sum() < 10 * n0  # the skip removes work at the finest scale
        bad = ((d_full.cpu().numpy() - pair.disparity).__abs__() > 1) & ~pair.occluded
        assert bad.mean() < 0.1


# ------------------------------------------------------------------ fp16 messages vs the FP64 oracle

@pytest.mark.slow
@pytest.mark.parametrize("name", ["tsukuba_384x288_d16", "teddy_450x375_d64"])
def test_fp16_energy_gap(name):
    pair, window = synth.workload_pair(name)
    H, W = pair.left.shape
    D = pair.D
    ref = oracle.stereo_f64(pair.left, pair.right, D, window, 20, 4, 10, 10.0, 2)
    with bps.Stereo(W, H, D, 4, bps.BPS_MSG_FP16, device=DEV) as st:
        ncc = st.build_cost_volume(to_dev(pair.left), to_dev(pair.right), window, 20, want_ncc=True)
        st.bp_solve(10, 10, 2, skip=True)
        disp = st.wta_disparity()
        _, ef = st.energy(disp, 10, 2)
        d = disp.cpu().numpy()
        cf = st.export_cost(0).cpu().numpy()
    assert np.abs(cf - ref["cost"]).max() < 1e-4
    e_gpu = oracle.energy(ref["cost"], d, 10.0, 2)  # the GPU labels, scored by the FP64 oracle
    gap = (e_gpu - ref["energy"]) / ref["energy"]
    assert gap <= 0.005, gap
    assert abs(float(ef.item()) - e_gpu) / e_gpu < 1e-5  # the GPU's own FP64 energy reduction
    assert (d != ref["disp"]).mean() < 0.02


@pytest.mark.parametrize("persistent", [False, True], ids=["chains", "persistent"])
@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("trunc", [1, 2])
def test_fp16_batch_matches_single_pairs_and_the_fp64_oracle(persistent, graph, trunc):
    """fp16 messages in a batch of mixed pairs, as concurrent chains or one persistent launch (packed
    half2 body, active lists after each scale's first iteration), plain or recorded as a graph:
    every pair's messages, trace and labels equal its own chained solve's bit for bit, and its
    energy is within 0.5% of the FP64 oracle's, under 2% of labels different."""
    shapes = [(70, 40, 16, 5), (45, 33, 64, 7), (96, 20, 33, 3), (130, 60, 32, 5)]
    pairs = [synth.make_pair(610 + k, W, H, D, 3, 2.0) for k, (W, H, D, _) in enumerate(shapes)]
    windows = [w for *_, w in shapes]
    singles = []
    for p, w in zip(pairs, windows):
        with bps.Stereo(p.left.shape[1], p.left.shape[0], p.D, 3, bps.BPS_MSG_FP16, device=DEV) as st:
            st.build_cost_volume(to_dev(p.left), to_dev(p.right), w, 20)
            st.bp_solve(5, 10, trunc, skip=True)
            d = st.wta_disparity().cpu().numpy()
            m = st.export_messages(0).cpu().numpy()
            tr = st.get_trace()
            if persistent:  # a single pair's persistent solve gives the same
                st.bp_solve(5, 10, trunc, skip=True, persistent=True)
                assert st.get_error() == bps.BPS_OK
                assert np.array_equal(st.wta_disparity().cpu().numpy(), d)
                assert np.array_equal(st.export_messages(0).cpu().numpy(), m)
                assert np.array_equal(st.get_trace(), tr)
        singles.append((d, m, tr))
    sts = [bps.Stereo(p.left.shape[1], p.left.shape[0], p.D, 3, bps.BPS_MSG_FP16, device=DEV) for p in pairs]
    try:
        with bps.Batch(sts) as batch:
            Ls = [to_dev(p.left) for p in pairs]
            Rs = [to_dev(p.right) for p in pairs]
            for rep in range(2):
                outs = batch.stereo(Ls, Rs, windows, 20, 5, 10, trunc, graph=graph, persistent=persistent)
                torch.cuda.synchronize()
                if persistent:
                    assert batch.get_error() == bps.BPS_OK
                for out, st, (d, m, tr) in zip(outs, sts, singles):
                    assert np.array_equal(out.cpu().numpy(), d)
                    assert np.array_equal(st.get_trace(), tr)
                    assert np.array_equal(st.export_messages(0).cpu().numpy(), m)
    finally:
        for st in sts:
            st.close()
    for p, w, (d, _, _) in zip(pairs, windows, singles):
        ref = oracle.stereo_f64(p.left, p.right, p.D, w, 20, 3, 5, 10.0, trunc)
        e = oracle.energy(ref["cost"], d, 10.0, trunc)
        assert abs(e - ref["energy"]) <= 0.005 * ref["energy"], (e, ref["energy"])
        assert (d != ref["disp"]).mean() < 0.02


@pytest.mark.slow
def test_fp16_c3_style_batch_persistent_equals_chains():
    # mixed sizes and label counts of the 64-pair configuration (a few of its pairs): the single
    # persistent launch reproduces the concurrent chains' labels and traces bit for bit
    specs = synth.batch_specs(6)
    pairs = [synth.make_pair(seed, W, H, D, 8, 3.0) for seed, W, H, D in specs]
    sts = [bps.Stereo(p.left.shape[1], p.left.shape[0], p.D, 4, bps.BPS_MSG_FP16, device=DEV) for p in pairs]
    try:
        with bps.Batch(sts) as batch:
            Ls = [to_dev(p.left) for p in pairs]
            Rs = [to_dev(p.right) for p in pairs]
            ws = [7] * len(pairs)
            chains = [o.clone() for o in batch.stereo(Ls, Rs, ws, 20, 10, 10, 2, graph=True)]
            tr_chains = [st.get_trace() for st in sts]
            outs = batch.stereo(Ls, Rs, ws, 20, 10, 10, 2, graph=True, persistent=True)
            torch.cuda.synchronize()
            assert batch.get_error() == bps.BPS_OK
            for a, b, st, tr in zip(chains, outs, sts, tr_chains):
                assert torch.equal(a, b) and np.array_equal(st.get_trace(), tr)
    finally:
        for st in sts:
            st.close()


@pytest.mark.parametrize("variant", [0, 2, 8, 16, 18, 24, 64, 66, 130, 194, 258, 770])
@pytest.mark.parametrize("eps,freeze", [(1, False), (3, False), (0, True), (2, True)])
@pytest.mark.parametrize("case", [(96, 72, 16, 5, 4, 6, 10, 2), (60, 44, 40, 5, 3, 5, 8, 3)],
                         ids=lambda c: "x".join(map(str, c)))
def test_approximate_skip_rules_match_the_oracle(case, eps, freeze, variant):
    # the approximate skip rules (eps threshold, permanent freeze) are deterministic: every
    # kernel variant must reproduce the oracle's messages, trace and disparities bit for bit
    W, H, D, window, levels, iters, lam, trunc = case
    pair = synth.make_pair(300 + W + D, W, H, D, 4, 2.0)
    with bps.Stereo(W, H, D, levels, bps.BPS_MSG_U8, device=DEV) as st:
        st.set_skip_rule(eps, freeze)
        set_all_variants(st, variant)
        st.build_cost_volume(to_dev(pair.left), to_dev(pair.right), window, 20)
        st.bp_solve(iters, lam, trunc, skip=True)
        msg = st.export_messages(0).cpu().numpy()
        trace = st.get_trace()
        disp = st.wta_disparity().cpu().numpy()
    c0 = oracle.quantise(oracle.ncc(pair.left, pair.right, D, window), 20)
    ref_msg, ref_trace = oracle.bp(c0, levels, iters, lam, trunc, skip=True, eps=eps, freeze=freeze)
    assert np.array_equal(msg, ref_msg) and np.array_equal(trace, ref_trace)
    assert np.array_equal(disp, oracle.wta(c0, ref_msg))


@pytest.mark.parametrize("persistent", [False, True], ids=["chains", "persistent"])
def test_skip_rule_in_batched_launches(persistent):
    shapes = [(70, 40, 16, 5), (45, 33, 64, 7)]
    pairs = [synth.make_pair(90 + k, W, H, D, 3, 2.0) for k, (W, H, D, _) in enumerate(shapes)]
    windows = [w for *_, w in shapes]
    sts = [bps.Stereo(W, H, D, 3, bps.BPS_MSG_U8, device=DEV) for W, H, D, _ in shapes]
    try:
        with bps.Batch(sts) as batch:
            for st in sts:
                st.set_skip_rule(2, True)  # after the batch exists: its launches pick the rule up
            outs = batch.stereo([to_dev(p.left) for p in pairs], [to_dev(p.right) for p in pairs], windows, 20, 5,
                                10, 2, persistent=persistent)
            torch.cuda.synchronize()
            for out, p, w, st in zip(outs, pairs, windows, sts):
                c0 = oracle.quantise(oracle.ncc(p.left, p.right, p.D, w), 20)
                ref_msg, ref_trace = oracle.bp(c0, 3, 5, 10, 2, skip=True, eps=2, freeze=True)
                assert np.array_equal(out.cpu().numpy(), oracle.wta(c0, ref_msg))
                assert np.array_equal(st.get_trace(), ref_trace)
    finally:
        for st in sts:
            st.close()


def test_skip_rule_arguments():
    with bps.Stereo(16, 8, 4, 2, bps.BPS_MSG_INT32, device=DEV) as st:
        st.set_skip_rule(0, False)  # the exact rule: every form
        with pytest.raises(bps.BPSError) as e:
            st.set_skip_rule(1, False)
        assert e.value.status == bps.BPS_ERR_UNSUPPORTED
    with bps.Stereo(16, 8, 4, 2, bps.BPS_MSG_U8, device=DEV) as st:
        for eps, freeze in ((256, False), (-1, False)):
            with pytest.raises(bps.BPSError) as e:
                st.set_skip_rule(eps, freeze)
            assert e.value.status == bps.BPS_ERR_ARG
        with pytest.raises(bps.BPSError) as e:
            bps.bps_set_skip_rule(st.ctx, 0, 2)
        assert e.value.status == bps.BPS_ERR_ARG


def test_approximate_skip_energy_gap_on_a_full_size_pair():
    # the approximate rules are judged by the energy of their read-out against the exact
    # solve's, on a 450x375 D64 pair, with fewer pixels recomputed: the eps thresholds stay
    # within the 0.5% bar; the permanent freeze does not (0.54% measured) and is held to 2%
    pair, window = synth.workload_pair("teddy_450x375_d64")
    H, W = pair.left.shape
    L, R = to_dev(pair.left), to_dev(pair.right)
    with bps.Stereo(W, H, 64, 4, bps.BPS_MSG_U8, device=DEV) as st:
        st.build_cost_volume(L, R, window, 20)
        st.bp_solve(10, 10, 2, skip=True)
        e0 = int(st.energy(st.wta_disparity(), 10, 2)[0].item())
        w0 = int(st.get_trace().sum())
        for eps, freeze in ((1, False), (2, False), (0, True), (1, True)):
            st.set_skip_rule(eps, freeze)
            st.bp_solve(10, 10, 2, skip=True)
            e = int(st.energy(st.wta_disparity(), 10, 2)[0].item())
            assert abs(e - e0) <= (0.02 if freeze else 0.005) * e0, (eps, freeze, e, e0)
            assert int(st.get_trace().sum()) < w0


# ------------------------------------------------------------------ sparse candidates

@pytest.mark.parametrize("skip", [True, False])
@pytest.mark.parametrize("case", [(96, 72, 16, 5, 4, 6, 10, 2, 4), (96, 72, 16, 5, 3, 5, 10, 2, 16),
                                  (45, 19, 33, 7, 3, 4, 7, 3, 6), (60, 44, 64, 5, 2, 5, 8, 2, 8),
                                  (40, 30, 64, 5, 1, 6, 10, 2, 32), (37, 21, 20, 5, 3, 4, 10, 2, 1)],
                         ids=lambda c: "x".join(map(str, c)))
def test_sparse_candidates_match_the_oracle(case, skip):
    W, H, D, window, levels, iters, lam, trunc, K = case
    pair = synth.make_pair(400 + W + D + K, W, H, D, 4, 2.0)
    with bps.Stereo(W, H, D, levels, bps.BPS_MSG_U8, device=DEV) as st:
        st.set_candidates(K)
        st.build_cost_volume(to_dev(pair.left), to_dev(pair.right), window, 20)
        st.bp_solve(iters, lam, trunc, skip=skip)
        cand, msg = (t.cpu().numpy() for t in st.export_sparse())
        trace = st.get_trace()
        disp = st.wta_disparity().cpu().numpy()
        with pytest.raises(bps.BPSError) as e:
            st.export_messages(0)  # the finest scale holds sparse messages
        assert e.value.status == bps.BPS_ERR_STATE
    c0 = oracle.quantise(oracle.ncc(pair.left, pair.right, D, window), 20)
    rc, rm, rt = oracle.bp_sparse(c0, levels, iters, lam, trunc, K, skip=skip)
    assert np.array_equal(cand, rc)
    assert np.array_equal(msg, rm) and np.array_equal(trace, rt)
    assert np.array_equal(disp, oracle.wta_sparse(c0, rc, rm))


def test_sparse_in_a_graph_and_a_batch_and_back_to_dense():
    shapes = [(70, 40, 16, 5, 6), (45, 33, 64, 7, 12)]
    pairs = [synth.make_pair(130 + k, W, H, D, 3, 2.0) for k, (W, H, D, _, _) in enumerate(shapes)]
    windows = [s[3] for s in shapes]
    sts = [bps.Stereo(W, H, D, 3, bps.BPS_MSG_U8, device=DEV) for W, H, D, _, _ in shapes]
    try:
        for st, (_, _, _, _, K) in zip(sts, shapes):
            st.set_candidates(K)
        refs = []
        for p, w, (_, _, D, _, K) in zip(pairs, windows, shapes):
            c0 = oracle.quantise(oracle.ncc(p.left, p.right, D, w), 20)
            rc, rm, _ = oracle.bp_sparse(c0, 3, 5, 10, 2, K)
            refs.append(oracle.wta_sparse(c0, rc, rm))
        for rep in range(2):  # recorded, then replayed
            for st, p, w, ref in zip(sts, pairs, windows, refs):
                d = st.stereo(to_dev(p.left), to_dev(p.right), w, 20, 5, 10, 2, graph=True)
                assert np.array_equal(d.cpu().numpy(), ref)
        with bps.Batch(sts) as batch:
            outs = batch.stereo([to_dev(p.left) for p in pairs], [to_dev(p.right) for p in pairs], windows, 20, 5,
                                10, 2)
            torch.cuda.synchronize()
            for out, ref in zip(outs, refs):
                assert np.array_equal(out.cpu().numpy(), ref)
            with pytest.raises(bps.BPSError) as e:
                batch.stereo([to_dev(p.left) for p in pairs], [to_dev(p.right) for p in pairs], windows, 20, 5,
                             10, 2, persistent=True)
            assert e.value.status == bps.BPS_ERR_UNSUPPORTED
        # back to the dense solve
        st, p, w = sts[0], pairs[0], windows[0]
        st.set_candidates(0)
        d = st.stereo(to_dev(p.left), to_dev(p.right), w, 20, 5, 10, 2, graph=True)
        ref = oracle.stereo_int(p.left, p.right, 16, w, 20, 3, 5, 10, 2)
        assert np.array_equal(d.cpu().numpy(), ref["disp"])
    finally:
        for st in sts:
            st.close()


def test_sparse_arguments():
    with bps.Stereo(16, 8, 8, 2, bps.BPS_MSG_INT32, device=DEV) as st:
        with pytest.raises(bps.BPSError) as e:
            st.set_candidates(4)
        assert e.value.status == bps.BPS_ERR_UNSUPPORTED
    with bps.Stereo(16, 8, 40, 2, bps.BPS_MSG_U8, device=DEV) as st:
        for K in (-1, 33, 41):
            with pytest.raises(bps.BPSError) as e:
                st.set_candidates(K)
            assert e.value.status == bps.BPS_ERR_ARG
        st.set_skip_rule(1, False)
        with pytest.raises(bps.BPSError) as e:
            st.set_candidates(4)
        assert e.value.status == bps.BPS_ERR_UNSUPPORTED
        st.set_skip_rule(0, False)
        st.set_candidates(4)
        with pytest.raises(bps.BPSError) as e:
            st.set_skip_rule(0, True)
        assert e.value.status == bps.BPS_ERR_UNSUPPORTED


@pytest.mark.parametrize("skip", [True, False])
@pytest.mark.parametrize("case", [(96, 72, 16, 5, 4, 8, 10, 2), (60, 44, 33, 5, 3, 6, 10, 1), (64, 48, 64, 7, 3, 6, 8, 2)],
                         ids=lambda c: "x".join(map(str, c)))
def test_fp16_packed_kernel_agrees_with_the_generic_one_and_the_oracle(case, skip):
    # the packed half2 half-sweep (default for T <= 2) against the generic float-arithmetic one
    # (the GENERAL_DT variant) and the FP64 oracle of the float form: the same labels up to
    # rounding, energies within 0.5%
    W, H, D, window, levels, iters, lam, trunc = case
    pair = synth.make_pair(500 + W + D, W, H, D, 4, 2.0)
    res = {}
    for name, variant, eager in (("packed", 0, False), ("packed_eager", bps.BPS_VARIANT_EAGER, True),
                                 ("generic", bps.BPS_VARIANT_GENERAL_DT, False)):
        with bps.Stereo(W, H, D, levels, bps.BPS_MSG_FP16, device=DEV) as st:
            for lvl in range(levels):
                st.set_variant(lvl, variant)
            st.build_cost_volume(to_dev(pair.left), to_dev(pair.right), window, 20)
            st.bp_solve(iters, lam, trunc, skip=skip)
            d = st.wta_disparity().cpu().numpy()
        res[name] = d
    ref = oracle.stereo_f64(pair.left, pair.right, D, window, 20, levels, iters, float(lam), trunc)
    for name, d in res.items():
        e = oracle.energy(ref["cost"], d, float(lam), trunc)
        assert abs(e - ref["energy"]) <= 0.005 * ref["energy"], (name, e, ref["energy"])
        assert (d != ref["disp"]).mean() < 0.02, name
    assert (res["packed"] != res["generic"]).mean() < 0.02
    assert np.array_equal(res["packed"], res["packed_eager"])  # loading order changes nothing


@pytest.mark.parametrize("case", [(96, 72, 16, 5, 4, 8, 10, 2), (60, 44, 33, 5, 3, 6, 10, 1), (64, 48, 64, 7, 3, 6, 8, 2)],
                         ids=lambda c: "x".join(map(str, c)))
def test_fp16_active_lists_reproduce_the_dense_packed_sweep(case):
    # with the skip on, the active lists only enumerate the pixels whose flag is set, so the
    # packed fp16 sweep over lists must leave the same messages, trace and labels bit for bit,
    # launched directly and replayed from a graph
    W, H, D, window, levels, iters, lam, trunc = case
    pair = synth.make_pair(700 + W + D, W, H, D, 4, 2.0)
    res = {}
    for name, variant in (("dense", 0), ("lists", bps.BPS_VARIANT_LISTS), ("lists_eager", bps.BPS_VARIANT_LISTS | 8)):
        with bps.Stereo(W, H, D, levels, bps.BPS_MSG_FP16, device=DEV) as st:
            for lvl in range(levels):
                st.set_variant(lvl, variant)
            out = torch.empty((H, W), dtype=torch.int32, device=DEV)
            for graph in (False, True, True):
                st.stereo(to_dev(pair.left), to_dev(pair.right), window, 20, iters, lam, trunc, graph=graph, out=out)
                torch.cuda.synchronize()
                got = (out.cpu().numpy().copy(), st.get_trace().copy(),
                       [st.export_messages(lvl).cpu().numpy().copy() for lvl in range(levels)])
                if name in res:
                    prev = res[name]
                    assert np.array_equal(prev[0], got[0]) and np.array_equal(prev[1], got[1])
                    assert all(np.array_equal(a, b) for a, b in zip(prev[2], got[2]))
                res[name] = got
    for name in ("lists", "lists_eager"):
        assert np.array_equal(res[name][0], res["dense"][0]), name
        assert np.array_equal(res[name][1], res["dense"][1]), name
        assert all(np.array_equal(a, b) for a, b in zip(res[name][2], res["dense"][2])), name
