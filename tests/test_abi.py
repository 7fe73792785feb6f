"""The C ABI library builds, loads without a GPU and exports every entry point that
include/bpstereo.h declares; host-only argument checks return the documented codes."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1709_06509_gb300 as bps
from paper_1709_06509_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bpstereo.h")


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return bps.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bps_\w+)\s*\(", text)))


def test_header_declares_the_path():
    names = declared_functions()
    for n in ("bps_build_cost_volume", "bps_bp_solve", "bps_wta_disparity", "bps_energy", "bps_create",
              "bps_destroy", "bps_workspace_bytes"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", bps.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (bps_\w+)", out))
    assert set(names) <= exported


def test_binding_covers_every_entry_point():
    for n in declared_functions():
        assert n in bps._SIGS, n
        assert hasattr(bps, n) or n == "bps_status_string", n


def test_status_strings(lib):
    assert bps.status_string(bps.BPS_OK) == "ok"
    for code in (bps.BPS_ERR_ARG, bps.BPS_ERR_UNSUPPORTED, bps.BPS_ERR_CUDA, bps.BPS_ERR_WORKSPACE,
                 bps.BPS_ERR_TIMEOUT, bps.BPS_ERR_STATE):
        assert bps.status_string(code) not in ("ok", "unknown status")
    assert bps.status_string(-99) == "unknown status"


def test_workspace_bytes_validation(lib):
    assert bps.bps_workspace_bytes(0, 5, 4, 1, bps.BPS_MSG_U8) == 0
    assert bps.bps_workspace_bytes(5, 5, 0, 1, bps.BPS_MSG_U8) == 0
    assert bps.bps_workspace_bytes(5, 5, bps.BPS_MAX_D + 1, 1, bps.BPS_MSG_U8) == 0
    assert bps.bps_workspace_bytes(5, 5, 4, 0, bps.BPS_MSG_U8) == 0
    assert bps.bps_workspace_bytes(5, 5, 4, bps.BPS_MAX_LEVELS + 1, bps.BPS_MSG_U8) == 0
    assert bps.bps_workspace_bytes(5, 5, 4, 1, 7) == 0
    small = bps.bps_workspace_bytes(96, 72, 16, 4, bps.BPS_MSG_U8)
    big = bps.bps_workspace_bytes(96, 72, 16, 4, bps.BPS_MSG_INT32)
    assert 0 < small < big
    assert bps.bps_workspace_bytes(450, 375, 64, 4, bps.BPS_MSG_U8) % 256 == 0
    # the u8 form stores about a quarter of the int32 form's message bytes
    assert bps.bps_workspace_bytes(1920, 1080, 256, 4, bps.BPS_MSG_U8) < 0.4 * bps.bps_workspace_bytes(
        1920, 1080, 256, 4, bps.BPS_MSG_INT32)


def test_create_rejects_bad_arguments_without_touching_the_gpu(lib):
    ctx = ctypes.c_void_p()
    assert lib.bps_create(None, 8, 8, 4, 1, 1, None, 0) == bps.BPS_ERR_ARG
    assert lib.bps_create(ctypes.byref(ctx), 0, 8, 4, 1, 1, None, 0) == bps.BPS_ERR_ARG
    assert ctx.value is None
    need = bps.bps_workspace_bytes(8, 8, 4, 1, bps.BPS_MSG_U8)
    # too small, then misaligned caller workspace
    assert lib.bps_create(ctypes.byref(ctx), 8, 8, 4, 1, 1, 256, need - 1) == bps.BPS_ERR_WORKSPACE
    assert lib.bps_create(ctypes.byref(ctx), 8, 8, 4, 1, 1, 4096 + 16, need) == bps.BPS_ERR_WORKSPACE
    assert lib.bps_destroy(None) == bps.BPS_OK
    assert lib.bps_build_cost_volume(None, None, None, 8, 3, 20, None, None) == bps.BPS_ERR_ARG
    assert lib.bps_bp_solve(None, 1, 1, 1, 1, 0, None, None) == bps.BPS_ERR_ARG
    assert lib.bps_wta_disparity(None, None, None) == bps.BPS_ERR_ARG
    assert lib.bps_energy(None, None, 1, 1, None, None, None) == bps.BPS_ERR_ARG


def test_binding_constants_match_the_header():
    # every #define of the header has the same value in the binding
    text = open(HEADER).read()
    for name, value in re.findall(r"#define\s+(BPS_\w+)\s+(-?\d+)\b", text):
        assert getattr(bps, name) == int(value), name


def test_autotuner_candidate_sets():
    # scales small enough for the cluster launch get the small-scale set, scales of at least
    # LIST_MIN_LANES lanes also get the list and staged forms, and direction-parallel variants
    # are dropped where a pixel needs more than 8 lane groups (more than 128 labels)
    from paper_1709_06509_gb300 import autotune as at

    tiny = at._candidates(1000, 4)
    assert set(tiny) == set(at.SMALL_CANDIDATES)
    mid = at._candidates(at.LIST_MIN_LANES, 4)
    assert set(mid) == set(at.SMALL_CANDIDATES) | set(at.LARGE_CANDIDATES) and len(mid) == len(set(mid))
    big = at._candidates(at.CLUSTER_MAX_LANES + 1, 4)
    assert set(big) == set(at.LARGE_CANDIDATES)
    wide = at._candidates(at.CLUSTER_MAX_LANES + 1, 16)
    dp = bps.BPS_VARIANT_DPAR | bps.BPS_VARIANT_DPAR_LISTS
    assert wide and all(not (v & dp) for v in wide)
    assert all(v & bps.BPS_VARIANT_LISTS for v in at.LARGE_CANDIDATES if v & bps.BPS_VARIANT_STAGED_LISTS)
    # the blocking-depth axis: depth 2 only when asked for, on the scales that get the large set
    assert not any(v & bps.BPS_VARIANT_BLOCK2 for v in big + mid + tiny)
    deep = at._candidates(at.CLUSTER_MAX_LANES + 1, 4, depths=(1, 2))
    assert set(deep) == set(at.LARGE_CANDIDATES) | set(at.BLOCKED_CANDIDATES) and len(deep) == len(set(deep))
    assert set(at._candidates(1000, 4, depths=(1, 2))) == set(at.SMALL_CANDIDATES)
    assert all(v & bps.BPS_VARIANT_BLOCK2 for v in at.BLOCKED_CANDIDATES)
    assert set(at.CANDIDATES) == set(at.SMALL_CANDIDATES) | set(at.LARGE_CANDIDATES) | set(at.BLOCKED_CANDIDATES)


def test_every_autotuner_candidate_has_an_exact_gpu_test():
    # no sweep variant the autotuner can pick lacks an oracle-exact GPU test
    import importlib.util

    from paper_1709_06509_gb300 import autotune

    spec = importlib.util.spec_from_file_location("gpu_parity", os.path.join(os.path.dirname(__file__),
                                                                             "test_gpu_parity.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    assert set(autotune.CANDIDATES) <= set(mod.SWEEP_VARIANTS_TESTED)
