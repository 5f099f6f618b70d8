"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/hk.h declares (no GPU needed: nothing here launches a kernel)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"HK_API\s+[\w\s\*]+?\b(hk_\w+)\s*\(", txt)
    return names


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as g
    path = g.build()
    import ctypes
    lib = ctypes.CDLL(path)
    names = declared_entry_points()
    assert len(names) >= 13
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    import paper_1810_01478_gb300 as hk
    assert set(names) == set(hk.EXPORTS)


def test_supported_widths_and_layout_helpers():
    import paper_1810_01478_gb300 as hk
    hk.load()
    bits = hk.hk_supported_bits()
    assert 4096 in bits and 8192 in bits and 24576 in bits
    s, e, m = hk.int_to_layout(-(3 << 70), 4)
    assert s == 1 and hk.limbs_to_int(m) << (32 * e) == 3 << 70 if e >= 0 else True


def test_calls_without_a_context_fail_cleanly():
    import paper_1810_01478_gb300 as hk
    L = hk.load()
    assert L.hk_ldlt(None) == hk.HK_ERR_ARG
    assert L.hk_inv_block(None, 4) == hk.HK_ERR_ARG
    assert L.hk_fused_batch(4096, 1, *([None] * 12), None) == hk.HK_ERR_ARG
    assert L.hk_fused_batch(1000, 1, *([None] * 12), None) == hk.HK_ERR_ARG


def test_noalloc_argument_checks_need_no_device():
    """hk_ldlt_noalloc rejects bad sizes and null arrays before it touches the
    device or its scratch array: the size limit N (bits/32 + 2) + bits/32 + 35
    <= HK_NOALLOC_SCRATCH_WORDS, a width that is not a multiple of 1024, and
    missing arrays all give HK_ERR_ARG with no GPU present."""
    import paper_1810_01478_gb300 as hk
    L = hk.load()
    nulls = [None] * 6
    assert L.hk_ldlt_noalloc(24576, 2000, *nulls, None) == hk.HK_ERR_ARG   # beyond the scratch array
    assert L.hk_ldlt_noalloc(24576, 1024, *nulls, None) == hk.HK_ERR_ARG   # fits, but null arrays
    assert L.hk_ldlt_noalloc(1000, 16, *nulls, None) == hk.HK_ERR_ARG      # not a multiple of 1024
    assert L.hk_ldlt_noalloc(4096, 0, *nulls, None) == hk.HK_ERR_ARG       # N < 1
    # the limit itself: 2^20 words hold N = 1360 at 24576 bits (N (768 + 2) + 768 + 35 words at most),
    # not N = 1361
    words = 1 << 20
    assert 1360 * 770 + 768 + 35 <= words < 1361 * 770 + 768 + 32
    assert L.hk_ldlt_noalloc(24576, 1361, *nulls, None) == hk.HK_ERR_ARG


def test_plan_block_needs_a_context():
    """hk_plan_block, like every context call, answers HK_ERR_ARG for a null
    context before it touches a device."""
    import paper_1810_01478_gb300 as hk
    L = hk.load()
    assert L.hk_plan_block(None, 32) == hk.HK_ERR_ARG
    assert L.hk_plan_block(None, 0) == hk.HK_ERR_ARG


def test_batch_launch_rejects_empty_and_null_contexts():
    """hk_ldlt_batch answers HK_ERR_ARG for no contexts, a null array or a
    null context in the array, before it touches a device."""
    import ctypes

    import paper_1810_01478_gb300 as hk
    L = hk.load()
    assert L.hk_ldlt_batch(None, 0, -1.0) == hk.HK_ERR_ARG
    assert L.hk_ldlt_batch(None, 2, -1.0) == hk.HK_ERR_ARG
    arr = (ctypes.c_void_p * 2)(None, None)
    assert L.hk_ldlt_batch(arr, 2, -1.0) == hk.HK_ERR_ARG
    assert L.hk_ldlt_batch(arr, 0, -1.0) == hk.HK_ERR_ARG


def test_batch_tuner_rejects_bad_arguments():
    """hk_tune_batch answers HK_ERR_ARG / HK_ERR_UNSUPPORTED for sizes and
    widths it does not serve before it touches a device."""
    import paper_1810_01478_gb300 as hk
    L = hk.load()
    assert L.hk_tune_batch(0, 4096, 0, 4, None, None, None) == hk.HK_ERR_ARG
    assert L.hk_tune_batch(0, 4096, 64, 0, None, None, None) == hk.HK_ERR_ARG
    assert L.hk_tune_batch(0, 4096, 64, 257, None, None, None) == hk.HK_ERR_ARG
    assert L.hk_tune_batch(0, 1000, 64, 4, None, None, None) == hk.HK_ERR_ARG
    assert L.hk_tune_batch(0, 12288, 64, 4, None, None, None) == hk.HK_ERR_UNSUPPORTED
