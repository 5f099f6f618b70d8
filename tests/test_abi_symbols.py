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
