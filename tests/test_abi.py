"""Host-side checks of the C ABI library (no GPU needed): it builds for
sm_103a, loads, and exports every entry point declared in include/rss.h."""
import os
import re
import ctypes

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rss.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rss_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for need in ["rss_build_tree", "rss_factor", "rss_apply", "rss_solve", "rss_free"]:
        assert need in names


def test_library_exports_every_declared_symbol():
    from paper_1609_08130_gb300 import rss
    rss.build()
    L = ctypes.CDLL(rss.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
    # the binding knows every declared entry point
    assert set(_declared()) <= set(rss._SIGS)


def test_free_is_null_safe_and_errors_are_reported():
    from paper_1609_08130_gb300 import rss
    L = rss.lib()
    L.rss_free(None)
    h = ctypes.c_void_p()
    st = L.rss_build_tree(None, -1, 2, 64, ctypes.byref(h))
    assert st == rss.RSS_EINVAL
    assert b"bad arguments" in L.rss_last_error()
    st = L.rss_build_tree(None, 10, 4, 64, ctypes.byref(h))
    assert st == rss.RSS_EINVAL
