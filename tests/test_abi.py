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


def test_autotune_table_host_api():
    """The autotuner's table is host state: a shape is accepted for a key
    exactly when it is a candidate for the key's box-width class (the rule
    the binding's shape_fits states, plus several CTAs per box at width 256
    only with two threads per column), the table returns what was set with
    the candidate timings zero (nothing timed), and clearing empties it."""
    from paper_1609_08130_gb300 import rss
    L = rss.lib()
    L.rss_autotune_clear()
    try:
        want = {}
        for width in (64, 128, 256):
            for cls, (tpc, g, ctas, rows) in enumerate(rss.AUTOTUNE_SHAPES):
                ok = rss.shape_fits(width, tpc, g, rows) and not (width == 256 and ctas > 1 and tpc != 2)
                st = L.rss_autotune_set(8, width, cls, tpc, g, ctas, rows)
                assert st == (rss.RSS_OK if ok else rss.RSS_EINVAL), (width, tpc, g, ctas, rows, st)
                if ok:
                    want[(8, width, cls)] = (tpc, g, ctas, rows)
        assert L.rss_autotune_set(3, 64, 0, 1, 1, 1, 1) == rss.RSS_EINVAL  # element size
        assert L.rss_autotune_set(4, 96, 0, 1, 1, 1, 1) == rss.RSS_EINVAL  # width class
        assert L.rss_autotune_set(4, 64, 41, 1, 1, 1, 1) == rss.RSS_EINVAL  # phase class
        got = {(t["elem_bytes"], t["width"], t["phase_class"]): (t["tpc"], t["groups"], t["ctas"], t["rows"])
               for t in rss.autotune_table()}
        assert got == want
        assert all(u == 0 for t in rss.autotune_table() for u in t["us"])
        nb = ctypes.c_size_t(4)
        buf = (ctypes.c_int32 * 1)()
        assert L.rss_autotune_table(buf, ctypes.byref(nb)) == rss.RSS_EINVAL  # buffer too small
        assert nb.value == 4 * len(want) * (7 + len(rss.AUTOTUNE_SHAPES))
    finally:
        L.rss_autotune_clear()
    assert rss.autotune_table() == [] and rss.autotune_elim_table() == []
