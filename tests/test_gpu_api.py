"""Boundary entry points beyond the factor and its sweeps: the statistics as
JSON (the form of the interface's stats call), consistent with the integer
form and with the tree."""
import numpy as np
import pytest

from paper_1609_08130_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1609_08130_gb300 as p
    p.build()
    return p


@pytest.mark.parametrize("flags", [0, 4])
def test_stats_json_matches_stats(pkg, flags):
    pts = torch.from_numpy(inputs.grid_points(64, 2)).cuda()
    f = pkg.Factorization(pts, 0, 1e-6, leaf=64, prec=pkg.MIXED, profile=True, flags=flags)
    st = f.stats()
    js = f.stats_json()
    assert js["n"] == st["n"] == 4096 and js["boxes"] == st["nbox"] and js["top_block"] == st["ntop"]
    assert js["precision"] == "fp32" and js["colours_per_level"] == (4 if flags else 9)
    assert js["factor_bytes"] == st["factor_bytes"] and js["used_bytes"] == st["used_bytes"]
    np.testing.assert_array_equal(js["box_k"], st["k"])
    np.testing.assert_array_equal(js["box_b"], st["b"])
    np.testing.assert_array_equal(js["box_nj"], st["nj"])
    # per-depth sums agree with the per-box records; the leaves hold every point
    for lv in js["levels"]:
        sel = st["depth"] == lv["depth"]
        assert lv["boxes"] == int(sel.sum()) and lv["k_sum"] == int(st["k"][sel].sum())
    leaf = [lv for lv in js["levels"] if lv["depth"] == js["maxdepth"]][0]
    assert leaf["b_sum"] == 4096
    assert js["profile_ms"]["id"] > 0 and js["profile_ms"]["schur"] > 0


def _busy(torch):
    """Queue some tens of milliseconds of work on the current stream."""
    a = torch.randn(8192, 8192, device="cuda", dtype=torch.float32)
    for _ in range(8):
        a = (a @ a) * 1e-4
    return a


def test_async_calls_return_before_their_work_is_done(pkg):
    """RSS_FLAG_ASYNC: rss_solve and rss_apply return once their work is
    queued behind earlier work on the stream (the stream is still busy on
    return), and give the same bits as the synchronous factor once the
    stream is synchronised; without the flag the stream is idle on return."""
    pts = torch.from_numpy(inputs.grid_points(128, 2)).cuda()
    fs = pkg.Factorization(pts, 0, 1e-6, leaf=64, prec=pkg.MIXED)
    fa = pkg.Factorization(pts, 0, 1e-6, leaf=64, prec=pkg.MIXED, flags=pkg.rss.FLAG_ASYNC)
    fa.sync()
    x = torch.from_numpy(inputs.rhs(3, len(pts), 2)).cuda()
    for op in ("solve", "apply"):
        ref = getattr(fs, op)(x)
        _busy(torch)
        y = getattr(fa, op)(x)
        assert not torch.cuda.current_stream().query(), op  # still queued
        fa.sync()
        assert torch.equal(y, ref), op
        _busy(torch)
        getattr(fs, op)(x)
        assert torch.cuda.current_stream().query(), op  # the synchronous call waited


def test_async_factor_reports_a_device_error_later(pkg):
    """Two points at distance exactly 1 make K = 0 (log 1 = 0); with
    diag = 0 the matrix is zero and the top block's LU meets a zero pivot.
    The synchronous factor returns RSS_ENUMERIC; the asynchronous one
    returns RSS_OK and rss_sync reports RSS_ENUMERIC once."""
    pts = torch.tensor([[0.0, 0.0], [1.0, 0.0]], dtype=torch.float64).cuda()
    with pytest.raises(pkg.RSSError) as e:
        pkg.Factorization(pts, 0, 1e-6, leaf=64, prec=pkg.FP64, diag=0.0)
    assert e.value.status == pkg.rss.RSS_ENUMERIC
    f = pkg.Factorization(pts, 0, 1e-6, leaf=64, prec=pkg.FP64, diag=0.0, flags=pkg.rss.FLAG_ASYNC)
    with pytest.raises(pkg.RSSError) as e:
        f.sync()
    assert e.value.status == pkg.rss.RSS_ENUMERIC
    f.sync()  # reported once
