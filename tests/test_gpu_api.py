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
