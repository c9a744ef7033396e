"""The paper's parallel schedule with 2^d colours per level (Sec. 5) on the
GPU (RSS_FLAG_COLOUR_2D) against the oracle's phase-parallel schedule with
2^d colours (every box of a phase builds its lists and ID matrix from the
state at the phase start; shared near-field blocks receive additive Schur
updates).  The two compute the same factorization up to the order of those
additions, so apply and solve must agree within 10 eps, like the default
3^d schedule against the sequential oracle.
"""
import numpy as np
import pytest

import oracle
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


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = {
    "grid2d": (lambda: inputs.grid_points(64, 2), 0, 1e-6, 64),
    "random2d": (lambda: inputs.random_points(21, 3000, 2), 0, 1e-6, 64),
    "grid3d": (lambda: inputs.grid_points(16, 3), 1, 1e-3, 64),
    "grid2d_leaf16": (lambda: inputs.grid_points(64, 2), 0, 1e-6, 16),
}


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", list(CASES))
def test_colour2d_matches_oracle(pkg, case, prec):
    mk, kind, eps, leaf = CASES[case]
    pts = mk()
    n = len(pts)
    f = pkg.Factorization(_cuda(pts), kind, eps, leaf=leaf, prec=pkg.FP64 if prec == "fp64" else pkg.MIXED,
                          flags=pkg.rss.FLAG_COLOUR_2D)
    of = oracle.Factor(oracle.Tree(pts, leaf), kind, eps, schedule=2)
    st = f.stats()
    ob = of.boxes()
    # same boxes in the same (2^d colour-major, Morton) order; box sizes above
    # the leaves follow the children's ranks, which may differ near ties
    assert st["nbox"] == len(ob)
    assert [b["depth"] for b in ob] == st["depth"].tolist()
    leaf = st["depth"] == st["maxdepth"]
    assert [b["b"] for b in ob if b["depth"] == st["maxdepth"]] == st["b"][leaf].tolist()
    if prec == "fp64":
        assert np.mean(np.array([b["k"] for b in ob]) == st["k"]) > 0.9
    x = inputs.rhs(11, n, 3)
    Ax = oracle.matvec(pts, kind, x)
    Fo = of.apply(x)
    Fg = f.apply(_cuda(x)).cpu().numpy()
    assert np.linalg.norm(Fg - Fo) / np.linalg.norm(Fo) <= 10 * eps
    ea_g = np.linalg.norm(Ax - Fg) / np.linalg.norm(Ax)
    ea_o = np.linalg.norm(Ax - Fo) / np.linalg.norm(Ax)
    assert ea_g <= ea_o + 10 * eps
    So = of.solve(Ax)
    Sg = f.solve(_cuda(Ax)).cpu().numpy()
    assert np.linalg.norm(Sg - So) / np.linalg.norm(So) <= 10 * eps
    # more than four columns take the one-CTA-per-box sweeps
    X6 = inputs.rhs(12, n, 6)
    np.testing.assert_allclose(f.solve(_cuda(X6)).cpu().numpy(), of.solve(X6), rtol=0,
                               atol=10 * eps * np.abs(of.solve(X6)).max())


def test_colour2d_runs_fewer_phases(pkg):
    """2^d colours: 4 ID launches per level in 2D (8 x 8 and 4 x 4 boxes on
    the 64^2 grid: 8 phases), against 9 per level with 3^d colours (18)."""
    pts = _cuda(inputs.grid_points(64, 2))
    counts = {}
    for flags in (0, pkg.rss.FLAG_COLOUR_2D):
        f = pkg.Factorization(pts, 0, 1e-6, leaf=64, prec=pkg.MIXED, profile=True,
                              flags=flags | pkg.rss.FLAG_NO_AUTOTUNE)
        counts[flags] = f.profile()["id"]["launches"]
    assert counts[0] == 18 and counts[pkg.rss.FLAG_COLOUR_2D] == 8, counts


def test_colour2d_refined_solve(pkg):
    """GMRES-IR with the 2^d-colour FP32 factor reaches 1e-10, checked with
    the oracle's matvec on sampled rows."""
    pts = inputs.grid_points(128, 2)
    f = pkg.Factorization(_cuda(pts), 0, 1e-6, leaf=64, prec=pkg.MIXED, flags=pkg.rss.FLAG_COLOUR_2D)
    b = inputs.rhs(1, len(pts), 2)
    x, iters, rel = f.solve_refined(_cuda(b), tol=1e-10, maxit=10)
    assert rel <= 1e-10
    rows = np.arange(0, len(pts), 97)
    r = b[:, rows] - oracle.matvec(pts, 0, x.cpu().numpy(), rows=rows)
    assert np.abs(r).max() <= 1e-9 * np.abs(b).max()
