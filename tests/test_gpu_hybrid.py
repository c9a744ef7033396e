"""The hybrid factorization RS-WS (Sec. 3.4, Algorithm 2) on the GPU
(RSS_FLAG_HYBRID) against the oracle's (hybrid=True): at every depth a weak
pass (each box compressed against everything outside it, eliminated against
its own skeleton) then the strong pass, and a last weak pass at depth 1.
Same boxes in the same order, apply and solve within 10 eps of the oracle,
the GPU's own apply error within 10 eps of the oracle's, less memory in all
and a smaller top block than RS-S (the paper's reason for the hybrid), GMRES-IR to
1e-10 with the FP32 hybrid factor."""
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
    "grid3d": (lambda: inputs.grid_points(12, 3), 1, 1e-3, 27),
}


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", list(CASES))
def test_hybrid_matches_oracle(pkg, case, prec):
    mk, kind, eps, leaf = CASES[case]
    pts = mk()
    n = len(pts)
    P = _cuda(pts)
    pr = pkg.FP64 if prec == "fp64" else pkg.MIXED
    f = pkg.Factorization(P, kind, eps, leaf=leaf, prec=pr, flags=pkg.rss.FLAG_HYBRID)
    of = oracle.Factor(oracle.Tree(pts, leaf), kind, eps, hybrid=True)
    st = f.stats()
    ob = of.boxes()
    assert st["nbox"] == len(ob)
    assert [b["depth"] for b in ob] == st["depth"].tolist()
    assert min(st["depth"]) == 1  # the last weak pass
    # weak boxes eliminate against their skeleton only: |J| = k
    weak = np.array([b["weak"] for b in ob], dtype=bool)
    np.testing.assert_array_equal(st["nj"][weak], st["k"][weak])
    if prec == "fp64":
        assert np.mean(np.array([b["k"] for b in ob]) == st["k"]) > 0.9
    x = inputs.rhs(13, n, 3)
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
    # against RS-S on the same GPU: a smaller top block and less memory in
    # all (box records plus the dense top block; on a small 3D grid the box
    # records alone can be larger, the weak passes keep more skeletons)
    f0 = pkg.Factorization(P, kind, eps, leaf=leaf, prec=pr)
    s0 = f0.stats()
    assert st["ntop"] < s0["ntop"]
    assert st["used_bytes"] + 8 * st["ntop"] ** 2 < s0["used_bytes"] + 8 * s0["ntop"] ** 2


def test_hybrid_refined_solve(pkg):
    pts = inputs.grid_points(128, 2)
    f = pkg.Factorization(_cuda(pts), 0, 1e-6, leaf=64, prec=pkg.MIXED, flags=pkg.rss.FLAG_HYBRID)
    b = inputs.rhs(2, len(pts), 2)
    x, iters, rel = f.solve_refined(_cuda(b), tol=1e-10, maxit=10)
    assert rel <= 1e-10
    rows = np.arange(0, len(pts), 101)
    r = b[:, rows] - oracle.matvec(pts, 0, x.cpu().numpy(), rows=rows)
    assert np.abs(r).max() <= 1e-9 * np.abs(b).max()


def test_hybrid_refuses_the_2d_schedule(pkg):
    P = _cuda(inputs.grid_points(32, 2))
    with pytest.raises(pkg.RSSError) as e:
        pkg.Factorization(P, 0, 1e-6, leaf=64, flags=pkg.rss.FLAG_HYBRID | pkg.rss.FLAG_COLOUR_2D)
    assert e.value.status == pkg.rss.RSS_EINVAL
