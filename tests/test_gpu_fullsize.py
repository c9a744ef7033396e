"""GPU parity on the paths the full-size workloads take.

The 512 x 512 step (N = 262144) runs colour phases of about 455 boxes; some
launch choices switch at 300 boxes per phase (the one-launch elimination, the
ID's default fold shape), so the oracle comparison is repeated on a problem
whose phases are that large: a 128 x 128 grid with leaves of at most 4
points (4096 leaves, about 455 boxes per leaf phase; the oracle's dense
state is 2 GB).  At the full size itself, where no dense oracle fits, the
apply error of the FP32 and FP64 factors is measured against the FFT form of A
(rss_matvec), which the parity suite pins to the oracle's direct sum; the
error is reported as a norm over the whole vector, per leaf box and per
entry, so that an error confined to a few boxes is not averaged away.
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


@pytest.fixture(scope="module")
def large_phases():
    """128^2 grid, leaf 4, eps 1e-6: the oracle factor and reference vectors."""
    pts = inputs.grid_points(128, 2)
    eps = 1e-6
    of = oracle.Factor(oracle.Tree(pts, 4), 0, eps)
    x = inputs.rhs(11, len(pts), 2)
    Ax = oracle.matvec(pts, 0, x)
    return dict(pts=pts, eps=eps, of=of, x=x, Ax=Ax, Fo=of.apply(x), So=of.solve(Ax))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("tuned", [True, False])
def test_phases_of_many_boxes_match_oracle(pkg, large_phases, prec, tuned):
    """Colour phases of >= 300 boxes (the one-launch elimination and the
    large-phase ID shapes, autotuned or the built-in defaults) against the
    oracle: apply and solve within 10 eps."""
    P = large_phases
    pts, eps, of = P["pts"], P["eps"], P["of"]
    f = pkg.Factorization(_cuda(pts), 0, eps, leaf=4, prec=pkg.FP64 if prec == "fp64" else pkg.MIXED,
                          flags=0 if tuned else pkg.rss.FLAG_NO_AUTOTUNE)
    st = f.stats()
    ob = of.boxes()
    assert st["nbox"] == len(ob)
    assert [b["depth"] for b in ob] == st["depth"].tolist()
    leaf_boxes = int(np.sum(st["depth"] == st["maxdepth"]))
    assert leaf_boxes // 9 >= 300, leaf_boxes  # 9 colour phases per level
    if prec == "fp64":
        assert np.mean(np.array([b["k"] for b in ob]) == st["k"]) > 0.9
    Fg = f.apply(_cuda(P["x"])).cpu().numpy()
    rel = np.linalg.norm(Fg - P["Fo"]) / np.linalg.norm(P["Fo"])
    assert rel <= 10 * eps, rel
    Sg = f.solve(_cuda(P["Ax"])).cpu().numpy()
    rel_s = np.linalg.norm(Sg - P["So"]) / np.linalg.norm(P["So"])
    assert rel_s <= 10 * eps, rel_s
    ea = np.linalg.norm(P["Ax"] - Fg) / np.linalg.norm(P["Ax"])
    assert ea <= 10 * eps, ea


def _leaf_rows(pkg, pts_gpu, leaf):
    """Original indices of the points of every leaf box of the tree."""
    tr = pkg.Tree(pts_gpu, leaf)
    perm = tr.perm()
    nd = tr.nodes()
    out = []
    for node in np.nonzero(nd["depth"] == tr.maxdepth)[0]:
        s, c = int(nd["start"][node]), int(nd["count"][node])
        out.append(perm[s:s + c])
    return out


def test_full_size_apply_error(pkg, capsys):
    """512^2 grid (N = 262144), eps 1e-6: ||Ax - Fx|| / ||Ax|| within 10 eps
    against the FFT operator, for the FP32 factor the bench times and for the
    FP64 factor; per leaf box, ||(Ax - Fx)_B|| / ||(Ax)_B||.  The FP64
    factor's error is the method's (about 1e-9 here, the oracle's size at
    N = 4096-16384), and no box may exceed 10 eps.  The FP32 factor's error
    is FP32 rounding of the stored blocks, amplified in a box by the size of
    its interpolation matrix T (x_S += T x_R): reported, and bounded by 100
    eps per box; GMRES-IR removes it."""
    eps = 1e-6
    pts = _cuda(inputs.grid_points(512, 2))
    x = _cuda(inputs.rhs(1, pts.shape[0], 2))
    leaves = _leaf_rows(pkg, pts, 64)
    out = {}
    for prec in (pkg.MIXED, pkg.FP64):
        f = pkg.Factorization(pts, 0, eps, leaf=64, prec=prec)
        Ax = f.matvec(x).cpu().numpy()
        res = Ax - f.apply(x).cpu().numpy()
        glob = np.linalg.norm(res) / np.linalg.norm(Ax)
        worst_box = max(np.linalg.norm(res[:, rows]) / np.linalg.norm(Ax[:, rows]) for rows in leaves)
        worst_entry = np.abs(res).max() / np.abs(Ax).max()
        out[prec] = (glob, worst_box, worst_entry)
        del f
    with capsys.disabled():
        for prec, name in ((pkg.MIXED, "FP32"), (pkg.FP64, "FP64")):
            g, wb, we = out[prec]
            print(f"\n512^2 {name} factor apply error: global {g:.2e}, worst leaf box {wb:.2e}, "
                  f"worst entry {we:.2e} (eps {eps:g})")
    g, wb, _ = out[pkg.FP64]
    assert g <= 10 * eps and wb <= 10 * eps, out[pkg.FP64]
    g, wb, _ = out[pkg.MIXED]
    assert g <= 10 * eps, g
    assert wb <= 100 * eps, wb


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["grid2d", "grid3d", "random2d"])
def test_logdet_matches_oracle(pkg, case, prec):
    """rss_logdet against the oracle's log |det F| (Sec. 3.3: the product of
    the diagonal blocks' determinants) at eps 1e-6.  Both approximate
    log |det A|.  FP64: within 10 eps relative.  FP32 factor: by first-order
    perturbation, log det (F + dF) - log det F = tr(F^{-1} dF), at most
    N ||F^{-1}|| ||dF||; with ||F^{-1}|| <= 2 for these second-kind matrices
    and ||dF|| / ||F|| estimated by the relative difference of the two
    factors' applies to random vectors, the bar is 2 N times that."""
    mk = {"grid2d": (lambda: inputs.grid_points(64, 2), 0),
          "grid3d": (lambda: inputs.grid_points(16, 3), 1),
          "random2d": (lambda: inputs.random_points(21, 3000, 2), 0)}[case]
    pts, kind = mk[0](), mk[1]
    n = len(pts)
    eps = 1e-6
    of = oracle.Factor(oracle.Tree(pts, 64), kind, eps)
    f = pkg.Factorization(_cuda(pts), kind, eps, leaf=64, prec=pkg.FP64 if prec == "fp64" else pkg.MIXED)
    ld_o = of.logdet()
    ld_g = float(f.logdet()[0])
    if prec == "fp64":
        tol = 10 * eps * abs(ld_o)
    else:
        x = inputs.rhs(17, n, 2)
        yo = of.apply(x)
        d = np.linalg.norm(f.apply(_cuda(x)).cpu().numpy() - yo) / np.linalg.norm(yo)
        assert d <= 10 * eps
        tol = 2 * n * d
    assert abs(ld_g - ld_o) <= tol, (ld_g, ld_o, tol)
