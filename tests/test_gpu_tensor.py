"""The FP32 factor's Schur-complement update on the tensor cores (tcgen05,
three TF32 products per K step) against the same update on the FP32 SIMT
units, and both against the oracle.  The two paths compute the same
factorization up to FP32 rounding; the TF32 split keeps the tensor-core path
at FP32 accuracy, so the factors must agree to FP32 level and each must meet
the 10 eps parity bar against the FP64 oracle.

Cases cover one and several 128-row tiles of J (|J| up to a few hundred at
the 2D leaves, over a thousand at upper levels), ranks r below and above the
64-wide staged K chunk (the 32^3 grid's upper level, checked against the
exact operator: too large for the dense oracle), ragged tiles and the
2^d-colour schedule whose shared pair blocks take atomic updates.
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
    "grid2d_64": (lambda: inputs.grid_points(64, 2), 0, 1e-6, 64, 0),
    "grid2d_48_leaf40": (lambda: inputs.grid_points(48, 2), 0, 1e-6, 40, 0),
    "random2d": (lambda: inputs.random_points(21, 3000, 2), 0, 1e-6, 64, 0),
    "grid3d_16": (lambda: inputs.grid_points(16, 3), 1, 1e-3, 64, 0),
    "grid3d_32": (lambda: inputs.grid_points(32, 3), 1, 1e-3, 64, 0),
    "grid2d_64_colour2": (lambda: inputs.grid_points(64, 2), 0, 1e-6, 64, 4),
}


@pytest.mark.parametrize("case", list(CASES))
def test_tensor_core_schur_matches_simt_and_oracle(pkg, case):
    mk, kind, eps, leaf, flags = CASES[case]
    pts = mk()
    n = len(pts)
    P = _cuda(pts)
    f_tc = pkg.Factorization(P, kind, eps, leaf=leaf, prec=pkg.MIXED, flags=flags)
    f_sm = pkg.Factorization(P, kind, eps, leaf=leaf, prec=pkg.MIXED, flags=flags | pkg.rss.FLAG_NO_TENSOR_CORES)
    st = f_tc.stats()
    if case == "grid3d_32":
        # boxes eliminating more than one staged K chunk of 64
        assert (st["b"] - st["k"]).max() > 64
    assert st["nj"].max() > 128  # several row tiles of J
    x = inputs.rhs(5, n, 2)
    y_tc = f_tc.apply(_cuda(x)).cpu().numpy()
    y_sm = f_sm.apply(_cuda(x)).cpu().numpy()
    assert np.linalg.norm(y_tc - y_sm) / np.linalg.norm(y_sm) <= 1e-5
    if n > 8192:
        # too large for the dense oracle: the exact operator instead
        Ax = f_tc.matvec(_cuda(x)).cpu().numpy()
        assert np.linalg.norm(y_tc - Ax) / np.linalg.norm(Ax) <= 10 * eps
        return
    of = oracle.Factor(oracle.Tree(pts, leaf), kind, eps, schedule=2 if flags else 0)
    yo = of.apply(x)
    assert np.linalg.norm(y_tc - yo) / np.linalg.norm(yo) <= 10 * eps
    s_tc = f_tc.solve(_cuda(yo)).cpu().numpy()
    so = of.solve(yo)
    assert np.linalg.norm(s_tc - so) / np.linalg.norm(so) <= 10 * eps


def test_tensor_core_schur_full_size_refined(pkg):
    """The bench's 512^2 step with the tensor-core update: GMRES-IR reaches
    1e-10 with as few inner iterations as with the SIMT update."""
    P = _cuda(inputs.grid_points(512, 2))
    b = _cuda(inputs.rhs(1, P.shape[0], 4))
    res = {}
    for flags in (0, pkg.rss.FLAG_NO_TENSOR_CORES):
        f = pkg.Factorization(P, 0, 1e-6, leaf=64, prec=pkg.MIXED, flags=flags)
        _, iters, rel = f.solve_refined(b, tol=1e-10, maxit=10)
        res[flags] = (iters, rel)
        del f
    assert res[0][1] <= 1e-10 and res[0][0] <= res[pkg.rss.FLAG_NO_TENSOR_CORES][0], res
