"""Generalized square root on the GPU (the remark after Eq. 3.11): for
symmetric positive definite A, F = V D V^T and F^{1/2} = V C with D = C C^T.
A square root is not unique (F^{1/2} Q is one too for orthogonal Q), so the
checks are what defines one, not a comparison with the oracle's numbers:
  - F^{1/2} (F^{1/2})^T x = F x (the factor's own apply);
  - ||(F^{1/2})^T x||^2 = x^T F x, and within 10 eps of x^T A x from the
    oracle's direct sum;
  - eps = 0 keeps every DOF in the top block, D = A, and F^{1/2} is the
    Cholesky factor of A itself (unique): numpy's, in the tree order;
  - a negative definite matrix is refused.
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
    "grid2d": (lambda: inputs.grid_points(64, 2), 0, 1e-6, {}),
    "random2d": (lambda: inputs.random_points(21, 3000, 2), 0, 1e-6, {}),
    "grid3d": (lambda: inputs.grid_points(16, 3), 1, 1e-3, {}),
    "first_kind2d": (lambda: inputs.grid_points(64, 2), 0, 1e-6,
                     {"diag": inputs.cell_self_integral(0, 1 / 64), "weight": 1 / 64 ** 2}),
}


@pytest.mark.parametrize("flags", [0, 4])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", list(CASES))
def test_square_root_reproduces_the_factor(pkg, case, prec, flags):
    mk, kind, eps, mat = CASES[case]
    pts = mk()
    n = len(pts)
    f = pkg.Factorization(_cuda(pts), kind, eps, leaf=64, prec=pkg.FP64 if prec == "fp64" else pkg.MIXED,
                          flags=flags, **mat)
    x = inputs.rhs(31, n, 3)
    xg = _cuda(x)
    Fx = f.apply(xg).cpu().numpy()
    ssx = f.sqrt_apply(f.sqrt_apply(xg, transpose=True)).cpu().numpy()
    tol = 1e-11 if prec == "fp64" else 1e-5
    assert np.linalg.norm(ssx - Fx) / np.linalg.norm(Fx) <= tol
    # ||(F^{1/2})^T x||^2 = x^T F x, and close to x^T A x
    st = f.sqrt_apply(xg, transpose=True).cpu().numpy()
    q_f = np.sum(x * Fx, axis=1)
    q_s = np.sum(st * st, axis=1)
    np.testing.assert_allclose(q_s, q_f, rtol=tol)
    Ax = oracle.matvec(pts, kind, x, diag=mat.get("diag", 1.0), w=mat.get("weight"))
    q_a = np.sum(x * Ax, axis=1)
    np.testing.assert_allclose(q_s, q_a, rtol=10 * eps)


def test_square_root_exact_limit_is_cholesky(pkg):
    """eps = 0: no compression, every DOF stays in the top block, D = A and
    F^{1/2} = chol(A) (lower), applied in the tree order of the DOFs."""
    pts = inputs.grid_points(24, 2)
    n = len(pts)
    f = pkg.Factorization(_cuda(pts), 0, 0.0, leaf=64, prec=pkg.FP64)
    assert f.stats()["ntop"] == n
    A = oracle.dense_matrix(pts, 0)
    perm = pkg.Tree(_cuda(pts), 64).perm()  # tree order -> original index
    Lt = np.linalg.cholesky(A[np.ix_(perm, perm)])
    x = inputs.rhs(5, n, 2)
    want = np.empty_like(x)
    want[:, perm] = (Lt @ x[:, perm].T).T
    got = f.sqrt_apply(_cuda(x)).cpu().numpy()
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())


def test_square_root_refuses_an_indefinite_matrix(pkg):
    pts = _cuda(inputs.grid_points(32, 2))
    f = pkg.Factorization(pts, 0, 1e-6, leaf=64, prec=pkg.FP64, diag=-1.0)
    with pytest.raises(pkg.RSSError) as e:
        f.sqrt_apply(_cuda(inputs.rhs(1, 1024, 1)))
    assert e.value.status == pkg.rss.RSS_ENUMERIC


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["grid2d", "random2d", "grid3d"])
def test_symmetric_storage(pkg, case, prec):
    """RSS_FLAG_SYMMETRIC_STORAGE keeps E only (G = E^T for the symmetric
    kernels, Sec. 3.3): the same factorization up to rounding, with |J| r
    fewer entries per box, within 10 eps of the oracle; the solve, the
    apply, the refined solve and the square root all read E transposed."""
    mk, kind, eps, mat = CASES[case]
    pts = mk()
    n = len(pts)
    P = _cuda(pts)
    pr = pkg.FP64 if prec == "fp64" else pkg.MIXED
    f0 = pkg.Factorization(P, kind, eps, leaf=64, prec=pr)
    f1 = pkg.Factorization(P, kind, eps, leaf=64, prec=pr, flags=pkg.rss.FLAG_SYMMETRIC_STORAGE)
    s0, s1 = f0.stats(), f1.stats()
    np.testing.assert_array_equal(s0["k"], s1["k"])
    saved = int(np.sum(s1["nj"] * (s1["b"] - s1["k"]))) * (8 if prec == "fp64" else 4)
    assert s0["used_bytes"] - s1["used_bytes"] == saved
    x = inputs.rhs(41, n, 6)  # 6 columns: the one-CTA-per-box sweeps too
    xg = _cuda(x)
    tol = 1e-12 if prec == "fp64" else 2e-6
    for op in ("apply", "solve"):
        a0 = getattr(f0, op)(xg).cpu().numpy()
        a1 = getattr(f1, op)(xg).cpu().numpy()
        assert np.linalg.norm(a1 - a0) / np.linalg.norm(a0) <= tol, op
        a4 = getattr(f1, op)(xg[:4]).cpu().numpy()  # the chunked solve sweeps
        assert np.linalg.norm(a4 - a1[:4]) / np.linalg.norm(a1[:4]) <= tol, op
    of = oracle.Factor(oracle.Tree(pts, 64), kind, eps)
    yo = of.apply(x)
    assert np.linalg.norm(f1.apply(xg).cpu().numpy() - yo) / np.linalg.norm(yo) <= 10 * eps
    _, _, rel = f1.solve_refined(_cuda(yo[:2]), tol=1e-10, maxit=10)
    assert rel <= 1e-10
    ssx = f1.sqrt_apply(f1.sqrt_apply(xg[:2], transpose=True)).cpu().numpy()
    Fx = f1.apply(xg[:2]).cpu().numpy()
    assert np.linalg.norm(ssx - Fx) / np.linalg.norm(Fx) <= (1e-11 if prec == "fp64" else 1e-5)
