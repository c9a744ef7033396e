"""The paper's own examples are first-kind equations (Sec. 4, Examples 1
and 2): piecewise-constant collocation on a grid, K_ij = h^d K(x_i - x_j) off
the diagonal and the integral of K over the cell on it.  The library takes
the diagonal and the weight through rss_kernel; nothing else changes.  GPU
against the oracle on the 64^2 grid (eps 1e-6) and the 16^3 grid (eps
1e-3):
  - apply within 10 eps of the oracle's, and the GPU's own apply error
    within 10 eps of the oracle's;
  - solve within the first-order perturbation bound of the two factors'
    difference, 2 cond(A) times the relative difference of their applies;
  - GMRES-IR to 1e-10, checked with the oracle's direct sum.
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


_CACHE = {}


def _reference(name):
    """Oracle factor, dense condition number and reference vectors."""
    if name not in _CACHE:
        w = inputs.workload(name)
        pts, kind, eps = w["pts"], w["kind"], w["eps"]
        A = oracle.dense_matrix(pts, kind, diag=w["diag"], w=w["weight"])
        of = oracle.Factor(oracle.Tree(pts, w["leaf"]), kind, eps, diag=w["diag"], w=w["weight"])
        x = inputs.rhs(3, len(pts), 2)
        Ax = (A @ x.T).T
        _CACHE[name] = dict(w=w, cond=np.linalg.cond(A), of=of, x=x, Ax=Ax, Fo=of.apply(x), So=of.solve(Ax))
    return _CACHE[name]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["laplace2d_grid64_first_kind", "laplace3d_grid16_first_kind"])
def test_first_kind_matches_oracle(pkg, name, prec):
    R = _reference(name)
    w = R["w"]
    eps = w["eps"]
    f = pkg.Factorization(_cuda(w["pts"]), w["kind"], eps, leaf=w["leaf"],
                          prec=pkg.FP64 if prec == "fp64" else pkg.MIXED, diag=w["diag"], weight=w["weight"])
    Fg = f.apply(_cuda(R["x"])).cpu().numpy()
    d = np.linalg.norm(Fg - R["Fo"]) / np.linalg.norm(R["Fo"])
    assert d <= 10 * eps, d
    ea_g = np.linalg.norm(R["Ax"] - Fg) / np.linalg.norm(R["Ax"])
    ea_o = np.linalg.norm(R["Ax"] - R["Fo"]) / np.linalg.norm(R["Ax"])
    assert ea_g <= ea_o + 10 * eps
    Sg = f.solve(_cuda(R["Ax"])).cpu().numpy()
    ds = np.linalg.norm(Sg - R["So"]) / np.linalg.norm(R["So"])
    assert ds <= 2 * R["cond"] * max(d, 1e-15), (ds, R["cond"], d)


@pytest.mark.parametrize("name", ["laplace2d_grid64_first_kind", "laplace3d_grid16_first_kind"])
def test_first_kind_refined_solve(pkg, name):
    """The FP32 factor preconditions GMRES-IR to 1e-10 on the first-kind
    matrix too (the paper runs CG with its factor instead, Sec. 4)."""
    w = inputs.workload(name)
    pts = w["pts"]
    f = pkg.Factorization(_cuda(pts), w["kind"], w["eps"], leaf=w["leaf"], prec=pkg.MIXED, diag=w["diag"],
                          weight=w["weight"])
    b = inputs.rhs(9, len(pts), 2)
    x, iters, rel = f.solve_refined(_cuda(b), tol=1e-10, maxit=20)
    assert rel <= 1e-10
    r = b - oracle.matvec(pts, w["kind"], x.cpu().numpy(), diag=w["diag"], w=w["weight"])
    assert np.linalg.norm(r) <= 2e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["laplace2d_grid64_first_kind", "laplace3d_grid16_first_kind", "laplace2d_grid64"])
def test_cg_with_the_factor(pkg, name, prec):
    """Conjugate gradients preconditioned with the factor (the paper's
    iterative solver, Sec. 4) reach 1e-10 on the first- and second-kind
    matrices, checked with the oracle's direct sum; the paper reports a
    handful of iterations (Tables 2 and 4: 2-7), and a factor accurate to
    eps needs about log(1e-10) / log(eps) of them."""
    w = inputs.workload(name)
    pts = w["pts"]
    mat = {k: w[k] for k in ("diag", "weight") if k in w}
    f = pkg.Factorization(_cuda(pts), w["kind"], w["eps"], leaf=w["leaf"],
                          prec=pkg.FP64 if prec == "fp64" else pkg.MIXED, **mat)
    b = inputs.rhs(21, len(pts), 3)
    x, iters, rel = f.solve_cg(_cuda(b), tol=1e-10, maxit=40)
    assert rel <= 1e-10 and iters <= 12, (iters, rel)
    r = b - oracle.matvec(pts, w["kind"], x.cpu().numpy(), diag=mat.get("diag", 1.0), w=mat.get("weight"))
    assert np.linalg.norm(r) <= 2e-10 * np.linalg.norm(b)
