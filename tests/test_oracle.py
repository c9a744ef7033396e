"""Pins for the CPU oracle: each test checks the oracle against something
other than itself (published test vectors, LAPACK through scipy, brute force,
closed forms, exactness limits and the paper's theorems)."""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_1609_08130_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------------------
# inputs
# ---------------------------------------------------------------------------

def test_splitmix64_vectors():
    for row in _golden("splitmix64.txt"):
        seed = int(row[0])
        want = [int(v, 16) for v in row[1:]]
        got = [int(v) for v in inputs.splitmix64(seed, len(want))]
        assert got == want


def test_normal_moments():
    z = inputs.normal(7, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.01
    u = inputs.uniform(3, 100000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01


def test_grid_points_are_cell_centres():
    p = inputs.grid_points(4, 2)
    assert p.shape == (16, 2)
    assert np.allclose(p[:4, 0], [0.125, 0.375, 0.625, 0.875]) and np.allclose(p[:4, 1], 0.125)
    p3 = inputs.grid_points(4, 3)
    assert p3.shape == (64, 3) and np.allclose(p3[16], [0.125, 0.125, 0.375])


# ---------------------------------------------------------------------------
# kernel entries
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim,kind", [(2, 0), (3, 1)])
def test_kernel_entries_match_libm(dim, kind):
    pts = inputs.random_points(11, 40, dim)
    A = oracle.dense_matrix(pts, kind, diag=1.0, w=0.5)
    for i, j in [(0, 1), (3, 17), (39, 2), (5, 5)]:
        if i == j:
            want = 1.0
        else:
            r = math.dist(pts[i], pts[j])
            want = 0.5 * (-math.log(r) / (2 * math.pi) if kind == 0 else 1.0 / (4 * math.pi * r))
        assert A[i, j] == pytest.approx(want, rel=1e-15, abs=0)


# ---------------------------------------------------------------------------
# tree: properties that fix the tree and the DOF order uniquely
# ---------------------------------------------------------------------------

def _check_tree(pts, leaf):
    tr = oracle.Tree(pts, leaf)
    perm = tr.perm()
    n, dim = pts.shape
    assert sorted(perm.tolist()) == list(range(n))
    nd = tr.nodes()
    x = pts[perm]
    children = {i: [] for i in range(tr.nnode)}
    for i in range(1, tr.nnode):
        children[int(nd["parent"][i])].append(i)
    for i in range(tr.nnode):
        t = int(nd["depth"][i])
        s, c = int(nd["start"][i]), int(nd["count"][i])
        lo = nd["coord"][i, :dim] * 2.0 ** -t
        hi = lo + 2.0 ** -t
        seg = x[s:s + c]
        assert np.all(seg >= lo) and np.all((seg < hi) | (hi >= 1.0))
        ch = children[i]
        if c > leaf and t < 20:
            assert ch, "over-full node must be split"
            # children partition the range in ascending child index
            assert int(nd["start"][ch[0]]) == s
            idx = [sum(((int(nd["coord"][q, d]) & 1) << d) for d in range(dim)) for q in ch]
            assert idx == sorted(idx)
            end = s
            for q in ch:
                assert int(nd["start"][q]) == end
                end += int(nd["count"][q])
            assert end == s + c
        else:
            assert not ch
            # stable: original indices ascending inside a leaf
            assert np.all(np.diff(perm[s:s + c]) > 0)
    return tr, nd


@pytest.mark.parametrize("case", ["grid2d", "grid3d", "random2d"])
def test_tree_structure(case):
    if case == "grid2d":
        pts, leaf = inputs.grid_points(32, 2), 64
    elif case == "grid3d":
        pts, leaf = inputs.grid_points(16, 3), 64
    else:
        pts, leaf = inputs.random_points(5, 3000, 2), 64
    tr, nd = _check_tree(pts, leaf)
    if case == "grid2d":
        assert tr.maxdepth == 2 and (nd["depth"] == 2).sum() == 16
    if case == "grid3d":
        assert tr.maxdepth == 2 and (nd["depth"] == 2).sum() == 64


def test_box_order_and_lists_brute_force():
    """Level order is colour-major (3^d colours) with same-colour boxes >= 3
    apart; near / ring cell lists equal a brute-force pairwise classification
    (Fig. 2); interior counts equal the closed forms."""
    golden = {int(r[0]): (int(r[1]), int(r[2])) for r in _golden("neighbor_counts.txt")}
    for pts, dim in [(inputs.grid_points(64, 2), 2), (inputs.grid_points(16, 3), 3),
                     (inputs.random_points(9, 5000, 2), 2)]:
        tr = oracle.Tree(pts, 64)
        nd = tr.nodes()
        x = pts[tr.perm()]
        for t in range(tr.maxdepth, 1, -1):
            boxes = tr.level_boxes(t)
            assert sorted(boxes.tolist()) == sorted(np.nonzero(nd["depth"] == t)[0].tolist())
            cols = [sum((int(nd["coord"][b, d]) % 3) * 3 ** d for d in range(dim)) for b in boxes]
            assert cols == sorted(cols)
            cells = np.minimum(np.floor(x * 2 ** t).astype(np.int64), 2 ** t - 1)
            for q, b in enumerate(boxes):
                bc = nd["coord"][b, :dim]
                for q2 in range(q + 1, len(boxes)):
                    if cols[q2] != cols[q]:
                        break
                    assert np.abs(nd["coord"][boxes[q2], :dim] - bc).max() >= 3
                delta = cells - bc
                dist = np.abs(delta).max(axis=1)
                codes = ((delta + 2) * (5 ** np.arange(dim))).sum(axis=1)
                want_near = sorted(set(codes[dist == 1].tolist()))
                want_ring = sorted(set(codes[dist == 2].tolist()))
                near, ring = tr.box_lists(int(b))
                assert near.tolist() == want_near and ring.tolist() == want_ring
                if np.all(bc >= 2) and np.all(bc <= 2 ** t - 3) and dim in golden and pts.shape[0] in (4096,):
                    assert (len(near), len(ring)) == golden[dim]


# ---------------------------------------------------------------------------
# dense building blocks against LAPACK
# ---------------------------------------------------------------------------

def test_cpqr_matches_lapack_pivots():
    rng = np.random.default_rng(0)
    for m, n in [(50, 20), (200, 64), (30, 40)]:
        M = rng.standard_normal((m, n)) @ np.diag(np.logspace(0, -8, n)) @ rng.standard_normal((n, n))
        k, perm, T, rd = oracle.cpqr_id(M, 0.0)
        _, R, P = sla.qr(M, pivoting=True, mode="economic")
        kk = min(m, n)
        # greedy pivoting: same first pivots as LAPACK's dgeqp3 on generic data
        assert perm[:10].tolist() == P[:10].tolist()
        assert np.allclose(rd[:kk], np.abs(np.diag(R))[:kk], rtol=1e-6, atol=1e-12 * rd[0])


def test_cpqr_id_bound_and_rank():
    rng = np.random.default_rng(1)
    # exactly rank 5
    M = rng.standard_normal((80, 5)) @ rng.standard_normal((5, 30))
    k, perm, T, rd = oracle.cpqr_id(M, 1e-10)
    assert k == 5
    assert np.allclose(M[:, perm[k:]], M[:, perm[:k]] @ T, atol=1e-10 * np.abs(M).max())
    # decaying spectrum: ||M_R - M_S T||_2 <= sqrt(n-k) eps |R_11| (greedy pivoting)
    U, _ = np.linalg.qr(rng.standard_normal((300, 60)))
    V, _ = np.linalg.qr(rng.standard_normal((60, 60)))
    M = U @ np.diag(np.logspace(0, -14, 60)) @ V.T
    for eps in [1e-3, 1e-6, 1e-9]:
        k, perm, T, rd = oracle.cpqr_id(M, eps)
        err = np.linalg.norm(M[:, perm[k:]] - M[:, perm[:k]] @ T, 2)
        assert err <= math.sqrt(60 - k) * eps * rd[0] * 1.0001
        assert rd[k - 1] > eps * rd[0] and (k == 60 or rd[k] <= eps * rd[0])
    # zero matrix: rank 0
    k, perm, T, rd = oracle.cpqr_id(np.zeros((10, 4)), 1e-6)
    assert k == 0


def test_lu_matches_lapack():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((37, 37))
    LU, piv, info = oracle.lu(A)
    lu_ref, piv_ref = sla.lu_factor(A)
    perm_ref = np.arange(37)
    for i, p in enumerate(piv_ref):
        perm_ref[[i, p]] = perm_ref[[p, i]]
    assert info == 0
    assert piv.tolist() == perm_ref.tolist()
    assert np.allclose(LU, lu_ref, rtol=1e-12, atol=1e-12)
    S = np.ones((3, 3))
    assert oracle.lu(S)[2] != 0


def test_dense_solve_backward_error():
    pts = inputs.grid_points(24, 2)
    A = oracle.dense_matrix(pts, 0)
    b = inputs.normal(1, len(pts))
    x = oracle.dense_solve(A, b)
    n = len(pts)
    assert np.linalg.norm(A @ x - b) / (np.linalg.norm(A, 2) * np.linalg.norm(x)) <= 10 * n * 1.1e-16
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-12, atol=1e-12)


def test_matvec_matches_dense():
    pts = inputs.random_points(4, 300, 3)
    x = inputs.normal(2, 300)
    A = oracle.dense_matrix(pts, 1)
    assert np.allclose(oracle.matvec(pts, 1, x), A @ x, rtol=1e-13, atol=1e-13)
    rows = np.array([5, 0, 299])
    assert np.allclose(oracle.matvec(pts, 1, x, rows=rows), (A @ x)[rows], rtol=1e-13)


# ---------------------------------------------------------------------------
# RS-S factorization (Algorithm 1)
# ---------------------------------------------------------------------------

def _problem(case):
    if case == "grid2d":
        return inputs.grid_points(64, 2), 0
    if case == "grid3d":
        return inputs.grid_points(16, 3), 1
    if case == "random2d":
        return inputs.random_points(21, 3000, 2), 0
    raise KeyError(case)


@pytest.mark.parametrize("case", ["grid2d", "grid3d", "random2d"])
def test_factor_exact_limit(case):
    """eps -> 0: every step is exact block elimination (Sec. 2.1), so F = A
    and F^{-1} b equals the dense solve (Eq. 3.10, 3.11)."""
    pts, kind = _problem(case)
    n = len(pts)
    tr = oracle.Tree(pts, 64)
    f = oracle.Factor(tr, kind, 1e-14)
    assert f.info == 0
    A = oracle.dense_matrix(pts, kind)
    x = inputs.normal(3, n)
    assert np.linalg.norm(f.apply(x) - A @ x) / np.linalg.norm(A @ x) < 1e-12
    b = inputs.normal(4, n)
    xs = np.linalg.solve(A, b)
    assert np.linalg.norm(f.solve(b) - xs) / np.linalg.norm(xs) < 1e-11
    sign, ld = np.linalg.slogdet(A)
    assert abs(f.logdet() - ld) < 1e-9 * max(1.0, abs(ld))


def test_factor_without_compression_is_exact():
    """eps = 0 keeps every column as skeleton (k = |B|): F = A."""
    pts, kind = _problem("grid2d")
    tr = oracle.Tree(pts[::4].copy(), 64)
    f = oracle.Factor(tr, kind, 0.0)
    for b in f.boxes():
        assert b["r"] == 0 or b["k"] == b["b"]
    p = pts[::4]
    A = oracle.dense_matrix(p, kind)
    x = inputs.normal(5, len(p))
    assert np.allclose(f.apply(x), A @ x, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("case", ["grid2d", "grid3d", "random2d"])
def test_factor_invariants(case):
    """Theorem 3.1 (B-P interactions untouched), Corollary 3.2 (far field
    original at each level start) and the final block-diagonal form of D
    (Sec. 3.3.3), all checked on the whole matrix, bit for bit."""
    pts, kind = _problem(case)
    if len(pts) > 2000:
        pts = pts[: len(pts) // 2] if case != "grid2d" else inputs.grid_points(32, 2)
    tr = oracle.Tree(pts, 16 if case == "grid2d" else 32)
    f = oracle.Factor(tr, kind, 1e-6, check=True)
    assert f.nbox > 0 and f.violations == 0


@pytest.mark.parametrize("case,eps", [("grid2d", 1e-6), ("grid2d", 1e-3), ("grid3d", 1e-3),
                                      ("random2d", 1e-6)])
def test_factor_accuracy_band(case, eps):
    """The paper's tables show e_a ~ O(eps) (Tables 2 and 4); with the
    second-kind scaling here the apply error must stay below eps."""
    pts, kind = _problem(case)
    n = len(pts)
    tr = oracle.Tree(pts, 64)
    f = oracle.Factor(tr, kind, eps)
    x = inputs.normal(6, n)
    Ax = oracle.matvec(pts, kind, x)
    ea = np.linalg.norm(f.apply(x) - Ax) / np.linalg.norm(Ax)
    assert ea < eps
    xs = f.solve(Ax)
    assert np.linalg.norm(xs - x) / np.linalg.norm(x) < 10 * eps
    # some compression actually happened
    assert sum(b["r"] for b in f.boxes()) > n // 4


def test_apply_and_solve_are_inverse():
    """F^{-1} (F x) = x independently of eps (the factors are exact inverses
    of one another, Eq. 3.10 vs 3.11)."""
    pts, kind = _problem("random2d")
    tr = oracle.Tree(pts, 64)
    f = oracle.Factor(tr, kind, 1e-3)
    x = inputs.normal(8, len(pts))
    assert np.linalg.norm(f.solve(f.apply(x)) - x) / np.linalg.norm(x) < 1e-12


def test_symmetric_factors():
    """K symmetric => V_i = W_i^T (Sec. 3.3.3): E = G^T up to rounding."""
    pts, kind = _problem("grid2d")
    tr = oracle.Tree(pts, 64)
    f = oracle.Factor(tr, kind, 1e-6)
    for i in range(0, f.nbox, 7):
        d = f.box_data(i)
        if d["r"]:
            assert np.allclose(d["E"], d["G"].T, rtol=1e-9, atol=1e-12 * np.abs(d["E"]).max())


def test_proxy_surface_is_needed():
    """Planted mistake in the oracle's inputs: with only 4 proxy points the
    discretised Green's identity (Eq. 3.5, 3.6) cannot stand in for the far
    field outside the proxy surface, so the IDs stop compressing the true far
    field and the apply error must rise well above the one with the paper's
    64 points (Sec. 4, Example 1)."""
    pts, kind = _problem("grid2d")
    tr = oracle.Tree(pts, 64)
    x = inputs.normal(9, len(pts))
    Ax = oracle.matvec(pts, kind, x)
    good = oracle.Factor(tr, kind, 1e-9, nproxy=64)
    bad = oracle.Factor(tr, kind, 1e-9, nproxy=4)
    eg = np.linalg.norm(good.apply(x) - Ax) / np.linalg.norm(Ax)
    eb = np.linalg.norm(bad.apply(x) - Ax) / np.linalg.norm(Ax)
    assert eb > 10 * eg


# Per-box checks of the ID inside a factorization (Definition 2.1, Sec. 3.2)
_ID_CHECK_PROBLEMS = [  # (points, kernel, eps, leaf)
    ("grid2d", lambda: inputs.grid_points(64, 2), 0, 1e-6, 64),
    ("random2d", lambda: inputs.random_points(5, 3000, 2), 0, 1e-6, 32),
    ("grid3d", lambda: inputs.grid_points(12, 3), 1, 1e-3, 8),
]


@pytest.fixture
def no_plant():
    oracle.plant_mistake(0)
    yield
    oracle.plant_mistake(0)


@pytest.mark.parametrize("name,make,kind,eps,leaf", _ID_CHECK_PROBLEMS, ids=[p[0] for p in _ID_CHECK_PROBLEMS])
def test_every_box_id_meets_its_bounds(no_plant, name, make, kind, eps, leaf):
    """For every box of a factorization, on the ID matrix the box actually
    formed and the current matrix:
      - the column-pivoted QR bound ||M_R - M_S T||_F <= sqrt(r) eps |R_11|
        (each trailing column of R is no longer than the pivot that stopped
        the reduction, which is at most eps |R_11|);
      - proxy validity: the same T compresses the box's whole far field
        (ring and beyond, both halves) to eps, ||X_R - X_S T||_2 <= eps ||X||_2
        (Sec. 3.2: the proxy rows stand in for everything outside the ring).
    The Theorem 3.1 / Corollary 3.2 counts stay zero too."""
    f = oracle.Factor(oracle.Tree(make(), leaf), kind, eps, check=True)
    assert f.nbox > 0
    assert f.violations == 0
    assert f.id_violations == 0, f.id_worst
    assert f.proxy_violations == 0, f.proxy_worst
    assert 0.0 < f.id_worst <= 1.0 and 0.0 < f.proxy_worst <= 1.0


def test_id_checks_catch_planted_mistakes(no_plant):
    """Planted mistakes in the oracle that make some IDs invalid must be
    counted by the per-box checks:
      - the ID matrix built from only half of the ring (cells at x offset
        >= 0): sources left out sit partly inside the proxy surface, so
        nothing in M stands for them and the far field is not compressed;
      - pivoting dropped (columns taken in order): the truncation at
        |R_jj| <= eps |R_11| no longer bounds the trailing columns;
      - 4 proxy points instead of 64: too few to stand in for the far field."""
    pts = inputs.random_points(5, 3000, 2)
    tr = oracle.Tree(pts, 32)
    oracle.plant_mistake(2)
    f = oracle.Factor(tr, 0, 1e-6, check=True)
    assert f.proxy_violations > 0 and f.proxy_worst > 1.0
    oracle.plant_mistake(4)
    f = oracle.Factor(oracle.Tree(inputs.grid_points(12, 3), 8), 1, 1e-3, check=True)
    assert f.id_violations > 0 and f.id_worst > 1.0
    oracle.plant_mistake(0)
    f = oracle.Factor(oracle.Tree(inputs.grid_points(64, 2), 64), 0, 1e-6, check=True, nproxy=4)
    assert f.proxy_violations > 0 and f.id_violations == 0


def test_shifted_or_small_proxy_surfaces_stay_valid(no_plant):
    """Not every change of the proxy surface is a mistake: a circle centred one
    box side off still holds the box, and one of a quarter of the radius
    still separates the box from the far field (only more skeletons are kept);
    together with the explicit ring rows both still give IDs that compress
    the whole far field to eps.  The checks measure validity, not the surface."""
    pts = inputs.grid_points(64, 2)
    tr = oracle.Tree(pts, 64)
    ranks = {}
    for plant in (0, 1, 3):
        oracle.plant_mistake(plant)
        f = oracle.Factor(tr, 0, 1e-6, check=True)
        assert f.id_violations == 0 and f.proxy_violations == 0
        ranks[plant] = sum(b["k"] for b in f.boxes())
    assert ranks[3] > ranks[0]


def test_degenerate_sizes():
    # fewer points than one leaf: no skeletonization, F = dense LU
    pts = inputs.random_points(2, 50, 2)
    tr = oracle.Tree(pts, 64)
    f = oracle.Factor(tr, 0, 1e-6)
    assert f.nbox == 0 and f.ntop == 50
    A = oracle.dense_matrix(pts, 0)
    b = inputs.normal(1, 50)
    assert np.allclose(f.solve(b), np.linalg.solve(A, b), rtol=1e-12)
    # empty problem
    tr0 = oracle.Tree(np.zeros((0, 2)), 64)
    f0 = oracle.Factor(tr0, 0, 1e-6, w=1.0)
    assert f0.ntop == 0


def test_logdet_is_that_of_the_factor():
    """At eps > 0 the oracle's log det (sum of log |U_jj| over the boxes' and
    the top block's LU) is log |det F| of the operator it applies: F formed
    column by column from apply() on the identity, then a dense LU.  A
    missing box, a wrong diagonal or a dropped top block moves it."""
    pts = inputs.grid_points(16, 2)
    n = len(pts)
    f = oracle.Factor(oracle.Tree(pts, 16), 0, 1e-4)
    Fd = np.stack([f.apply(np.eye(n)[:, c].copy()) for c in range(n)], axis=1)
    sign, ld = np.linalg.slogdet(Fd)
    assert sign != 0
    assert abs(f.logdet() - ld) <= 1e-10 * max(1.0, abs(ld)), (f.logdet(), ld)
    # the compression is real: F is not A, and neither is its determinant
    _, lda = np.linalg.slogdet(oracle.dense_matrix(pts, 0))
    assert np.linalg.norm(Fd - oracle.dense_matrix(pts, 0)) > 1e-9
    assert abs(lda - ld) < 1e-2


# ---------------------------------------------------------------------------
# first-kind workloads as in Sec. 4 (Examples 1 and 2)
# ---------------------------------------------------------------------------

def test_cell_self_integral_closed_forms():
    """The closed forms of the cell integrals against an independent route:
    cutting the unit square into two triangles (the unit cube into three
    pyramids) about the singular corner leaves smooth integrals, done by
    adaptive quadrature.  Square: int log(x^2+y^2) = -1 + int_0^1 log(1+s^2) ds.
    Cube: int 1/|z| = (3/2) int_[0,1]^2 (1+s^2+t^2)^(-1/2) ds dt."""
    from scipy import integrate
    sq = -1.0 + integrate.quad(lambda s: math.log1p(s * s), 0.0, 1.0, epsabs=1e-14, epsrel=1e-14)[0]
    cube = 1.5 * integrate.dblquad(lambda t, s: 1.0 / math.sqrt(1.0 + s * s + t * t), 0.0, 1.0, 0.0, 1.0,
                                   epsabs=1e-13, epsrel=1e-13)[0]
    for h in (1.0 / 64, 1.0 / 512, 0.3):
        a = 0.5 * h
        # [-a,a]^2 = four copies of [0,a]^2; log|z| = log(z^2)/2; scale by a^2
        want2 = -(4.0 * a * a * 0.5 * (sq + 2.0 * math.log(a))) / (2.0 * math.pi)
        assert inputs.cell_self_integral(0, h) == pytest.approx(want2, rel=1e-12)
        want3 = 8.0 * a * a * cube / (4.0 * math.pi)
        assert inputs.cell_self_integral(1, h) == pytest.approx(want3, rel=1e-12)


def _first_kind(side, dim):
    pts = inputs.grid_points(side, dim)
    h = 1.0 / side
    kind = 0 if dim == 2 else 1
    return pts, kind, inputs.cell_self_integral(kind, h), h ** dim


def test_first_kind_exact_limit():
    """eps -> 0 on the first-kind matrix (diagonal = cell integral, off the
    diagonal h^d K): exact block elimination, F = A and the dense solve."""
    pts, kind, d, w = _first_kind(24, 2)
    n = len(pts)
    A = oracle.dense_matrix(pts, kind, diag=d, w=w)
    f = oracle.Factor(oracle.Tree(pts, 64), kind, 1e-14, diag=d, w=w)
    x = inputs.normal(11, n)
    assert np.linalg.norm(f.apply(x) - A @ x) / np.linalg.norm(A @ x) < 1e-12
    b = inputs.normal(12, n)
    xs = np.linalg.solve(A, b)
    assert np.linalg.norm(f.solve(b) - xs) / np.linalg.norm(xs) < 1e-10


@pytest.mark.parametrize("side,dim,eps", [(32, 2, 1e-6), (32, 2, 1e-3), (12, 3, 1e-3)])
def test_first_kind_accuracy(side, dim, eps):
    """The paper's examples are first kind and its tables show e_a = O(eps)
    (Tables 2 and 4): the apply error stays below eps; the solve error obeys
    the first-order perturbation bound ||F^{-1} - A^{-1}|| <= ||A^{-1}|| ||A - F|| ||F^{-1}||,
    i.e. at most 2 cond(A) e_a in relative terms."""
    pts, kind, d, w = _first_kind(side, dim)
    n = len(pts)
    A = oracle.dense_matrix(pts, kind, diag=d, w=w)
    f = oracle.Factor(oracle.Tree(pts, 64 if dim == 2 else 27), kind, eps, diag=d, w=w)
    x = inputs.normal(13, n)
    Ax = A @ x
    ea = np.linalg.norm(f.apply(x) - Ax) / np.linalg.norm(Ax)
    assert ea < eps
    es = np.linalg.norm(f.solve(Ax) - x) / np.linalg.norm(x)
    assert es <= 2.0 * np.linalg.cond(A) * max(ea, 1e-15)
    assert sum(b["r"] for b in f.boxes()) > n // 8  # compression happened


# ---------------------------------------------------------------------------
# RS-WS, the hybrid factorization (Sec. 3.4, Algorithm 2)
# ---------------------------------------------------------------------------

def _stored_entries(f):
    """Entries of T, LU(X_RR), E and G over the boxes, plus the top LU."""
    return sum(b["k"] * b["r"] + b["r"] ** 2 + 2 * b["nj"] * b["r"] for b in f.boxes()) + f.ntop ** 2


@pytest.mark.parametrize("case", ["grid2d", "grid3d_12", "random2d"])
def test_hybrid_exact_limit(case):
    """eps -> 0: weak and strong steps are exact block eliminations, so the
    RS-WS factor reproduces A, its solve the dense solve and its log det
    log |det A|.  (3D: a 12^3 grid with leaves of 27 points, three levels.)"""
    if case == "grid3d_12":
        pts, kind, leaf = inputs.grid_points(12, 3), 1, 27
    else:
        (pts, kind), leaf = _problem(case), 64
    n = len(pts)
    f = oracle.Factor(oracle.Tree(pts, leaf), kind, 1e-14, hybrid=True)
    assert f.info == 0
    A = oracle.dense_matrix(pts, kind)
    x = inputs.normal(3, n)
    assert np.linalg.norm(f.apply(x) - A @ x) / np.linalg.norm(A @ x) < 1e-12
    b = inputs.normal(4, n)
    xs = np.linalg.solve(A, b)
    assert np.linalg.norm(f.solve(b) - xs) / np.linalg.norm(xs) < 1e-11
    _, ld = np.linalg.slogdet(A)
    assert abs(f.logdet() - ld) < 1e-9 * max(1.0, abs(ld))


def test_hybrid_schedule_and_invariants():
    """Algorithm 2's order: at each depth >= 2 a weak pass over every box, then
    a strong pass over the same boxes; a last weak pass at depth 1.  A weak
    step eliminates R against S only (|J| = k).  The weak steps change no
    block outside a box, so Theorem 3.1 / Corollary 3.2 still hold at every
    strong step, and the end result is block diagonal (checked on the whole
    matrix by the oracle's check mode)."""
    pts, kind = _problem("grid2d")
    tr = oracle.Tree(pts, 64)
    f = oracle.Factor(tr, kind, 1e-6, hybrid=True, check=True)
    assert f.violations == 0
    boxes = f.boxes()
    seq = [(b["depth"], b["weak"]) for b in boxes]
    depths = sorted({d for d, _ in seq}, reverse=True)
    assert depths[-1] == 1 and all(w == 1 for d, w in seq if d == 1)
    pos = 0
    for d in depths:
        run = [w for dd, w in seq[pos:] if dd == d]
        nb = len(run)
        pos += nb
        if d >= 2:
            half = nb // 2
            assert run == [1] * half + [0] * half
    for b in boxes:
        if b["weak"]:
            assert b["nj"] == b["k"] and b["nnear"] == 0
    # the strong-only factor of the same tree, for contrast: no weak steps
    g = oracle.Factor(tr, kind, 1e-6)
    assert not any(b["weak"] for b in g.boxes())


@pytest.mark.parametrize("case,eps", [("grid2d", 1e-6), ("grid3d", 1e-3), ("random2d", 1e-6)])
def test_hybrid_accuracy_and_storage(case, eps):
    """RS-WS keeps e_a = O(eps) (the paper's tables) and, as the paper finds
    for its examples, stores less than RS-S: its near-field compression
    shrinks the boxes' J and the top block."""
    pts, kind = _problem(case)
    n = len(pts)
    tr = oracle.Tree(pts, 64)
    A = oracle.dense_matrix(pts, kind)
    x = inputs.normal(6, n)
    Ax = A @ x
    h = oracle.Factor(tr, kind, eps, hybrid=True)
    ea = np.linalg.norm(h.apply(x) - Ax) / np.linalg.norm(Ax)
    assert ea < eps
    assert np.linalg.norm(h.solve(Ax) - x) / np.linalg.norm(x) < 10 * eps
    s = oracle.Factor(tr, kind, eps)
    assert _stored_entries(h) < _stored_entries(s)
    assert h.ntop < s.ntop


# ---------------------------------------------------------------------------
# colour phases run in parallel (Sec. 5)
# ---------------------------------------------------------------------------

def _schedule_problems():
    return [(inputs.grid_points(32, 2), 0, 1e-6, 64), (inputs.random_points(21, 3000, 2), 0, 1e-6, 64),
            (inputs.grid_points(12, 3), 1, 1e-3, 27)]


def test_parallel_phases_with_3d_colours_equal_the_sequential_factor():
    """With 3^d colours the boxes of a phase are >= 3 cells apart, so a phase
    whose boxes all start from the phase-start state (as the GPU runs it)
    gives exactly the factor of one box after another: apply and solve agree
    bit for bit, and the invariants hold."""
    for pts, kind, eps, leaf in _schedule_problems():
        tr = oracle.Tree(pts, leaf)
        x = inputs.normal(17, len(pts))
        f0 = oracle.Factor(tr, kind, eps, schedule=0)
        f1 = oracle.Factor(tr, kind, eps, schedule=1, check=True)
        assert f1.violations == 0
        assert np.array_equal(f0.apply(x), f1.apply(x))
        assert np.array_equal(f0.solve(x), f1.solve(x))


def test_parallel_phases_with_2d_colours():
    """The paper's 2^d colouring (Sec. 5): same-phase boxes can be two cells
    apart, so a box's ring holds DOFs another box of the phase eliminates;
    run in parallel, the factor differs from the one-after-another order but
    is as valid: exact as eps -> 0, e_a < eps, Theorem 3.1 / Corollary 3.2
    and the final block-diagonal form hold."""
    for pts, kind, eps, leaf in _schedule_problems():
        n = len(pts)
        tr = oracle.Tree(pts, leaf)
        A = oracle.dense_matrix(pts, kind)
        x = inputs.normal(18, n)
        Ax = A @ x
        f2 = oracle.Factor(tr, kind, eps, schedule=2, check=True)
        assert f2.violations == 0 and f2.info == 0
        ea = np.linalg.norm(f2.apply(x) - Ax) / np.linalg.norm(Ax)
        assert ea < eps
        assert np.linalg.norm(f2.solve(Ax) - x) / np.linalg.norm(x) < 10 * eps
        f0 = oracle.Factor(tr, kind, eps, schedule=0)
        assert not np.array_equal(f0.apply(x), f2.apply(x))
        fe = oracle.Factor(tr, kind, 1e-14, schedule=2)
        assert np.linalg.norm(fe.apply(x) - Ax) / np.linalg.norm(Ax) < 1e-12


# ---------------------------------------------------------------------------
# generalized square root (the remark after Eq. 3.11)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("hybrid", [False, True])
def test_square_root_reproduces_the_factor(hybrid):
    """K positive definite (second kind here: eigenvalues near 1): with the
    Cholesky blocks of D, F^{1/2} (F^{1/2})^T applies F itself, for RS-S and
    RS-WS alike."""
    for pts, kind, eps, leaf in _schedule_problems():
        f = oracle.Factor(oracle.Tree(pts, leaf), kind, eps, hybrid=hybrid)
        x = inputs.normal(19, len(pts))
        Fx = f.apply(x)
        SSx = f.sqrt_apply(f.sqrt_apply(x, transpose=True))
        assert np.linalg.norm(SSx - Fx) / np.linalg.norm(Fx) < 1e-13


def test_square_root_exact_limit():
    """eps -> 0: F = A, so F^{1/2} is a square root of A up to an orthogonal
    factor (the paper's remark): ||(F^{1/2})^T x||^2 = x^T A x."""
    for pts, kind, _, leaf in _schedule_problems():
        f = oracle.Factor(oracle.Tree(pts, leaf), kind, 1e-14)
        A = oracle.dense_matrix(pts, kind)
        x = inputs.normal(20, len(pts))
        q = float(np.sum(f.sqrt_apply(x, transpose=True) ** 2))
        assert q == pytest.approx(float(x @ A @ x), rel=1e-12)


def test_square_root_needs_a_definite_matrix():
    """A negative definite matrix (diagonal -1, small off-diagonal) has no
    real Cholesky blocks: the square root is refused, not silently wrong."""
    pts = inputs.grid_points(32, 2)
    f = oracle.Factor(oracle.Tree(pts, 64), 0, 1e-6, diag=-1.0)
    with pytest.raises(ValueError):
        f.sqrt_apply(inputs.normal(21, len(pts)))


def test_cholesky_variant():
    """Positive definite K: X_RR and the top block by Cholesky (the paper's
    choice for D in that case) give the factor of the LU variant up to
    rounding and the same log det; G = E^T exactly (one of the two need be
    stored); eps -> 0 is still exact; invariants hold."""
    for pts, kind, eps, leaf in _schedule_problems():
        n = len(pts)
        tr = oracle.Tree(pts, leaf)
        A = oracle.dense_matrix(pts, kind)
        x = inputs.normal(22, n)
        fl = oracle.Factor(tr, kind, eps)
        fc = oracle.Factor(tr, kind, eps, cholesky=True, check=True)
        assert fc.info == 0 and fc.violations == 0
        yl = fl.apply(x)
        assert np.linalg.norm(fc.apply(x) - yl) / np.linalg.norm(yl) < 1e-12
        assert abs(fc.logdet() - fl.logdet()) < 1e-10 * max(1.0, abs(fl.logdet()))
        for i in range(fc.nbox):
            d = fc.box_data(i)
            assert np.array_equal(d["G"], d["E"].T)
        fe = oracle.Factor(tr, kind, 1e-14, cholesky=True)
        Ax = A @ x
        assert np.linalg.norm(fe.apply(x) - Ax) / np.linalg.norm(Ax) < 1e-12
        assert np.linalg.norm(fe.solve(Ax) - x) / np.linalg.norm(x) < 1e-11


def test_cholesky_refuses_an_indefinite_block():
    """A negative definite matrix: the first Cholesky block fails and the
    factor reports it (info != 0) instead of storing garbage."""
    pts = inputs.grid_points(32, 2)
    f = oracle.Factor(oracle.Tree(pts, 64), 0, 1e-6, diag=-1.0, cholesky=True)
    assert f.info != 0
