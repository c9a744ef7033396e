"""Rank-proposal network on the GPU: forward, gradient and Adam step of the
library's CUDA kernels against the FP64 reference (oracle/mlp.py), the box
features against closed forms on a uniform grid, and what the trained
network gains: the same factor with smaller storage reservations, and a
mispredicting network costing a retry, never accuracy."""
import numpy as np
import pytest

from oracle import mlp as omlp
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


def _theta(seed=3):
    th = omlp.init_params(inputs.uniform(seed, omlp.NPARAM))
    th += 0.05 * (inputs.uniform(seed + 100, omlp.NPARAM) - 0.5)  # non-zero biases too
    return th.astype(np.float32)


def _data(seed, n):
    X = inputs.uniform(seed, n * 16).reshape(n, 16).astype(np.float32)
    X[:, 13:] = 0.0
    y = inputs.uniform(seed + 1, n).astype(np.float32)
    return X, y


def test_forward_matches_oracle(pkg):
    th = _theta()
    m = pkg.Mlp(th)
    X, _ = _data(7, 1000)  # 31 full tiles of 32 and a ragged one
    got = m.predict(X).cpu().numpy()
    want, _ = omlp.forward(omlp.bf16_round(th), X)
    np.testing.assert_allclose(got, want, rtol=0, atol=2e-5 * max(1.0, np.abs(want).max()))


def test_gradient_matches_oracle(pkg):
    th = _theta(5)
    m = pkg.Mlp(th)
    X, y = _data(9, 5000)  # several CTAs' partial sums
    g, loss = m.grad(X, y)
    g = g.cpu().numpy().astype(np.float64)
    tb = omlp.bf16_round(th)
    want = omlp.backward(tb, X, y)
    assert loss == pytest.approx(omlp.loss(tb, X, y), rel=1e-5)
    assert np.linalg.norm(g - want) <= 1e-3 * np.linalg.norm(want)
    big = np.abs(want) > 1e-2 * np.abs(want).max()
    np.testing.assert_allclose(g[big], want[big], rtol=1e-3)


def test_adam_steps_match_oracle(pkg):
    th = _theta(8)
    X, y = _data(13, 300)
    m = pkg.Mlp(th)
    lr = 1e-3
    # reference: Adam on the gradients the GPU computes at each step's weights
    ref = th.astype(np.float64)
    mm = np.zeros_like(ref)
    vv = np.zeros_like(ref)
    for t in (1, 2, 3):
        g, _ = m.grad(X, y)
        ref, mm, vv = omlp.adam_step(ref, mm, vv, g.cpu().numpy().astype(np.float64), t, lr)
        m.train(X, y, iters=1, lr=lr)
        np.testing.assert_allclose(m.params(), ref, rtol=0, atol=2e-6)


def test_training_reduces_loss(pkg):
    X, _ = _data(21, 2000)
    # a smooth target the network can fit
    y = (0.3 + 0.4 * np.tanh(2.0 * X[:, 3] - X[:, 5]) * X[:, 8]).astype(np.float32)
    m = pkg.Mlp(seed=1)
    l0 = omlp.loss(omlp.bf16_round(m.params()), X, y)
    l1 = m.train(X, y, iters=400, lr=3e-3)
    l2 = omlp.loss(omlp.bf16_round(m.params()), X, y)
    assert l1 < 0.2 * l0 and l2 < 0.2 * l0


def test_seeded_init_matches_definition(pkg):
    """rss_mlp_create(NULL, seed): Glorot-uniform from SplitMix64(seed)."""
    m = pkg.Mlp(seed=42)
    want = omlp.init_params(inputs.uniform(42, omlp.NPARAM))
    np.testing.assert_allclose(m.params(), want, rtol=0, atol=1e-7)


def test_features_on_uniform_grid(pkg):
    """Leaf boxes of the 64 x 64 grid hold 64 points each; an interior leaf
    box has 8 near and 16 ring cells of 64 points (Sec. 3.2)."""
    pts = inputs.grid_points(64, 2)
    f = pkg.Factorization(torch.from_numpy(pts).cuda(), 0, 1e-6, leaf=64, prec=pkg.MIXED)
    st = f.stats()
    feat, rank = f.box_features()
    assert feat.shape == (st["nbox"], 16)
    np.testing.assert_array_equal(rank, st["k"])
    leaf = st["depth"] == 3
    interior = leaf & (feat[:, 6] == 1.0) & (feat[:, 7] == 1.0)
    assert interior.sum() == 16  # leaf coordinates 2..5 in both directions of the 8 x 8 leaf grid
    fi = feat[interior][0]
    np.testing.assert_allclose(fi[:13], [0, 0, 0.6, np.log2(65) / 10, np.log2(1 + 8 * 64) / 10,
                                         np.log2(1 + 16 * 64) / 10, 1, 1, 1, 1, 0.3, np.log2(65) / 10, 0.5],
                               rtol=1e-6)
    assert not feat[:, 13:].any()


def _training_set(pkg):
    """Features and rank fractions from factorizations of small workloads
    (2D grids and random points at several tolerances, a 3D grid)."""
    Xs, ys = [], []
    cases = [(inputs.grid_points(64, 2), 0, e) for e in (1e-3, 1e-6, 1e-9)] + \
            [(inputs.grid_points(128, 2), 0, 1e-6), (inputs.random_points(31, 6000, 2), 0, 1e-6),
             (inputs.random_points(32, 3000, 2), 0, 1e-4), (inputs.grid_points(16, 3), 1, 1e-3),
             (inputs.grid_points(16, 3), 1, 1e-6)]
    for pts, kind, eps in cases:
        f = pkg.Factorization(torch.from_numpy(pts).cuda(), kind, eps, leaf=64, prec=pkg.MIXED)
        feat, rank = f.box_features()
        st = f.stats()
        keep = st["b"] > 0
        Xs.append(feat[keep])
        ys.append((rank[keep] / st["b"][keep]).astype(np.float32))
    return np.concatenate(Xs), np.concatenate(ys)


def test_proposal_presizes_storage_same_factor(pkg):
    """The trained network reserves much less storage than the full-size
    reservation and the factor is bit-identical (the QR decides every rank)."""
    X, y = _training_set(pkg)
    m = pkg.Mlp(seed=7)
    loss = m.train(X, y, iters=3000, lr=3e-3)
    assert loss < 5e-3, loss
    for pts, eps in [(inputs.grid_points(256, 2), 1e-6), (inputs.random_points(77, 20000, 2), 1e-6)]:
        P = torch.from_numpy(pts).cuda()
        f0 = pkg.Factorization(P, 0, eps, leaf=64, prec=pkg.MIXED)
        f1 = pkg.Factorization(P, 0, eps, leaf=64, prec=pkg.MIXED, mlp=m)
        s0, s1 = f0.stats(), f1.stats()
        assert s1["proposal"] == 1 and s1["retried"] == 0 and s0["proposal"] == 0
        np.testing.assert_array_equal(s0["k"], s1["k"])
        assert s0["used_bytes"] == s1["used_bytes"]
        assert s1["reserved_bytes"] >= s1["used_bytes"]
        assert s1["reserved_bytes"] <= 0.7 * s0["reserved_bytes"], (s1["reserved_bytes"], s0["reserved_bytes"])
        x = torch.from_numpy(inputs.rhs(3, pts.shape[0], 2)).cuda()
        assert torch.equal(f0.apply(x), f1.apply(x))
        assert torch.equal(f0.solve(x), f1.solve(x))


def test_mispredicting_proposal_retries_same_factor(pkg):
    """A network predicting k = b for every box reserves almost nothing; the
    overflow space runs out, the factorization is redone with full-size
    reservations and the result is the same."""
    p = np.zeros(omlp.NPARAM, dtype=np.float32)
    p[-1] = 1.0  # output = b4 = 1: every column a skeleton
    m = pkg.Mlp(p)
    pts = torch.from_numpy(inputs.grid_points(128, 2)).cuda()
    f0 = pkg.Factorization(pts, 0, 1e-6, leaf=64, prec=pkg.MIXED)
    f1 = pkg.Factorization(pts, 0, 1e-6, leaf=64, prec=pkg.MIXED, mlp=m)
    s1 = f1.stats()
    assert s1["retried"] == 1 and s1["proposal"] == 0
    x = torch.from_numpy(inputs.rhs(4, pts.shape[0], 1)).cuda()
    assert torch.equal(f0.solve(x), f1.solve(x))


def test_underpredicting_proposal_uses_overflow(pkg):
    """Constant proposals a little above the true skeleton fraction leave
    some boxes short of their reservation: those take overflow space (or,
    when it runs out, the factorization is redone); the factor is the same."""
    pts = torch.from_numpy(inputs.grid_points(128, 2)).cuda()
    f0 = pkg.Factorization(pts, 0, 1e-6, leaf=64, prec=pkg.MIXED)
    s0 = f0.stats()
    x = torch.from_numpy(inputs.rhs(5, pts.shape[0], 1)).cuda()
    want = f0.solve(x)
    frac = float(np.median(s0["k"] / np.maximum(s0["b"], 1)))
    used_overflow = False
    for c in np.arange(0.08, 0.26, 0.01):
        p = np.zeros(omlp.NPARAM, dtype=np.float32)
        p[-1] = frac + c
        f1 = pkg.Factorization(pts, 0, 1e-6, leaf=64, prec=pkg.MIXED, mlp=pkg.Mlp(p))
        s1 = f1.stats()
        assert torch.equal(f1.solve(x), want)
        if s1["retried"]:
            continue
        r = s1["b"] - s1["k"]
        short = (r > s1["rres"]) | (s1["nj"] * r > s1["njres"] * s1["rres"])
        assert (s1["overflow_bytes"] > 0) == bool(short.any())
        used_overflow |= bool(short.any())
        if used_overflow:
            break
    assert used_overflow
