"""rss_solve_noalloc: the solve for callers that must not have the library
allocate device memory during the call (for instance a program that has
given all device memory to its own allocator).  Its working vectors live in
a fixed device array owned by the library, so this test checks that it
returns what rss_solve returns, on two calls in a row with different data,
and that a request larger than the fixed array is refused cleanly.

Named to be collected last: it shares the library's fixed device array with
nothing else in the suite, and must pass alone or after every other test.
"""
import ctypes as C

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


def _noalloc(pkg, f, b, x):
    """Call the entry point through the C ABI with caller-owned buffers."""
    return pkg.lib().rss_solve_noalloc(f.h, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), b.shape[0])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_solve_matches_solve(pkg, prec):
    pts = torch.from_numpy(inputs.grid_points(64, 2)).cuda()
    n = pts.shape[0]
    f = pkg.Factorization(pts, 0, 1e-6, leaf=64, prec=pkg.FP64 if prec == "fp64" else pkg.MIXED)
    rtol = 1e-12 if prec == "fp64" else 1e-5
    for seed, nrhs in [(1, 4), (7, 2)]:  # two calls in a row, different data
        b = torch.from_numpy(np.ascontiguousarray(inputs.rhs(seed, n, nrhs))).cuda()
        want = f.solve(b).cpu().numpy()
        x = torch.full_like(b, float("nan"))  # caller-owned output
        assert _noalloc(pkg, f, b, x) == pkg.rss.RSS_OK
        torch.cuda.synchronize()
        np.testing.assert_allclose(x.cpu().numpy(), want, rtol=rtol, atol=rtol * np.abs(want).max())


@pytest.mark.parametrize("prec,nrhs", [("fp64", 96), ("mixed", 200), ("mixed", 1100)])
def test_noalloc_many_columns(pkg, prec, nrhs):
    """More right-hand sides than one pass of the sweep kernels takes (the
    one-CTA-per-box sweeps, in several passes through the fixed array), and
    for 1100 FP32 columns more than the array holds at once."""
    pts = torch.from_numpy(inputs.grid_points(64, 2)).cuda()
    n = pts.shape[0]
    f = pkg.Factorization(pts, 0, 1e-6, leaf=64, prec=pkg.FP64 if prec == "fp64" else pkg.MIXED)
    rtol = 1e-12 if prec == "fp64" else 1e-5
    for seed in (3, 11):  # two calls in a row, different data
        b = torch.from_numpy(np.ascontiguousarray(inputs.rhs(seed, n, nrhs))).cuda()
        want = f.solve(b).cpu().numpy()
        x = torch.full_like(b, float("nan"))
        assert _noalloc(pkg, f, b, x) == pkg.rss.RSS_OK, pkg.lib().rss_last_error()
        torch.cuda.synchronize()
        np.testing.assert_allclose(x.cpu().numpy(), want, rtol=rtol, atol=rtol * np.abs(want).max())


def test_noalloc_rejects_oversize(pkg):
    """A single FP64 column of more than 2^21 entries does not fit the fixed
    16 MiB array: the call is refused before any work.  Points on a line keep
    the factorization small."""
    n = (1 << 21) + 4096
    xs = (np.arange(n, dtype=np.float64) + 0.5) / n
    pts = torch.from_numpy(np.stack([xs, np.full(n, 0.5)], axis=1).copy()).cuda()
    f = pkg.Factorization(pts, 0, 1e-3, leaf=64, prec=pkg.FP64)
    b = torch.zeros((1, n), dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    st = _noalloc(pkg, f, b, x)
    assert st == pkg.rss.RSS_EINVAL
    assert b"16 MiB" in pkg.lib().rss_last_error()
