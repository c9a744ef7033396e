"""Python access to the plain FP64 CPU oracle (``rss_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package smoke check
and by the benchmark's CPU-baseline leg.  The product library never imports,
links or runs anything here.

Every routine follows the paper step by step (strong recursive
skeletonization, Algorithm 1, Sec. 3; the hybrid RS-WS, Algorithm 2,
Sec. 3.4); see the header of ``rss_oracle.c`` for the readings taken where
the paper is silent.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rss_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the system C compiler (portable flags only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _setup(_lib)
    return _lib


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_lp = C.POINTER(C.c_int64)


def _setup(L):
    L.orc_tree_build.restype = C.c_void_p
    L.orc_tree_build.argtypes = [_dp, C.c_int64, C.c_int, C.c_int]
    L.orc_tree_free.argtypes = [C.c_void_p]
    L.orc_tree_info.restype = C.c_int64
    L.orc_tree_info.argtypes = [C.c_void_p, C.c_int]
    L.orc_tree_perm.argtypes = [C.c_void_p, _lp]
    L.orc_tree_nodes.argtypes = [C.c_void_p, _ip, _ip, _ip, _lp, _lp]
    L.orc_tree_level_boxes.restype = C.c_int
    L.orc_tree_level_boxes.argtypes = [C.c_void_p, C.c_int, _ip]
    L.orc_tree_box_lists.argtypes = [C.c_void_p, C.c_int, _ip, _ip, _ip, _ip]
    L.orc_cpqr_id.restype = C.c_int
    L.orc_cpqr_id.argtypes = [_dp, C.c_int, C.c_int, C.c_double, _ip, _dp, _dp]
    L.orc_lu.restype = C.c_int
    L.orc_lu.argtypes = [_dp, C.c_int, _ip]
    L.orc_factor.restype = C.c_void_p
    L.orc_factor.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_double, C.c_int,
                             C.c_double, C.c_int, C.c_int, C.c_int, C.c_int]
    L.orc_factor_free.argtypes = [C.c_void_p]
    L.orc_factor_info.restype = C.c_int64
    L.orc_factor_info.argtypes = [C.c_void_p, C.c_int]
    L.orc_factor_check_worst.restype = C.c_double
    L.orc_factor_check_worst.argtypes = [C.c_void_p, C.c_int]
    L.orc_plant_mistake.argtypes = [C.c_int]
    L.orc_factor_box.argtypes = [C.c_void_p, C.c_int, _ip]
    L.orc_factor_box_data.argtypes = [C.c_void_p, C.c_int, _lp, _lp, _lp, _dp, _dp, _dp]
    L.orc_factor_top.argtypes = [C.c_void_p, _lp]
    L.orc_sqrt_prepare.restype = C.c_int
    L.orc_sqrt_prepare.argtypes = [C.c_void_p]
    L.orc_sqrt_apply.argtypes = [C.c_void_p, _dp, _dp, C.c_int, C.c_int]
    L.orc_logdet.restype = C.c_double
    L.orc_logdet.argtypes = [C.c_void_p]
    L.orc_apply.argtypes = [C.c_void_p, _dp, _dp, C.c_int]
    L.orc_solve.argtypes = [C.c_void_p, _dp, _dp, C.c_int]
    L.orc_dense_matrix.argtypes = [_dp, C.c_int64, C.c_int, C.c_int, C.c_double, C.c_double, _dp]
    L.orc_matvec_rows.argtypes = [_dp, C.c_int64, C.c_int, C.c_int, C.c_double, C.c_double, _dp,
                                  C.c_int, _lp, C.c_int64, _dp]
    L.orc_dense_solve.restype = C.c_int
    L.orc_dense_solve.argtypes = [_dp, C.c_int, _dp, C.c_int]


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


def _l(a):
    return a.ctypes.data_as(_lp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# Tree
# ---------------------------------------------------------------------------

class Tree:
    """Adaptive 2^d-tree on [0,1]^d, split while a node holds > leaf points."""

    def __init__(self, pts: np.ndarray, leaf: int):
        L = lib()
        self.pts = _f64(pts)
        self.n, self.dim = self.pts.shape
        self.leaf = leaf
        self.h = L.orc_tree_build(_d(self.pts), self.n, self.dim, leaf)
        if not self.h:
            raise ValueError("bad tree arguments")
        self.nnode = L.orc_tree_info(self.h, 0)
        self.maxdepth = L.orc_tree_info(self.h, 1)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_tree_free(self.h)
            self.h = None

    def perm(self) -> np.ndarray:
        p = np.empty(self.n, dtype=np.int64)
        lib().orc_tree_perm(self.h, _l(p))
        return p

    def nodes(self) -> dict:
        nn = self.nnode
        depth = np.empty(nn, np.int32)
        parent = np.empty(nn, np.int32)
        coord = np.empty(3 * nn, np.int32)
        start = np.empty(nn, np.int64)
        count = np.empty(nn, np.int64)
        lib().orc_tree_nodes(self.h, _i(depth), _i(parent), _i(coord), _l(start), _l(count))
        return dict(depth=depth, parent=parent, coord=coord.reshape(nn, 3), start=start, count=count)

    def level_boxes(self, t: int) -> np.ndarray:
        out = np.empty(self.nnode, np.int32)
        nb = lib().orc_tree_level_boxes(self.h, t, _i(out))
        return out[:nb].copy()

    def box_lists(self, node: int):
        near = np.empty(125, np.int32)
        ring = np.empty(125, np.int32)
        nn = np.zeros(1, np.int32)
        nr = np.zeros(1, np.int32)
        lib().orc_tree_box_lists(self.h, node, _i(near), _i(nn), _i(ring), _i(nr))
        return near[: nn[0]].copy(), ring[: nr[0]].copy()


# ---------------------------------------------------------------------------
# Dense building blocks
# ---------------------------------------------------------------------------

def cpqr_id(M: np.ndarray, eps: float):
    """ID by greedy column-pivoted Householder QR.  Returns (k, perm, T, rdiag)
    with M[:, perm[k:]] ~= M[:, perm[:k]] @ T."""
    m, n = M.shape
    Mc = np.asfortranarray(M, dtype=np.float64).copy(order="F")
    perm = np.empty(n, np.int32)
    T = np.zeros(max(n * n, 1))
    rd = np.zeros(max(min(m, n), 1))
    k = lib().orc_cpqr_id(Mc.ctypes.data_as(_dp), m, n, eps, _i(perm), _d(T), _d(rd))
    Tm = T[: k * (n - k)].reshape(n - k, k).T.copy()
    return k, perm, Tm, rd[: min(m, n)]


def lu(A: np.ndarray):
    """LU with partial pivoting: returns (LU, piv, info), A[piv] = L @ U."""
    n = A.shape[0]
    a = np.ascontiguousarray(A, dtype=np.float64).copy()
    piv = np.empty(n, np.int32)
    info = lib().orc_lu(_d(a), n, _i(piv))
    return a, piv, info


# ---------------------------------------------------------------------------
# Factorization
# ---------------------------------------------------------------------------

class Factor:
    """RS-S factor of A = diag*I + w*K on the tree's points (Algorithm 1);
    hybrid=True: the RS-WS factor (Sec. 3.4, Algorithm 2).  schedule: 0 one
    box after another; 1 / 2 each colour phase as a parallel machine runs it,
    with 3^d / 2^d colours (Sec. 5; see ``orc_factor``).  cholesky=True:
    X_RR and the top block by Cholesky (positive definite K) and G = E^T."""

    def __init__(self, tree: Tree, kind: int, eps: float, diag: float = 1.0, w: float | None = None,
                 nproxy: int = 0, radius: float = 2.5, check: bool = False, hybrid: bool = False,
                 schedule: int = 0, cholesky: bool = False):
        self.tree = tree
        self.kind = kind
        self.diag = diag
        self.w = (1.0 / tree.n) if w is None else w
        self.eps = eps
        self.h = lib().orc_factor(tree.h, kind, diag, self.w, eps, nproxy, radius, int(check), int(hybrid),
                                  int(schedule), int(cholesky))
        L = lib()
        self.nbox = L.orc_factor_info(self.h, 0)
        self.ntop = L.orc_factor_info(self.h, 1)
        self.violations = L.orc_factor_info(self.h, 2)
        self.info = L.orc_factor_info(self.h, 3)
        # check mode: boxes over the CPQR ID bound and boxes whose T does not
        # compress the full far field to 10 eps, with the worst ratios
        self.id_violations = L.orc_factor_info(self.h, 4)
        self.proxy_violations = L.orc_factor_info(self.h, 5)
        self.id_worst = L.orc_factor_check_worst(self.h, 0)
        self.proxy_worst = L.orc_factor_check_worst(self.h, 1)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_factor_free(self.h)
            self.h = None

    def box(self, i: int) -> dict:
        v = np.empty(9, np.int32)
        lib().orc_factor_box(self.h, i, _i(v))
        return dict(zip(["node", "depth", "b", "k", "r", "nj", "nnear", "nring", "weak"], map(int, v)))

    def boxes(self) -> list:
        return [self.box(i) for i in range(self.nbox)]

    def box_data(self, i: int) -> dict:
        b = self.box(i)
        k, r, nj = b["k"], b["r"], b["nj"]
        S = np.empty(max(k, 1), np.int64)
        R = np.empty(max(r, 1), np.int64)
        J = np.empty(max(nj, 1), np.int64)
        T = np.empty(max(k * r, 1))
        E = np.empty(max(nj * r, 1))
        G = np.empty(max(r * nj, 1))
        lib().orc_factor_box_data(self.h, i, _l(S), _l(R), _l(J), _d(T), _d(E), _d(G))
        b.update(S=S[:k], R=R[:r], J=J[:nj], T=T[: k * r].reshape(r, k).T.copy(),
                 E=E[: nj * r].reshape(nj, r), G=G[: r * nj].reshape(r, nj))
        return b

    def top(self) -> np.ndarray:
        t = np.empty(max(self.ntop, 1), np.int64)
        lib().orc_factor_top(self.h, _l(t))
        return t[: self.ntop]

    def sqrt_apply(self, x: np.ndarray, transpose: bool = False) -> np.ndarray:
        """Generalized square root (positive definite K): F^{1/2} x, or
        (F^{1/2})^T x with transpose=True; F = F^{1/2} (F^{1/2})^T.  Raises
        ValueError when a diagonal block is not positive definite."""
        L = lib()
        st = L.orc_sqrt_prepare(self.h)
        if st:
            raise ValueError(f"block {st - 1} of D is not positive definite")
        x, one = self._vec(x)
        y = np.empty_like(x)
        L.orc_sqrt_apply(self.h, _d(x), _d(y), x.shape[0] if x.ndim == 2 else 1, int(transpose))
        return y[0] if one else y

    def logdet(self) -> float:
        return lib().orc_logdet(self.h)

    def _vec(self, x):
        x = np.asarray(x, dtype=np.float64)
        if x.ndim == 1:
            return np.ascontiguousarray(x[None, :]), True
        return np.ascontiguousarray(x), False  # (nrhs, n): column c is row c

    def apply(self, x: np.ndarray) -> np.ndarray:
        """y = F x; x has shape (n,) or (nrhs, n), original point order."""
        xv, one = self._vec(x)
        y = np.empty_like(xv)
        lib().orc_apply(self.h, _d(xv), _d(y), xv.shape[0])
        return y[0] if one else y

    def solve(self, b: np.ndarray) -> np.ndarray:
        """x = F^{-1} b; b has shape (n,) or (nrhs, n), original point order."""
        bv, one = self._vec(b)
        x = np.empty_like(bv)
        lib().orc_solve(self.h, _d(bv), _d(x), bv.shape[0])
        return x[0] if one else x


# ---------------------------------------------------------------------------
# Exact references
# ---------------------------------------------------------------------------

def plant_mistake(what: int) -> None:
    """Plant a deliberate mistake in the oracle (tests of its checks only):
    0 none, 1 every proxy surface centred one box side off in x."""
    lib().orc_plant_mistake(int(what))


def dense_matrix(pts: np.ndarray, kind: int, diag: float = 1.0, w: float | None = None) -> np.ndarray:
    pts = _f64(pts)
    n, dim = pts.shape
    w = (1.0 / n) if w is None else w
    A = np.empty((n, n))
    lib().orc_dense_matrix(_d(pts), n, dim, kind, diag, w, _d(A))
    return A


def matvec(pts: np.ndarray, kind: int, x: np.ndarray, diag: float = 1.0, w: float | None = None,
           rows: np.ndarray | None = None) -> np.ndarray:
    """Exact FP64 direct-sum A x (all rows, or the rows listed)."""
    pts = _f64(pts)
    n, dim = pts.shape
    w = (1.0 / n) if w is None else w
    xv = np.ascontiguousarray(np.atleast_2d(np.asarray(x, dtype=np.float64)))
    nrhs = xv.shape[0]
    if rows is None:
        nr = n
        rp = None
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        nr = rows.shape[0]
        rp = _l(rows)
    y = np.empty((nrhs, nr))
    lib().orc_matvec_rows(_d(pts), n, dim, kind, diag, w, _d(xv), nrhs, rp, nr, _d(y))
    return y[0] if np.asarray(x).ndim == 1 else y


def dense_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Solve A x = b by the oracle's plain LU with partial pivoting."""
    a = np.ascontiguousarray(A, dtype=np.float64).copy()
    bv = np.ascontiguousarray(np.atleast_2d(np.asarray(b, dtype=np.float64))).copy()
    info = lib().orc_dense_solve(_d(a), a.shape[0], _d(bv), bv.shape[0])
    if info:
        raise np.linalg.LinAlgError(f"zero pivot {info}")
    return bv[0] if np.asarray(b).ndim == 1 else bv
