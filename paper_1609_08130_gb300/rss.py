"""Thin Python binding of the RS-S C ABI (include/rss.h).

Argument marshalling only: every step of the factorization, apply and solve
runs in the CUDA kernels of ``librss.so``.  Device buffers are torch CUDA
tensors; the binding passes their data pointers and the current stream.
There is no fallback: if the library is missing or no GPU is present the
calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_CSRC = os.path.join(_HERE, "csrc")
_INC = os.path.join(os.path.dirname(_HERE), "include")
LIB_PATH = os.path.join(_HERE, "librss.so")
SOURCES = ["api.cu", "kernels.cu", "refine.cu", "mlp.cu", "logdet.cu", "schur_tc.cu", "tree.cu"]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
              "-Xcompiler", "-fPIC", "-shared"]

RSS_OK, RSS_EINVAL, RSS_ENOMEM, RSS_ECUDA, RSS_ENUMERIC, RSS_ETIMEOUT, RSS_ENOTCONV = range(7)
LAPLACE2D_LOG, LAPLACE3D_INV = 0, 1
FP64, MIXED = 0, 1
FLAG_LARGE_BOX_PATH = 1
FLAG_NO_AUTOTUNE = 2
FLAG_COLOUR_2D = 4
FLAG_NO_TENSOR_CORES = 8
FLAG_SYMMETRIC_STORAGE = 16
FLAG_HYBRID = 32
FLAG_ASYNC = 64


def _nvcc():
    for c in [os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"]:
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def build(force: bool = False) -> str:
    """Compile librss.so in-tree for sm_103a (translation units in parallel)."""
    srcs = [os.path.join(_CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(_CSRC, h) for h in ("common.cuh", "internal.h", "tc.cuh")] + \
        [os.path.join(_INC, "rss.h")]
    if not force and os.path.exists(LIB_PATH) and \
            os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(d) for d in deps):
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = [_nvcc(), *NVCC_FLAGS, "--threads", "4", "-o", tmp, *srcs]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class RSSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"rss status {status}: {msg}")
        self.status = status


class _Kernel(C.Structure):
    _fields_ = [("kind", C.c_int), ("diag", C.c_double), ("weight", C.c_double)]


class _Options(C.Structure):
    _fields_ = [("prec", C.c_int), ("n_proxy", C.c_int), ("proxy_radius", C.c_double),
                ("use_graphs", C.c_int), ("stream", C.c_void_p), ("profile", C.c_int), ("flags", C.c_int),
                ("mlp", C.c_void_p)]


MLP_NFEAT = 16
MLP_NPARAM = 9473


_lib = None

# Every entry point declared in include/rss.h, with its ctypes signature.
_SIGS = {
    "rss_build_tree": (C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_int, C.POINTER(C.c_void_p)]),
    "rss_tree_query": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_size_t)]),
    "rss_factor": (C.c_int, [C.c_void_p, C.c_int64, C.c_int, _Kernel, C.c_double, C.c_int,
                             C.POINTER(_Options), C.POINTER(C.c_void_p)]),
    "rss_factor_batched": (C.c_int, [C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_int64), C.c_int, _Kernel,
                                     C.c_double, C.c_int, C.POINTER(_Options), C.POINTER(C.c_void_p)]),
    "rss_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "rss_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "rss_matvec": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "rss_sync": (C.c_int, [C.c_void_p]),
    "rss_solve_cg": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_int,
                               C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "rss_solve_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "rss_solve_refined": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_int,
                                    C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "rss_stats": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_size_t)]),
    "rss_logdet": (C.c_int, [C.c_void_p, C.c_void_p]),
    "rss_stats_json": (C.c_int, [C.c_void_p, C.c_char_p, C.POINTER(C.c_size_t)]),
    "rss_sqrt_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    "rss_profile": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_size_t)]),
    "rss_mlp_create": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.POINTER(C.c_void_p)]),
    "rss_mlp_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "rss_mlp_predict": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "rss_mlp_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                               C.POINTER(C.c_double)]),
    "rss_mlp_train": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_float,
                                C.POINTER(C.c_double)]),
    "rss_box_features": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]),
    "rss_autotune_table": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "rss_autotune_set": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]),
    "rss_autotune_clear": (None, []),
    "rss_autotune_elim_table": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "rss_free": (None, [C.c_void_p]),
    "rss_last_error": (C.c_char_p, []),
    "rss_kernel_launches": (C.c_int64, []),
}


def lib(load_only: bool = False):
    """Load librss.so (building it first if needed)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH) and not load_only:
            build()
        if not os.path.exists(LIB_PATH):
            raise RSSError(RSS_ECUDA, f"CUDA library not built: {LIB_PATH}")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def kernel_launches() -> int:
    """Kernel launches made by librss.so in this process so far."""
    return int(lib().rss_kernel_launches())


def autotune_table() -> list:
    """rss_autotune_table: [{elem_bytes, width, phase_class, tpc, groups, ctas, rows, us: [18 candidates]}]."""
    import numpy as np
    nb = C.c_size_t(0)
    _check(lib().rss_autotune_table(None, C.byref(nb)))
    buf = np.zeros(max(nb.value // 4, 1), dtype=np.int32)
    _check(lib().rss_autotune_table(C.c_void_p(buf.ctypes.data), C.byref(nb)))
    rl = 7 + len(AUTOTUNE_SHAPES)
    recs = buf[:nb.value // 4].reshape(-1, rl)
    return [dict(elem_bytes=int(r[0]), width=int(r[1]), phase_class=int(r[2]), tpc=int(r[3]), groups=int(r[4]),
                 ctas=int(r[5]), rows=int(r[6]), us=[int(x) for x in r[7:rl]]) for r in recs]


def autotune_elim_table() -> list:
    """rss_autotune_elim_table: [{elem_bytes, width, phase_class, split, ctas, us: [5 candidates]}]."""
    import numpy as np
    nb = C.c_size_t(0)
    _check(lib().rss_autotune_elim_table(None, C.byref(nb)))
    buf = np.zeros(max(nb.value // 4, 1), dtype=np.int32)
    _check(lib().rss_autotune_elim_table(C.c_void_p(buf.ctypes.data), C.byref(nb)))
    recs = buf[:nb.value // 4].reshape(-1, 10)
    return [dict(elem_bytes=int(r[0]), width=int(r[1]), phase_class=int(r[2]), split=int(r[3]), ctas=int(r[4]),
                 us=[int(x) for x in r[5:10]]) for r in recs]


ELIM_SHAPES = [(0, 1), (1, 1), (1, 2), (1, 4), (1, 8)]


# (threads per column, fold groups, CTAs per box, panel rows per thread in
# units of 32 FP32 / 16 FP64 rows); threads per column 0: the warp-per-panel
# form with `groups` warps (box width class 64 only)
AUTOTUNE_SHAPES = [(1, 1, 1, 1), (1, 2, 1, 1), (1, 4, 1, 1), (2, 1, 1, 1), (2, 2, 1, 1), (2, 4, 1, 1),
                   (4, 1, 1, 1), (4, 2, 1, 1), (2, 1, 4, 1), (2, 1, 8, 1), (4, 1, 4, 1), (4, 1, 8, 1),
                   (0, 2, 1, 1), (0, 4, 1, 1), (0, 8, 1, 1), (1, 1, 1, 2), (1, 2, 1, 2), (1, 4, 1, 2)]


def shape_fits(width: int, tpc: int, groups: int, rows: int = 1) -> bool:
    """Whether (tpc, groups, rows) is a candidate for a box-width class."""
    if rows != 1 and (rows != 2 or tpc != 1 or width > 128):
        return False
    if tpc == 0:
        return width == 64 and groups in (2, 4, 8)
    return width * tpc * groups <= (256 if tpc == 1 else 512)


def _check(st: int):
    if st != RSS_OK:
        raise RSSError(st, lib().rss_last_error().decode(errors="replace"))


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RSSError(RSS_ECUDA, "no CUDA device")
    return torch


def _dev_f64(t, shape_hint=None):
    torch = _torch()
    t = torch.as_tensor(t)
    if t.device.type != "cuda":
        t = t.to("cuda")
    return t.to(torch.float64).contiguous()


class Tree:
    """rss_build_tree: adaptive 2^d-tree; arrays copied out with rss_tree_query."""

    def __init__(self, pts, leaf: int = 64):
        pts = _dev_f64(pts)
        n, dim = pts.shape
        h = C.c_void_p()
        _check(lib().rss_build_tree(C.c_void_p(pts.data_ptr()), n, dim, leaf, C.byref(h)))
        self.h = h
        self.n, self.dim, self.leaf = n, dim, leaf
        s = self.query(6, "int64")
        self.nnode, self.maxdepth = int(s[0]), int(s[1])

    def query(self, what: int, dtype: str):
        import numpy as np
        nb = C.c_size_t(0)
        _check(lib().rss_tree_query(self.h, what, None, C.byref(nb)))
        buf = np.empty(max(nb.value // np.dtype(dtype).itemsize, 1), dtype=dtype)
        _check(lib().rss_tree_query(self.h, what, C.c_void_p(buf.ctypes.data), C.byref(nb)))
        return buf[: nb.value // np.dtype(dtype).itemsize]

    def perm(self):
        return self.query(0, "int64")

    def nodes(self):
        return dict(depth=self.query(1, "int32"), parent=self.query(2, "int32"),
                    coord=self.query(3, "int32").reshape(-1, 3), start=self.query(4, "int64"),
                    count=self.query(5, "int64"))

    def level_boxes(self, t: int):
        return self.query(100 + t, "int32")

    def box_lists(self, t: int):
        """Per box of depth t (elimination order): (near codes, ring codes)."""
        rec = self.query(200 + t, "int32")
        out, i = [], 0
        while i < len(rec):
            nn, nr = int(rec[i]), int(rec[i + 1])
            out.append((rec[i + 2:i + 2 + nn].copy(), rec[i + 2 + nn:i + 2 + nn + nr].copy()))
            i += 2 + nn + nr
        return out

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.rss_free(self.h)
            self.h = None


class Factorization:
    """rss_factor: RS-S factorization of A = diag*I + w*K on the given points.

    pts: (n, dim) float64 (moved to the GPU).  kind: 0 2D log kernel, 1 3D
    1/r kernel.  prec: FP64 or MIXED (FP32 factor).
    """

    def __init__(self, pts, kind: int, eps: float, leaf: int = 64, prec: int = FP64, diag: float = 1.0,
                 weight: float = 0.0, n_proxy: int = 0, proxy_radius: float = 0.0, stream=None,
                 profile: bool = False, flags: int = 0, mlp=None, use_graphs: bool = True):
        torch = _torch()
        pts = _dev_f64(pts)
        self.n, self.dim = pts.shape
        self.prec = prec
        st = stream if stream is not None else torch.cuda.current_stream()
        self.stream = st
        opts = _Options(prec, n_proxy, proxy_radius, int(use_graphs), C.c_void_p(st.cuda_stream), int(profile), int(flags),
                        mlp.h if mlp is not None else None)
        h = C.c_void_p()
        _check(lib().rss_factor(C.c_void_p(pts.data_ptr()), self.n, self.dim, _Kernel(kind, diag, weight),
                                eps, leaf, C.byref(opts), C.byref(h)))
        self.h = h

    @classmethod
    def batched(cls, pts_list, kind: int, eps: float, leaf: int = 64, prec: int = FP64, diag: float = 1.0,
                weight: float = 0.0, n_proxy: int = 0, proxy_radius: float = 0.0, stream=None,
                profile: bool = False, flags: int = 0, mlp=None, use_graphs: bool = True):
        """rss_factor_batched: one handle for several independent problems;
        vectors are the problems' vectors concatenated in order."""
        torch = _torch()
        pts = [_dev_f64(p) for p in pts_list]
        dim = pts[0].shape[1]
        self = cls.__new__(cls)
        self.n = int(sum(p.shape[0] for p in pts))
        self.dim = dim
        self.prec = prec
        self.sizes = [int(p.shape[0]) for p in pts]
        st = stream if stream is not None else torch.cuda.current_stream()
        self.stream = st
        self._keep = pts
        opts = _Options(prec, n_proxy, proxy_radius, int(use_graphs), C.c_void_p(st.cuda_stream), int(profile), int(flags),
                        mlp.h if mlp is not None else None)
        arr = (C.c_void_p * len(pts))(*[p.data_ptr() for p in pts])
        ns = (C.c_int64 * len(pts))(*self.sizes)
        h = C.c_void_p()
        _check(lib().rss_factor_batched(len(pts), arr, ns, dim, _Kernel(kind, diag, weight), eps, leaf,
                                        C.byref(opts), C.byref(h)))
        self.h = h
        return self

    def _vec(self, x):
        torch = _torch()
        x = _dev_f64(x)
        one = x.dim() == 1
        if one:
            x = x.reshape(1, -1)
        if x.shape[1] != self.n:
            raise RSSError(RSS_EINVAL, "vector length does not match the factor")
        return x, one, torch.empty_like(x)

    def _call(self, fn, x):
        x, one, y = self._vec(x)
        _check(fn(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), x.shape[0]))
        return y[0] if one else y

    def apply(self, x):
        """y = F x; x of shape (n,) or (nrhs, n)."""
        return self._call(lib().rss_apply, x)

    def solve(self, b):
        """x = F^{-1} b; b of shape (n,) or (nrhs, n)."""
        return self._call(lib().rss_solve, b)

    def solve_refined(self, b, tol: float = 1e-10, maxit: int = 10, check: bool = True):
        """GMRES-IR solve of A x = b to relative residual tol.  Returns
        (x, inner iterations, final relative residual)."""
        b, one, x = self._vec(b)
        it = C.c_int(0)
        rr = C.c_double(0.0)
        st = lib().rss_solve_refined(self.h, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), b.shape[0],
                                     tol, maxit, C.byref(it), C.byref(rr))
        if check or st != RSS_ENOTCONV:
            _check(st)
        return (x[0] if one else x), it.value, rr.value

    def solve_cg(self, b, tol: float = 1e-10, maxit: int = 50, check: bool = True):
        """Conjugate gradients on A x = b preconditioned with the factor.
        Returns (x, iterations, final relative residual)."""
        b, one, x = self._vec(b)
        it = C.c_int(0)
        rr = C.c_double(0.0)
        st = lib().rss_solve_cg(self.h, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), b.shape[0], tol, maxit,
                                C.byref(it), C.byref(rr))
        if check or st != RSS_ENOTCONV:
            _check(st)
        return (x[0] if one else x), it.value, rr.value

    def sqrt_apply(self, x, transpose: bool = False):
        """Generalized square root: F^{1/2} x, or (F^{1/2})^T x."""
        x, one, y = self._vec(x)
        _check(lib().rss_sqrt_apply(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), x.shape[0],
                                    int(transpose)))
        return y[0] if one else y

    def matvec(self, x):
        """Exact FP64 A x by direct summation."""
        return self._call(lib().rss_matvec, x)

    def sync(self):
        """rss_sync: wait for the factor's stream; raises RSSError for a
        device error recorded by asynchronous work (FLAG_ASYNC)."""
        _check(lib().rss_sync(self.h))

    def logdet(self):
        """rss_logdet: log|det F| per problem (numpy float64 array)."""
        import numpy as np
        out = np.zeros(len(getattr(self, "sizes", [self.n])), dtype=np.float64)
        _check(lib().rss_logdet(self.h, C.c_void_p(out.ctypes.data)))
        return out

    def stats(self) -> dict:
        import numpy as np
        nb = C.c_size_t(0)
        _check(lib().rss_stats(self.h, None, C.byref(nb)))
        buf = np.empty(nb.value // 8, dtype=np.int64)
        _check(lib().rss_stats(self.h, C.c_void_p(buf.ctypes.data), C.byref(nb)))
        nbox = int(buf[0])
        boxes = buf[11:11 + 6 * nbox].reshape(nbox, 6)
        return dict(nbox=nbox, ntop=int(buf[1]), factor_bytes=int(buf[2]), maxdepth=int(buf[3]),
                    n=int(buf[4]), prec=int(buf[5]), reserved_bytes=int(buf[6]), used_bytes=int(buf[7]),
                    overflow_bytes=int(buf[8]), retried=int(buf[9]), proposal=int(buf[10]),
                    depth=boxes[:, 0].copy(), b=boxes[:, 1].copy(), k=boxes[:, 2].copy(),
                    nj=boxes[:, 3].copy(), rres=boxes[:, 4].copy(), njres=boxes[:, 5].copy())

    def stats_json(self) -> dict:
        """rss_stats_json, parsed."""
        import json
        nb = C.c_size_t(0)
        _check(lib().rss_stats_json(self.h, None, C.byref(nb)))
        buf = C.create_string_buffer(nb.value)
        _check(lib().rss_stats_json(self.h, buf, C.byref(nb)))
        return json.loads(buf.value.decode())

    def box_features(self):
        """rss_box_features: (features (nbox, 16) float32, ranks (nbox,) int32)."""
        import numpy as np
        nbox = self.stats()["nbox"]
        feat = np.zeros((nbox, MLP_NFEAT), dtype=np.float32)
        rank = np.zeros(nbox, dtype=np.int32)
        _check(lib().rss_box_features(self.h, C.c_void_p(feat.ctypes.data), C.c_void_p(rank.ctypes.data), nbox))
        return feat, rank

    PROFILE_CLASSES = ["assemble", "id", "elim", "schur", "top_lu", "sweep", "top_solve", "permute",
                       "host_tree", "host_level", "host_wait", "refine_op", "inner_op"]

    def profile(self, reset: bool = False) -> dict:
        """Per-kernel-class {launches, ms, bytes, flops} (needs profile=True)."""
        import numpy as np
        nb = C.c_size_t(0)
        _check(lib().rss_profile(self.h, 0, None, C.byref(nb)))
        buf = np.empty(nb.value // 8)
        _check(lib().rss_profile(self.h, int(reset), C.c_void_p(buf.ctypes.data), C.byref(nb)))
        buf = buf.reshape(-1, 4)
        return {name: dict(launches=int(buf[i, 0]), ms=float(buf[i, 1]), bytes=float(buf[i, 2]),
                           flops=float(buf[i, 3])) for i, name in enumerate(self.PROFILE_CLASSES)}

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.rss_free(self.h)
            self.h = None


class Mlp:
    """rss_mlp_*: the rank-proposal network (16 -> 64 -> 64 -> 64 -> 1, tanh),
    evaluated and trained by the library's CUDA kernels.  params: FP32 host
    array of MLP_NPARAM values, or None for a seeded Glorot initialisation."""

    def __init__(self, params=None, seed: int = 0, stream=None):
        import numpy as np
        torch = _torch()
        st = stream if stream is not None else torch.cuda.current_stream()
        self.stream = st
        h = C.c_void_p()
        if params is not None:
            self._init = np.ascontiguousarray(params, dtype=np.float32)
            if self._init.size != MLP_NPARAM:
                raise RSSError(RSS_EINVAL, "wrong number of parameters")
            pp = C.c_void_p(self._init.ctypes.data)
        else:
            pp = None
        _check(lib().rss_mlp_create(pp, C.c_uint64(seed), C.c_void_p(st.cuda_stream), C.byref(h)))
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.rss_free(self.h)
            self.h = None

    def params(self):
        import numpy as np
        out = np.empty(MLP_NPARAM, dtype=np.float32)
        _check(lib().rss_mlp_params(self.h, C.c_void_p(out.ctypes.data)))
        return out

    @staticmethod
    def _f32(t):
        torch = _torch()
        t = torch.as_tensor(t)
        if t.device.type != "cuda":
            t = t.to("cuda")
        return t.to(torch.float32).contiguous()

    def predict(self, X):
        torch = _torch()
        X = self._f32(X)
        y = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
        _check(lib().rss_mlp_predict(self.h, C.c_void_p(X.data_ptr()), X.shape[0], C.c_void_p(y.data_ptr())))
        return y

    def grad(self, X, y):
        torch = _torch()
        X, y = self._f32(X), self._f32(y)
        g = torch.empty(MLP_NPARAM, dtype=torch.float32, device="cuda")
        loss = C.c_double()
        _check(lib().rss_mlp_grad(self.h, C.c_void_p(X.data_ptr()), C.c_void_p(y.data_ptr()), X.shape[0],
                                  C.c_void_p(g.data_ptr()), C.byref(loss)))
        return g, loss.value

    def train(self, X, y, iters: int, lr: float = 1e-3) -> float:
        X, y = self._f32(X), self._f32(y)
        loss = C.c_double()
        _check(lib().rss_mlp_train(self.h, C.c_void_p(X.data_ptr()), C.c_void_p(y.data_ptr()), X.shape[0],
                                   int(iters), C.c_float(lr), C.byref(loss)))
        return loss.value
