"""Python access to the FP64 CPU oracle (``h2_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this module; the CUDA library never
does.  It imports nothing from the CUDA package.

Every function mirrors one step of the data-driven H^2 construction
(arXiv 2206.01885): the tree and interaction lists (section 2.1, eq. (1)),
DataReduct (section 3.3), HiDR (Algorithm 1), getBasis (eqs. (3)-(5)), the
construction (Algorithm 2), the matvec, and the section 4.2 calibration.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "h2_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle_h2.so")
_lock = threading.Lock()
_lib = None

KERNELS = {"coulomb": 1, "gaussian": 2, "exponential": 3, "multiquadric": 4, "bump": 5, "power": 6,
           "cosdot": 7}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC",
               "-std=gnu11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
            L.or_tree_build.restype = vp
            L.or_tree_build.argtypes = [vp, i64, i32, i32, i64, i64]
            L.or_tree_lists.argtypes = [vp]
            L.or_tree_info.argtypes = [vp, vp, vp]
            L.or_tree_get.argtypes = [vp, i32, vp]
            L.or_admissible.argtypes = [vp, i32, i32]
            L.or_tree_free.argtypes = [vp]
            L.or_datareduct.restype = i64
            L.or_datareduct.argtypes = [vp, i32, vp, i64, i32, vp]
            L.or_datareduct_surface.restype = i64
            L.or_datareduct_surface.argtypes = [vp, i32, vp, i64, i32, vp]
            L.or_datareduct_fps.restype = i64
            L.or_datareduct_fps.argtypes = [vp, i32, vp, i64, i32, vp]
            L.or_hidr.restype = vp
            L.or_hidr.argtypes = [vp, i32, i32, vp, i32, i32]
            L.or_hidr_get.restype = i64
            L.or_hidr_get.argtypes = [vp, i32, i32, vp]
            L.or_hidr_free.argtypes = [vp]
            L.or_id.restype = i32
            L.or_id.argtypes = [vp, i32, i32, dbl, vp, vp]
            L.or_construct.restype = vp
            L.or_construct.argtypes = [vp, vp, i32, vp, dbl, vp, dbl]
            L.or_id_bound.restype = i32
            L.or_id_bound.argtypes = [i32, i32, vp, vp, dbl, i32]
            L.or_h2_exchanges.restype = i64
            L.or_h2_exchanges.argtypes = [vp]
            L.or_h2_rank.restype = i32
            L.or_h2_rank.argtypes = [vp, i32, i32]
            L.or_h2_skel.argtypes = [vp, i32, vp]
            L.or_h2_U.argtypes = [vp, i32, vp]
            L.or_h2_free.argtypes = [vp]
            L.or_matvec.argtypes = [vp, vp, vp]
            L.or_exact_rows.argtypes = [vp, i64, i32, i32, vp, vp, vp, i64, vp]
            L.or_dense_matvec.argtypes = [vp, i64, i32, i32, vp, vp, vp]
            L.or_calib_error.restype = dbl
            L.or_calib_error.argtypes = [i32, i32, vp, dbl, vp, i32, vp, i32, i32, vp, vp]
            L.or_calibrate.restype = i32
            L.or_calibrate.argtypes = [i32, i32, vp, dbl, vp, i32, vp, i32, i32]
            L.or_num_threads.restype = i32
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _kp(kparams) -> np.ndarray:
    a = np.zeros(4)
    a[: len(kparams)] = kparams
    return a


def _kid(kernel) -> int:
    return KERNELS[kernel] if isinstance(kernel, str) else int(kernel)


def num_threads() -> int:
    return lib().or_num_threads()


@dataclass
class Tree:
    """Cluster tree and interaction lists, all arrays copied out of the oracle."""
    handle: int
    n: int
    d: int
    B: int
    lo: np.ndarray
    side: float
    perm: np.ndarray
    key: np.ndarray
    x: np.ndarray
    level: np.ndarray
    parent: np.ndarray
    fchild: np.ndarray
    nchild: np.ndarray
    begin: np.ndarray
    end: np.ndarray
    prefix: np.ndarray
    lptr: np.ndarray
    near_ptr: np.ndarray
    near_idx: np.ndarray
    far_ptr: np.ndarray
    far_idx: np.ndarray
    _alive: list = field(default_factory=lambda: [True])

    @property
    def nnodes(self) -> int:
        return len(self.level)

    @property
    def nlevels(self) -> int:
        return len(self.lptr) - 1

    def is_leaf(self, i: int) -> bool:
        return self.nchild[i] == 0

    def far(self, i: int) -> np.ndarray:
        return self.far_idx[self.far_ptr[i]:self.far_ptr[i + 1]]

    def near(self, i: int) -> np.ndarray:
        return self.near_idx[self.near_ptr[i]:self.near_ptr[i + 1]]

    def admissible(self, i: int, j: int) -> bool:
        return bool(lib().or_admissible(self.handle, i, j))

    def free(self):
        if self._alive[0]:
            lib().or_tree_free(self.handle)
            self._alive[0] = False

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def tree_build(points: np.ndarray, leaf_size: int, tau=(7, 10)) -> Tree:
    """Adaptive Morton tree (section 2.1) plus near/far lists (eq. (1))."""
    L = lib()
    pts = np.ascontiguousarray(points, dtype=np.float64)
    if pts.ndim == 1:
        pts = pts[:, None]
    n, d = pts.shape
    h = L.or_tree_build(_p(pts), n, d, leaf_size, tau[0], tau[1])
    if not h:
        raise ValueError("invalid tree arguments")
    L.or_tree_lists(h)
    info = np.zeros(10, dtype=np.int64)
    geom = np.zeros(4)
    L.or_tree_info(h, _p(info), _p(geom))
    n, d, B, nn, nl, nnear, nfar = (int(v) for v in info[:7])

    def get(which, dtype, size):
        a = np.zeros(max(size, 1), dtype=dtype)
        if size > 0:
            L.or_tree_get(h, which, _p(a))
        return a[:size]

    t = Tree(handle=h, n=n, d=d, B=B, lo=geom[:d].copy(), side=float(geom[3]),
             perm=get(0, np.int64, n), key=get(1, np.uint64, n), x=get(14, np.float64, n * d).reshape(n, d),
             level=get(2, np.int32, nn), parent=get(3, np.int32, nn), fchild=get(4, np.int32, nn),
             nchild=get(5, np.int32, nn), begin=get(6, np.int64, nn), end=get(7, np.int64, nn),
             prefix=get(8, np.uint64, nn), lptr=get(9, np.int32, nl + 1),
             near_ptr=get(10, np.int64, nn + 1), near_idx=get(12, np.int32, nnear),
             far_ptr=get(11, np.int64, nn + 1), far_idx=get(13, np.int32, nfar))
    return t


DR_METHODS = {"volume": 0, "surface": 1, "fps": 2}


def datareduct(coords: np.ndarray, labels: np.ndarray, g: int, method: str = "volume") -> np.ndarray:
    """DataReduct(S, g^d) (section 3.3: volume- or surface-based, or farthest point sampling).  ``coords``
    indexed by label; ``labels`` the members of S.  Returns the sorted reduced
    labels."""
    L = lib()
    xs = np.ascontiguousarray(coords, dtype=np.float64)
    if xs.ndim == 1:
        xs = xs[:, None]
    S = np.ascontiguousarray(labels, dtype=np.int64)
    out = np.zeros(max(len(S), 1), dtype=np.int64)
    f = {0: L.or_datareduct, 1: L.or_datareduct_surface, 2: L.or_datareduct_fps}[DR_METHODS[method]]
    m = f(_p(xs), xs.shape[1], _p(S), len(S), g, _p(out))
    return out[:m].copy()


class Hidr:
    """X_i*, Y_i* of Algorithm 1.  ``il_reduce`` adds to each Y_i* the reduction
    of its interaction-list part alone (DataReduct over the union of X_j*,
    j in IL(i), on that part's own box), so |Y_i*| <= 2 g2^d."""

    def __init__(self, tree: Tree, g1: int, g2: int, need_y: np.ndarray | None = None, method: str = "volume",
                 il_reduce: bool = False):
        self.tree, self.g1, self.g2, self.il_reduce = tree, g1, g2, il_reduce
        flags = None
        if need_y is not None:
            flags = np.ascontiguousarray(need_y, dtype=np.uint8)
        self.handle = lib().or_hidr(tree.handle, g1, g2, _p(flags) if flags is not None else None,
                                    DR_METHODS[method], int(il_reduce))

    def get(self, node: int, which: str) -> np.ndarray | None:
        w = 0 if which == "x" else 1
        L = lib()
        n = L.or_hidr_get(self.handle, node, w, None)
        if n < 0:
            return None
        out = np.zeros(max(n, 1), dtype=np.int64)
        L.or_hidr_get(self.handle, node, w, _p(out))
        return out[:n]

    def __del__(self):
        try:
            lib().or_hidr_free(self.handle)
        except Exception:
            pass


def interp_decomp(A: np.ndarray, eps: float):
    """getBasis as a column-pivoted QR ID of A (m x c).  Returns (k, piv, T)
    with A[:, piv[k:]] ~= A[:, piv[:k]] @ T."""
    L = lib()
    m, c = A.shape
    a = np.asfortranarray(A, dtype=np.float64).copy(order="F")
    piv = np.zeros(max(c, 1), dtype=np.int32)
    T = np.zeros(max(min(m, c) * c, 1))
    k = L.or_id(a.ctypes.data_as(C.c_void_p), m, c, eps, _p(piv), _p(T))
    Tm = T[: k * (c - k)].reshape((c - k, k)).T.copy() if k > 0 else np.zeros((0, c))
    return k, piv[:c].copy(), Tm


def id_bound(k: int, piv: np.ndarray, T: np.ndarray, f: float, maxex: int | None = None):
    """The exchanges of eq. (3)'s bound ||G||_max <= f applied to an ID from
    interp_decomp.  Returns (number of exchanges, piv', T')."""
    c = len(piv)
    nr = c - k
    pv = np.ascontiguousarray(piv, dtype=np.int32).copy()
    t = np.zeros(max(k * nr, 1))
    t[: k * nr] = np.asarray(T, dtype=np.float64).T.reshape(-1)
    nex = lib().or_id_bound(k, nr, _p(pv), _p(t), f, 8 * k if maxex is None else maxex)
    return nex, pv, t[: k * nr].reshape((nr, k)).T.copy()


class H2:
    """Nested bases of Algorithm 2 and the H^2 matvec."""

    def __init__(self, tree: Tree, hidr: Hidr, kernel, kparams=(), eps: float = 1e-6,
                 need: np.ndarray | None = None, g_bound: float = 0.0):
        self.tree, self.hidr = tree, hidr
        self.kid = _kid(kernel)
        self.kp = _kp(kparams)
        flags = None if need is None else np.ascontiguousarray(need, dtype=np.uint8)
        self.handle = lib().or_construct(tree.handle, hidr.handle, self.kid, _p(self.kp), eps,
                                         _p(flags) if flags is not None else None, g_bound)

    def exchanges(self) -> int:
        return lib().or_h2_exchanges(self.handle)

    def rank(self, node: int) -> int:
        return lib().or_h2_rank(self.handle, node, 0)

    def ncand(self, node: int) -> int:
        return lib().or_h2_rank(self.handle, node, 1)

    def skeleton(self, node: int) -> np.ndarray:
        k = self.rank(node)
        out = np.zeros(max(k, 1), dtype=np.int64)
        if k > 0:
            lib().or_h2_skel(self.handle, node, _p(out))
        return out[:max(k, 0)]

    def U(self, node: int) -> np.ndarray:
        k, c = self.rank(node), self.ncand(node)
        out = np.zeros(max(k * c, 1))
        if k > 0:
            lib().or_h2_U(self.handle, node, _p(out))
        return out[: k * c].reshape((k, c)).T.copy() if k > 0 else np.zeros((c, 0))

    def matvec(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros(self.tree.n)
        lib().or_matvec(self.handle, _p(x), _p(y))
        return y

    def __del__(self):
        try:
            lib().or_h2_free(self.handle)
        except Exception:
            pass


def exact_rows(points, kernel, kparams, z, rows) -> np.ndarray:
    """(K z)_s = sum_j kappa(x_s, x_j) z_j for the given rows (pairwise sums)."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    if pts.ndim == 1:
        pts = pts[:, None]
    z = np.ascontiguousarray(z, dtype=np.float64)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.zeros(len(rows))
    kp = _kp(kparams)
    lib().or_exact_rows(_p(pts), pts.shape[0], pts.shape[1], _kid(kernel), _p(kp), _p(z), _p(rows),
                        len(rows), _p(out))
    return out


def dense_matvec(points, kernel, kparams, z) -> np.ndarray:
    pts = np.ascontiguousarray(points, dtype=np.float64)
    if pts.ndim == 1:
        pts = pts[:, None]
    z = np.ascontiguousarray(z, dtype=np.float64)
    y = np.zeros(pts.shape[0])
    kp = _kp(kparams)
    lib().or_dense_matvec(_p(pts), pts.shape[0], pts.shape[1], _kid(kernel), _p(kp), _p(z), _p(y))
    return y


def calib_error(d, kernel, kparams, id_tol, Z1, Z2, g):
    """Relative Frobenius error of the section 4.2 test problem at grid size g."""
    Z1 = np.ascontiguousarray(Z1, dtype=np.float64)
    Z2 = np.ascontiguousarray(Z2, dtype=np.float64)
    kp = _kp(kparams)
    k = C.c_int(0)
    m = C.c_int(0)
    e = lib().or_calib_error(d, _kid(kernel), _p(kp), id_tol, _p(Z1), len(Z1), _p(Z2), len(Z2), g,
                             C.byref(k), C.byref(m))
    return e, k.value, m.value


def calibrate(d, kernel, kparams, eps, Z1, Z2, gmax=16) -> int:
    """r1 = r2 = g^d from epsilon (section 4.2); gmax + 1 if no g <= gmax works."""
    Z1 = np.ascontiguousarray(Z1, dtype=np.float64)
    Z2 = np.ascontiguousarray(Z2, dtype=np.float64)
    kp = _kp(kparams)
    return lib().or_calibrate(d, _kid(kernel), _p(kp), eps, _p(Z1), len(Z1), _p(Z2), len(Z2), gmax)


def closure_down(tree: Tree, flags: np.ndarray) -> np.ndarray:
    """flags plus every descendant of a flagged node (nodes are numbered so
    that a parent precedes its children)."""
    f = np.asarray(flags, dtype=bool).copy()
    for i in range(1, tree.nnodes):
        if f[tree.parent[i]]:
            f[i] = True
    return f


def build_h2(points, kernel, kparams, leaf_size, eps, g1, g2, tau=(7, 10), g_bound=0.0, il_reduce=False):
    """Tree, lists, HiDR and the full construction, for small problems."""
    t = tree_build(points, leaf_size, tau)
    h = Hidr(t, g1, g2, il_reduce=il_reduce)
    H = H2(t, h, kernel, kparams, eps, g_bound=g_bound)
    return t, h, H
