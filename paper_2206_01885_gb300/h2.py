"""Python binding of the sm_103a H^2 library (``include/h2.h``).

Argument marshalling only: every step runs in the library's CUDA kernels.
PyTorch supplies device memory (CUDA tensors) and the current stream.  If the
shared library is missing this module raises instead of falling back to
anything else.

Names follow the C ABI: ``tree_build``, ``hidr_reduce``, ``construct``,
``matvec``, ``exact_rows``, ``calibrate``, ``free``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libh2gb300.so")

DR_METHODS = {"volume": 0, "surface": 1, "fps": 2}
HIDR_IL_REDUCE = 0x100  # H2_HIDR_IL_REDUCE, ORed into the method
HIDR_COPY_SETS = 0x200  # H2_HIDR_COPY_SETS
KERNELS = {"coulomb": 1, "gaussian": 2, "exponential": 3, "multiquadric": 4, "bump": 5, "power": 6,
           "cosdot": 7}
PRECISIONS = {"fp64": 0, "mixed": 1}
DTYPE_F64, DTYPE_F32 = 0, 1  # element types of h2_matvec vectors
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "TIMEOUT", 5: "NUMERIC", 6: "UNIMPLEMENTED",
          7: "STATE"}

TREE_FIELDS = {"perm": (0, np.int64), "keys": (1, np.uint64), "level": (2, np.int32), "parent": (3, np.int32),
               "fchild": (4, np.int32), "nchild": (5, np.int32), "begin": (6, np.int64), "end": (7, np.int64),
               "prefix": (8, np.uint64), "lptr": (9, np.int32), "near_ptr": (10, np.int64),
               "far_ptr": (11, np.int64), "near_idx": (12, np.int32), "far_idx": (13, np.int32),
               "info": (14, np.int64), "geom": (15, np.float64)}
MAT_FIELDS = {"rank": (0, np.int32), "ncand": (1, np.int32), "skel": (2, np.int32), "U": (3, np.float64),
              "info": (4, np.int64)}

_lib = None


class H2Error(RuntimeError):
    def __init__(self, call: str, status: int, msg: str):
        super().__init__(f"{call}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class _Params(C.Structure):
    _fields_ = [("leaf_size", C.c_int), ("tau_num", C.c_int), ("tau_den", C.c_int)]


class _ConstructOpts(C.Structure):
    _fields_ = [("g_bound", C.c_double), ("mem_mode", C.c_int), ("mem_fraction", C.c_double),
                ("fp64_products", C.c_int), ("tensor_core_products", C.c_int), ("fp64_qr", C.c_int)]


MEM_MODES = {"on_the_fly": 0, "store": 1, "auto": 2}  # H2_MEM_*


def lib():
    """Load the shared library (built by ``build.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing; build it with paper_2206_01885_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
        sig = {
            "h2_tree_build": [vp, i64, i32, i32, C.POINTER(_Params), vp, C.POINTER(vp)],
            "h2_tree_get": [vp, i32, vp, i64, C.POINTER(i64)],
            "h2_hidr_reduce": [vp, i32, i32, vp, C.POINTER(vp)],
            "h2_hidr_get": [vp, i32, vp, vp, i64, C.POINTER(i64)],
            "h2_construct": [vp, vp, i32, vp, dbl, i32, vp, C.POINTER(vp)],
            "h2_hidr_reduce_ex": [vp, i32, i32, i32, vp, C.POINTER(vp)],
            "h2_construct_ex": [vp, vp, i32, vp, dbl, i32, C.POINTER(_ConstructOpts), vp, C.POINTER(vp)],
            "h2_matvec_graph_create": [vp, vp, vp, i32, i32, i64, vp, C.POINTER(vp)],
            "h2_matvec_graph_launch": [vp, vp],
            "h2_autotune_leaf": [vp, i64, i32, i32, vp, i32, i32, i32, vp, dbl, i32, i32, vp, C.POINTER(i32), vp],
            "h2_matrix_get": [vp, i32, vp, i64, C.POINTER(i64)],
            "h2_matvec": [vp, vp, vp, i32, i32, i64, i32, vp],
            "h2_exact_rows": [vp, i32, vp, vp, vp, i64, vp, i32, vp],
            "h2_calibrate": [i32, i32, vp, dbl, vp, i32, vp, i32, i32, vp, C.POINTER(i32), C.POINTER(dbl)],
            "h2_free": [vp],
            "h2_get_stats": [vp, C.c_char_p, i64],
            "h2_sampled_error": [vp, vp, vp, i64, i64, vp, i32, vp],
            "h2_profile": [i32, i32],
            "h2_exact_rows_noalloc": [vp, i32, vp, vp, vp, i64, vp, vp],
            "h2_construct_batched": [i32, vp, vp, vp, vp, vp, vp, vp, vp],
            "h2_debug_fail_alloc": [i64, C.POINTER(i64)],
            "h2_fma_peak": [C.POINTER(dbl), C.POINTER(dbl), vp],
            "h2_tree_build_batched": [i32, vp, vp, i32, i32, vp, vp, vp],
            "h2_hidr_reduce_batched": [i32, vp, vp, vp, vp, vp, vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.h2_last_error.restype = C.c_char_p
        L.h2_last_error.argtypes = []
        _lib = L
    return _lib


def _check(call: str, st: int):
    if st != 0:
        raise H2Error(call, st, lib().h2_last_error().decode(errors="replace"))


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _kid(kernel) -> int:
    return KERNELS[kernel] if isinstance(kernel, str) else int(kernel)


def _kparams(kparams):
    a = (C.c_double * 4)()
    for i, v in enumerate(kparams or ()):
        a[i] = float(v)
    return a


def _is_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and x.is_cuda


def _ptr(x):
    """(pointer, on_device, keepalive) for a torch tensor or numpy array."""
    if _is_cuda(x):
        assert x.is_contiguous()
        return C.c_void_p(x.data_ptr()), 1, x
    a = np.ascontiguousarray(x)
    return a.ctypes.data_as(C.c_void_p), 0, a


def stats(handle) -> str:
    buf = C.create_string_buffer(2048)
    _check("h2_get_stats", lib().h2_get_stats(handle, buf, 2048))
    return buf.value.decode()


class _Handle:
    _h = None

    def free(self):
        if self._h:
            _check("h2_free", lib().h2_free(self._h))
            self._h = None

    def __del__(self):
        try:
            if self._h and _lib is not None:
                _lib.h2_free(self._h)
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def stats(self) -> str:
        return stats(self._h)


class Tree(_Handle):
    """h2_tree_build: Morton cluster tree and near/far interaction lists."""

    @classmethod
    def _wrap(cls, handle):
        t = cls.__new__(cls)
        t._h = handle
        info = t.get("info")
        t.n, t.d, t.B, t.nnodes, t.nlevels, t.nnear, t.nfar, t.q = (int(v) for v in info)
        return t

    def __init__(self, points, leaf_size: int, tau=(7, 10), stream=None):
        if not _is_cuda(points):
            points = np.ascontiguousarray(points, dtype=np.float64)
        n, d = points.shape
        p, on_dev, keep = _ptr(points)
        prm = _Params(int(leaf_size), int(tau[0]), int(tau[1]))
        h = C.c_void_p()
        _check("h2_tree_build", lib().h2_tree_build(p, n, d, on_dev, C.byref(prm), _stream(stream), C.byref(h)))
        self._h = h.value
        info = self.get("info")
        self.n, self.d, self.B, self.nnodes, self.nlevels, self.nnear, self.nfar, self.q = (int(v) for v in info)

    def get(self, what: str) -> np.ndarray:
        code, dt = TREE_FIELDS[what]
        ln = C.c_int64(0)
        _check("h2_tree_get", lib().h2_tree_get(self._h, code, None, 0, C.byref(ln)))
        out = np.zeros(max(ln.value, 1), dtype=dt)
        _check("h2_tree_get", lib().h2_tree_get(self._h, code, out.ctypes.data_as(C.c_void_p), out.size,
                                                 C.byref(ln)))
        return out[:ln.value]


class Hidr(_Handle):
    """h2_hidr_reduce: X_i*, Y_i* of Algorithm 1."""

    @classmethod
    def _wrap(cls, handle, tree):
        h = cls.__new__(cls)
        h._h = handle
        h.tree = tree
        return h

    def __init__(self, tree: Tree, g1: int, g2: int, stream=None, method: str = "volume", il_reduce: bool = False,
                 copy_sets: bool = False):
        """method: the DataReduct of section 3.3, "volume", "surface" or "fps".
        il_reduce: each Y_i* also takes the reduction of its interaction-list
        part alone, on that part's own box (H2_HIDR_IL_REDUCE).  copy_sets:
        the top-down sets are copied out and binned entry by entry
        (H2_HIDR_COPY_SETS; same result)."""
        h = C.c_void_p()
        flags = DR_METHODS[method] | (HIDR_IL_REDUCE if il_reduce else 0) | (HIDR_COPY_SETS if copy_sets else 0)
        _check("h2_hidr_reduce_ex", lib().h2_hidr_reduce_ex(tree.handle, int(g1), int(g2), flags,
                                                             _stream(stream), C.byref(h)))
        self._h = h.value
        self.tree = tree

    def get(self, which: str):
        """(counts[nnodes], data) for which in {'x', 'y'}."""
        w = 0 if which == "x" else 1
        nn = self.tree.nnodes
        counts = np.zeros(nn, dtype=np.int32)
        tot = C.c_int64(0)
        _check("h2_hidr_get", lib().h2_hidr_get(self._h, w, counts.ctypes.data_as(C.c_void_p), None, 0,
                                                 C.byref(tot)))
        data = np.zeros(max(tot.value, 1), dtype=np.int32)
        _check("h2_hidr_get", lib().h2_hidr_get(self._h, w, None, data.ctypes.data_as(C.c_void_p), data.size,
                                                 C.byref(tot)))
        return counts, data[:tot.value]


class H2Matrix(_Handle):
    """h2_construct: nested bases (Algorithm 2); .matvec applies K~."""

    def __init__(self, tree: Tree, hidr: Hidr, kernel, kparams=(), id_tol: float = 1e-6, precision="fp64",
                 stream=None, g_bound: float = 0.0, mem_mode: str = "on_the_fly", mem_fraction: float = 0.0,
                 fp64_products: bool = False, tensor_core_products: bool = False, fp64_qr: bool = False,
                 _handle=None):
        """g_bound = f > 1 bounds ||G||_max by f through exchanges after the
        QR (h2_construct_ex); 0 is the plain column-pivoted ID.  mem_mode:
        "on_the_fly" (coupling and nearfield blocks evaluated in every
        product), "store" (evaluated once and kept; single-vector products
        read them) or "auto" (stored when they fit in the float64 form);
        mem_fraction: the share of free device memory they may take (0: 0.5).
        fp64_products: in the float64 form, evaluate the 3D Coulomb products
        in float64 arithmetic instead of float-float.  tensor_core_products: in
        the mixed form, run the several-right-hand-side nearfield 16 columns at
        a time on the tensor cores.  fp64_qr: in the float64 form, keep the
        QR's trailing updates in float64 arithmetic instead of float-float."""
        if _handle is not None:  # built by construct_batched
            self._h = _handle
            self.tree = tree
            return
        h = C.c_void_p()
        kp = _kparams(kparams)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        opts = _ConstructOpts(float(g_bound), MEM_MODES[mem_mode], float(mem_fraction), int(bool(fp64_products)),
                              int(bool(tensor_core_products)), int(bool(fp64_qr)))
        _check("h2_construct_ex", lib().h2_construct_ex(tree.handle, hidr.handle, _kid(kernel), kp, float(id_tol),
                                                         prec, C.byref(opts), _stream(stream), C.byref(h)))
        self._h = h.value
        self.tree = tree

    def capture_matvec(self, x, y, stream=None) -> "MatvecGraph":
        """h2_matvec_graph_create: y = K~ x recorded as a CUDA graph on these
        device vectors (n entries, float64 or float32, contiguous, one dtype);
        .launch() replays it for x's contents at that time."""
        import torch
        n = self.tree.n
        ok = _is_cuda(x) and _is_cuda(y) and x.dtype == y.dtype and x.dtype in (torch.float64, torch.float32)
        if not ok or x.shape != (n,) or y.shape != (n,) or not (x.is_contiguous() and y.is_contiguous()):
            raise TypeError("x and y must be contiguous CUDA vectors of n entries and one float dtype")
        dt = DTYPE_F64 if x.dtype == torch.float64 else DTYPE_F32
        g = C.c_void_p()
        _check("h2_matvec_graph_create", lib().h2_matvec_graph_create(self._h, C.c_void_p(x.data_ptr()),
                                                                       C.c_void_p(y.data_ptr()), 1, dt, n,
                                                                       _stream(stream), C.byref(g)))
        return MatvecGraph(g.value, self, x, y)

    def get(self, what: str) -> np.ndarray:
        code, dt = MAT_FIELDS[what]
        ln = C.c_int64(0)
        _check("h2_matrix_get", lib().h2_matrix_get(self._h, code, None, 0, C.byref(ln)))
        out = np.zeros(max(ln.value, 1), dtype=dt)
        _check("h2_matrix_get", lib().h2_matrix_get(self._h, code, out.ctypes.data_as(C.c_void_p), out.size,
                                                     C.byref(ln)))
        return out[:ln.value]

    def matvec(self, x, y=None, stream=None):
        """y = K~ x for a vector x of n entries or an n x nrhs matrix of
        right-hand sides, float64 or float32 (y takes x's shape and dtype).  A
        CUDA tensor stays on the device; a host array is copied in and out by
        the library.  y, if given, must be a contiguous vector of x's dtype
        (single right-hand side only)."""
        n = self.tree.n
        if _is_cuda(x):
            import torch
            if x.dtype not in (torch.float64, torch.float32):
                raise TypeError("x must be float64 or float32")
            dt = DTYPE_F64 if x.dtype == torch.float64 else DTYPE_F32
            if x.dim() == 1:
                xc = x.contiguous()
                if y is None:
                    y = torch.empty_like(xc)
                _check("h2_matvec", lib().h2_matvec(self._h, C.c_void_p(xc.data_ptr()), C.c_void_p(y.data_ptr()), 1,
                                                     dt, n, 1, _stream(stream)))
                return y
            nrhs = x.shape[1]
            xt = x.t().contiguous()  # column-major n x nrhs, ld = n
            yt = torch.empty_like(xt)
            _check("h2_matvec", lib().h2_matvec(self._h, C.c_void_p(xt.data_ptr()), C.c_void_p(yt.data_ptr()), nrhs,
                                                 dt, n, 1, _stream(stream)))
            return yt.t()
        xa = np.asarray(x)
        fdt = np.float32 if xa.dtype == np.float32 else np.float64
        dt = DTYPE_F32 if fdt == np.float32 else DTYPE_F64
        nrhs = 1 if xa.ndim == 1 else xa.shape[1]
        xa = np.asfortranarray(xa, dtype=fdt)
        ya = np.zeros_like(xa, order="F") if y is None or xa.ndim == 2 else y
        _check("h2_matvec", lib().h2_matvec(self._h, xa.ctypes.data_as(C.c_void_p), ya.ctypes.data_as(C.c_void_p),
                                             nrhs, dt, n, 0, _stream(stream)))
        return ya


class MatvecGraph(_Handle):
    """A product recorded by H2Matrix.capture_matvec; holds its matrix and
    buffers alive."""

    def __init__(self, handle, A, x, y):
        self._h = handle
        self.A, self.x, self.y = A, x, y

    def launch(self, stream=None):
        _check("h2_matvec_graph_launch", lib().h2_matvec_graph_launch(self._h, _stream(stream)))
        return self.y


def tree_build(points, leaf_size, tau=(7, 10), stream=None) -> Tree:
    return Tree(points, leaf_size, tau, stream)


def hidr_reduce(tree, g1, g2, stream=None) -> Hidr:
    return Hidr(tree, g1, g2, stream)


def construct(tree, hidr, kernel, kparams=(), id_tol=1e-6, precision="fp64", stream=None) -> H2Matrix:
    return H2Matrix(tree, hidr, kernel, kparams, id_tol, precision, stream)


def tree_build_batched(points_list, leaf_sizes, tau=(7, 10), stream=None):
    """h2_tree_build_batched: one tree per point set (CUDA tensors, or host
    arrays; not mixed), leaf_sizes per set (or one for all), built
    concurrently on the GPU."""
    n = len(points_list)
    if n == 0:
        return []
    on_dev = _is_cuda(points_list[0])
    if any(_is_cuda(p) != on_dev for p in points_list):
        raise TypeError("point sets must be all CUDA tensors or all host arrays")
    keep = [p.contiguous() if on_dev else np.ascontiguousarray(p, dtype=np.float64) for p in points_list]
    d = keep[0].shape[1]
    if any(p.shape[1] != d for p in keep):
        raise ValueError("every point set needs the same dimension")
    ptrs = (C.c_void_p * n)(*[p.data_ptr() if on_dev else p.ctypes.data for p in keep])
    ns = (C.c_int64 * n)(*[p.shape[0] for p in keep])
    qs = [leaf_sizes] * n if isinstance(leaf_sizes, int) else list(leaf_sizes)
    prm = (_Params * n)(*[_Params(int(q), int(tau[0]), int(tau[1])) for q in qs])
    outs = (C.c_void_p * n)()
    _check("h2_tree_build_batched", lib().h2_tree_build_batched(n, ptrs, ns, d, int(on_dev), prm, _stream(stream),
                                                                 outs))
    return [Tree._wrap(outs[i]) for i in range(n)]


def hidr_reduce_batched(trees, g1s, g2s, il_reduce=False, method="volume", stream=None):
    """h2_hidr_reduce_batched: one Hidr per tree (g1, g2 per tree or one for
    all), reduced concurrently on the GPU."""
    n = len(trees)
    if n == 0:
        return []
    g1 = [g1s] * n if isinstance(g1s, int) else list(g1s)
    g2 = [g2s] * n if isinstance(g2s, int) else list(g2s)
    flags = DR_METHODS[method] | (HIDR_IL_REDUCE if il_reduce else 0)
    th = (C.c_void_p * n)(*[t.handle for t in trees])
    outs = (C.c_void_p * n)()
    _check("h2_hidr_reduce_batched", lib().h2_hidr_reduce_batched(n, th, (C.c_int * n)(*g1), (C.c_int * n)(*g2),
                                                                   (C.c_int * n)(*([flags] * n)), _stream(stream),
                                                                   outs))
    return [Hidr._wrap(outs[i], trees[i]) for i in range(n)]


def construct_batched(problems, stream=None):
    """h2_construct_batched: problems is a list of (tree, hidr, kernel,
    kparams, id_tol, precision); returns one H2Matrix per problem, built
    concurrently on the GPU."""
    n = len(problems)
    if n == 0:
        return []
    trees = (C.c_void_p * n)(*[p[0].handle for p in problems])
    hidrs = (C.c_void_p * n)(*[p[1].handle for p in problems])
    kids = (C.c_int * n)(*[_kid(p[2]) for p in problems])
    kps = (C.c_double * (4 * n))()
    for i, p in enumerate(problems):
        for a, v in enumerate(tuple(p[3])[:4]):
            kps[4 * i + a] = float(v)
    tols = (C.c_double * n)(*[float(p[4]) for p in problems])
    precs = (C.c_int * n)(*[PRECISIONS[p[5]] if isinstance(p[5], str) else int(p[5]) for p in problems])
    outs = (C.c_void_p * n)()
    _check("h2_construct_batched", lib().h2_construct_batched(n, trees, hidrs, kids, kps, tols, precs,
                                                               _stream(stream), outs))
    return [H2Matrix(p[0], p[1], p[2], _handle=outs[i]) for i, p in enumerate(problems)]


def autotune_leaf(points, candidates=(64, 128, 256), g=7, kernel="coulomb", kparams=(), id_tol=1e-5,
                  precision="mixed", reps=2, stream=None):
    """h2_autotune_leaf: the leaf size among candidates with the least device
    time of tree + HiDR + construction + one matvec on points (a CUDA tensor
    or host array, n x d float64).  Returns (best, {q: ms})."""
    c = list(candidates)
    cands = (C.c_int * len(c))(*c)
    times = (C.c_double * len(c))()
    best = C.c_int(0)
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    if _is_cuda(points):
        pts = points.contiguous()
        ptr, on_dev = C.c_void_p(pts.data_ptr()), 1
    else:
        pts = np.ascontiguousarray(points, dtype=np.float64)
        ptr, on_dev = pts.ctypes.data_as(C.c_void_p), 0
    n, d = pts.shape
    _check("h2_autotune_leaf", lib().h2_autotune_leaf(ptr, n, d, on_dev, cands, len(c), int(g), _kid(kernel),
                                                       _kparams(kparams), float(id_tol), prec, int(reps),
                                                       _stream(stream), C.byref(best), times))
    return best.value, {q: times[i] for i, q in enumerate(c)}


def matvec(A: H2Matrix, x, y=None, stream=None):
    return A.matvec(x, y, stream)


def exact_rows(tree: Tree, kernel, kparams, z, rows, out=None, stream=None):
    """(K z)_s for s in rows, float64 sums on the GPU."""
    kp = _kparams(kparams)
    if _is_cuda(z):
        import torch
        if out is None:
            out = torch.empty(len(rows), dtype=torch.float64, device=z.device)
        _check("h2_exact_rows", lib().h2_exact_rows(tree.handle, _kid(kernel), kp, C.c_void_p(z.data_ptr()),
                                                     C.c_void_p(rows.data_ptr()), len(rows),
                                                     C.c_void_p(out.data_ptr()), 1, _stream(stream)))
        return out
    za = np.ascontiguousarray(z, dtype=np.float64)
    ra = np.ascontiguousarray(rows, dtype=np.int64)
    oa = np.zeros(len(ra))
    _check("h2_exact_rows", lib().h2_exact_rows(tree.handle, _kid(kernel), kp, za.ctypes.data_as(C.c_void_p),
                                                 ra.ctypes.data_as(C.c_void_p), len(ra),
                                                 oa.ctypes.data_as(C.c_void_p), 0, _stream(stream)))
    return oa


def calibrate(dim, kernel, kparams, eps, z1, z2, gmax=16, stream=None):
    """Section 4.2: smallest g (r1 = r2 = g^dim) meeting the test; (g, error)."""
    kp = _kparams(kparams)
    a1 = np.ascontiguousarray(z1, dtype=np.float64)
    a2 = np.ascontiguousarray(z2, dtype=np.float64)
    g = C.c_int(0)
    err = C.c_double(0.0)
    _check("h2_calibrate", lib().h2_calibrate(int(dim), _kid(kernel), kp, float(eps), a1.ctypes.data_as(C.c_void_p),
                                               len(a1), a2.ctypes.data_as(C.c_void_p), len(a2), int(gmax),
                                               _stream(stream), C.byref(g), C.byref(err)))
    return g.value, err.value


def free(handle_obj):
    handle_obj.free()


def sampled_error(exact, approx, rows, stream=None):
    """||exact - approx[rows]|| / ||exact|| (section 6 metric on sampled rows).
    CUDA tensors give a CUDA scalar tensor; host arrays give a float."""
    L = lib()
    if _is_cuda(exact):
        import torch
        out = torch.empty(1, dtype=torch.float64, device=exact.device)
        _check("h2_sampled_error", L.h2_sampled_error(C.c_void_p(exact.data_ptr()), C.c_void_p(approx.data_ptr()),
                                                       C.c_void_p(rows.data_ptr()), len(rows), approx.numel(),
                                                       C.c_void_p(out.data_ptr()), 1, _stream(stream)))
        return out
    e = np.ascontiguousarray(exact, dtype=np.float64)
    a = np.ascontiguousarray(approx, dtype=np.float64)
    r = np.ascontiguousarray(rows, dtype=np.int64)
    out = C.c_double(0.0)
    _check("h2_sampled_error", L.h2_sampled_error(e.ctypes.data_as(C.c_void_p), a.ctypes.data_as(C.c_void_p),
                                                   r.ctypes.data_as(C.c_void_p), len(r), len(a), C.byref(out), 0,
                                                   _stream(stream)))
    return out.value


def profile(enable: bool = True, reset: bool = True):
    """Turn per-kernel CUDA-event timing on or off (and zero its totals)."""
    _check("h2_profile", lib().h2_profile(int(enable), int(reset)))


def _global_stats() -> dict:
    import json
    buf = C.create_string_buffer(8192)
    _check("h2_get_stats", lib().h2_get_stats(None, buf, 8192))
    return json.loads(buf.value.decode())


def kernel_times() -> dict:
    """{kernel: {"ms": total, "launches": n}} collected while profiling."""
    st = _global_stats()
    st.pop("launches_total", None)
    return st


def debug_fail_alloc(k: int) -> int:
    """Arm the library's k-th device allocation from now on to fail with
    H2_ERR_OOM (0 disarms); returns the allocations made since the last call."""
    made = C.c_int64(0)
    _check("h2_debug_fail_alloc", lib().h2_debug_fail_alloc(int(k), C.byref(made)))
    return made.value


def fma_peak(stream=None):
    """(float64, float32) fused multiply-add throughput of this GPU, TFLOP/s."""
    a, b = C.c_double(0.0), C.c_double(0.0)
    _check("h2_fma_peak", lib().h2_fma_peak(C.byref(a), C.byref(b), _stream(stream)))
    return a.value, b.value


def launches_total() -> int:
    """Kernel launches the library has made in this process."""
    return int(_global_stats()["launches_total"])
