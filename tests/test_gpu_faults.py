"""Error paths under device-allocation failure, injected on the host.

h2_debug_fail_alloc makes the k-th device allocation fail as if the device
were out of memory.  For every entry point that allocates (tree build, HiDR,
construction, matvec, exact rows) and for each of its allocations in turn,
the call must return H2_ERR_OOM, hand out no handle, and leave the context
and the existing handles usable: after each failure the same call, disarmed,
succeeds and its result equals the one computed before any failure (tree and
HiDR bit for bit, the product within 1e-14 row by row).  No GPU fault is
involved: the failure happens on the host before the allocator is called."""
import ctypes as C

import numpy as np
import pytest

from paper_2206_01885_gb300 import inputs as I
from rowcheck import assert_rows_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

OOM = 2


@pytest.fixture(scope="module")
def H2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_01885_gb300 import build as B
    B.build()
    from paper_2206_01885_gb300 import h2
    yield h2
    h2.debug_fail_alloc(0)


def _points():
    return torch.from_numpy(I.uniform_cube(3000, 3, seed=901)).cuda()


def _ks(count, cap=40):
    """every allocation index of a call, or an even spread of them plus both ends"""
    if count <= cap:
        return list(range(1, count + 1))
    return sorted(set(np.linspace(1, count, cap).round().astype(int).tolist()))


def _failing_calls(H2, make, check):
    """Count the allocations of make(); then fail each in turn and check the
    status, the absent handle and a clean retry."""
    H2.debug_fail_alloc(0)
    good = make()
    count = H2.debug_fail_alloc(0)
    assert count >= 1
    check(good)
    for k in _ks(count):
        H2.debug_fail_alloc(k)
        st, handle = make(raw=True)
        msg = H2.lib().h2_last_error()  # (read before the next call resets it)
        H2.debug_fail_alloc(0)
        assert st == OOM, (k, st, msg)
        assert b"injected" in msg, (k, msg)
        assert handle is None, k
        torch.cuda.synchronize()  # the context still works
        check(make())
    return count


def test_tree_build_oom(H2):
    P = _points()
    ref = H2.Tree(P, 64)
    want = {f: ref.get(f) for f in ("perm", "near_idx", "far_idx", "lptr")}

    def make(raw=False):
        if not raw:
            return H2.Tree(P, 64)
        prm = H2._Params(64, 7, 10)
        out = C.c_void_p()
        st = H2.lib().h2_tree_build(C.c_void_p(P.data_ptr()), P.shape[0], 3, 1, C.byref(prm), None, C.byref(out))
        return st, out.value

    def check(t):
        for f, w in want.items():
            assert np.array_equal(t.get(f), w), f
        t.free()

    _failing_calls(H2, make, check)


@pytest.mark.parametrize("il_reduce", [False, True])
def test_hidr_reduce_oom(H2, il_reduce):
    t = H2.Tree(_points(), 64)
    ref = H2.Hidr(t, 4, 5, il_reduce=il_reduce)
    want = [ref.get(w) for w in ("x", "y")]
    ref.free()
    flags = H2.HIDR_IL_REDUCE if il_reduce else 0

    def make(raw=False):
        if not raw:
            return H2.Hidr(t, 4, 5, il_reduce=il_reduce)
        out = C.c_void_p()
        st = H2.lib().h2_hidr_reduce_ex(t.handle, 4, 5, flags, None, C.byref(out))
        return st, out.value

    def check(h):
        for (c, d), (wc, wd) in zip([h.get(w) for w in ("x", "y")], want):
            assert np.array_equal(c, wc) and np.array_equal(d, wd)
        h.free()

    _failing_calls(H2, make, check)
    t.free()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_construct_and_matvec_oom(H2, prec):
    P = _points()
    t = H2.Tree(P, 64)
    hd = H2.Hidr(t, 4, 4)
    z = torch.from_numpy(I.standard_normal(3000, seed=902)).cuda()
    ref = H2.H2Matrix(t, hd, "coulomb", (), 1e-6, prec)
    want_y = ref.matvec(z).cpu().numpy()
    want_k = ref.get("rank")
    ref.free()
    pcode = H2.PRECISIONS[prec]

    def make(raw=False):
        if not raw:
            return H2.H2Matrix(t, hd, "coulomb", (), 1e-6, prec)
        out = C.c_void_p()
        st = H2.lib().h2_construct(t.handle, hd.handle, H2.KERNELS["coulomb"], None, 1e-6, pcode, None,
                                   C.byref(out))
        return st, out.value

    def check(A):
        assert np.array_equal(A.get("rank"), want_k)
        assert_rows_close(A.matvec(z).cpu().numpy(), want_y, 1e-14, "product after a failed construction")
        A.free()

    _failing_calls(H2, make, check)

    # the first product of a fresh matrix builds its coupling tiles: fail each
    # of that product's allocations, on a fresh matrix every time
    y = torch.empty_like(z)

    def first_product(A, k):
        H2.debug_fail_alloc(k)
        y.fill_(float("nan"))
        st = H2.lib().h2_matvec(A.handle, C.c_void_p(z.data_ptr()), C.c_void_p(y.data_ptr()), 1,
                                H2.DTYPE_F64, 3000, 1, None)
        return st, H2.debug_fail_alloc(0)

    A = H2.H2Matrix(t, hd, "coulomb", (), 1e-6, prec)
    st, first = first_product(A, 0)
    assert st == 0 and first >= 1
    A.free()
    for k in range(1, first + 1):
        A = H2.H2Matrix(t, hd, "coulomb", (), 1e-6, prec)
        H2.debug_fail_alloc(k)
        y.fill_(float("nan"))
        st = H2.lib().h2_matvec(A.handle, C.c_void_p(z.data_ptr()), C.c_void_p(y.data_ptr()), 1,
                                H2.DTYPE_F64, 3000, 1, None)
        msg = H2.lib().h2_last_error()
        H2.debug_fail_alloc(0)
        assert st == OOM and b"injected" in msg, (k, st, msg)
        torch.cuda.synchronize()
        assert_rows_close(A.matvec(z).cpu().numpy(), want_y, 1e-14, f"product after failed allocation {k}")
        A.free()
    hd.free()
    t.free()


def test_exact_rows_oom_host_buffers(H2):
    """The host-buffer exact rows stage z, rows and out on the device."""
    pts = I.uniform_cube(3000, 3, seed=903)
    t = H2.Tree(torch.from_numpy(pts).cuda(), 64)
    z = I.standard_normal(3000, seed=904)
    rows = I.sample_rows(3000, 40, seed=905)
    want = H2.exact_rows(t, "coulomb", (), z, rows)
    count = H2.debug_fail_alloc(0)
    H2.exact_rows(t, "coulomb", (), z, rows)
    count = H2.debug_fail_alloc(0)
    assert count >= 1
    for k in range(1, count + 1):
        H2.debug_fail_alloc(k)
        with pytest.raises(H2.H2Error) as e:
            H2.exact_rows(t, "coulomb", (), z, rows)
        H2.debug_fail_alloc(0)
        assert e.value.status == OOM, k
        assert np.array_equal(H2.exact_rows(t, "coulomb", (), z, rows), want)
    t.free()


def test_construct_with_stored_blocks_oom(H2):
    """Each allocation of a construction that stores its coupling and
    nearfield blocks (memory mode STORE), the block buffers included."""
    P = _points()
    t = H2.Tree(P, 64)
    hd = H2.Hidr(t, 4, 4)
    z = torch.from_numpy(I.standard_normal(3000, seed=906)).cuda()
    ref = H2.H2Matrix(t, hd, "coulomb", (), 1e-6, "fp64")
    want_y = ref.matvec(z).cpu().numpy()
    ref.free()
    opts = H2._ConstructOpts(0.0, H2.MEM_MODES["store"], 0.0)

    def make(raw=False):
        if not raw:
            return H2.H2Matrix(t, hd, "coulomb", (), 1e-6, "fp64", mem_mode="store")
        out = C.c_void_p()
        st = H2.lib().h2_construct_ex(t.handle, hd.handle, H2.KERNELS["coulomb"], None, 1e-6, 0, C.byref(opts),
                                      None, C.byref(out))
        return st, out.value

    def check(A):
        assert '"stored"' in A.stats()
        assert_rows_close(A.matvec(z).cpu().numpy(), want_y, 1e-13, "stored product after a failed construction")
        A.free()

    _failing_calls(H2, make, check)
    hd.free()
    t.free()
