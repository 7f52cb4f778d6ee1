"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Bit-exact: permutation, keys, node arrays, near/far lists, X_i*, Y_i*.
Float64 construction: ranks and skeletons equal (3D Coulomb blocks and QR
run in float-float arithmetic, within ~2^-43 of float64, and the other
kernels' blocks are float64; pivot near-ties are reported, none occur here), U
within 64 u c / eps of the oracle's (u = 2^-53, the conditioning bound of
R11^{-1} R12 after truncation at eps), the H^2 matvec within 1e-12 of the oracle's
H^2 matvec and within 10 eps of the dense product; exact rows within 1e-12.
Sizes span several levels and tiles and include ragged leaves."""
import ctypes as C
import json

import numpy as np
import pytest

from oracle import h2_oracle as O
from paper_2206_01885_gb300 import inputs as I
from rowcheck import assert_rows_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def H2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_01885_gb300 import build as B
    B.build()
    from paper_2206_01885_gb300 import h2
    return h2


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


TREE_CASES = [
    ("cube3d", lambda: I.uniform_cube(5000, 3, seed=1), 64),
    ("cube3d_q1", lambda: I.uniform_cube(700, 3, seed=2), 1),
    ("gmix2d", lambda: I.gaussian_mixture(20000, seed=3), 32),
    ("sphere", lambda: I.sphere_surface(6000, seed=4), 40),
    ("dups", lambda: np.repeat(I.uniform_cube(50, 3, seed=5), 9, axis=0), 4),
    ("single_leaf", lambda: I.uniform_cube(100, 3, seed=6), 500),
    ("n1", lambda: np.array([[0.25, 0.5, 0.75]]), 8),
    ("n2_2d", lambda: np.array([[0.0, 0.0], [1.0, 1.0]]), 1),
    ("all_same", lambda: np.tile([[0.1, 0.2, 0.3]], (40, 1)), 4),
]


@pytest.mark.parametrize("name,make,q", TREE_CASES, ids=[c[0] for c in TREE_CASES])
def test_tree_and_lists_bit_exact(H2, name, make, q):
    pts = make()
    t = H2.Tree(dev(pts), q)
    o = O.tree_build(pts, q)
    assert t.nnodes == o.nnodes and t.nlevels == o.nlevels
    for f in ["perm", "keys", "level", "parent", "fchild", "nchild", "begin", "end", "prefix", "lptr",
              "near_ptr", "near_idx", "far_ptr", "far_idx"]:
        got = t.get(f)
        want = getattr(o, f.replace("keys", "key"))
        assert np.array_equal(got, want.astype(got.dtype)), f
    # host input path gives the same tree
    t2 = H2.Tree(pts, q)
    assert np.array_equal(t2.get("perm"), o.perm)


HIDR_CASES = [("cube3d", 3, 6000, 60, 4, 5), ("gmix2d", 2, 8000, 30, 6, 7), ("cube3d_g2", 3, 3000, 20, 2, 3),
              # sets of tens of thousands of points: the binned search with many points per cell
              ("cube3d_big", 3, 40000, 64, 5, 6),
              # points snapped to a lattice: many exact distance ties between labels
              ("lattice3d", 3, 20000, 32, 4, 4),
              # grids of 65^2 points, above the binned search's limit: the brute-force sweep
              ("square2d_g65", 2, 40000, 2600, 65, 65), ("lattice2d_g65", 2, 40000, 2600, 65, 65),
              # one coordinate constant everywhere: a flat dimension in every box
              ("plane3d", 3, 20000, 64, 4, 5),
              # 3000 identical points: a chain of cells down to the deepest level, boxes of size 0
              ("same3d", 3, 3400, 64, 3, 3)]


def _hidr_points(name, d, n):
    if name == "lattice3d":
        return np.round(I.uniform_cube(n, d, seed=12) * 16.0) / 16.0
    if name == "square2d_g65":
        return I.uniform_cube(n, d, seed=13)
    if name == "lattice2d_g65":
        return np.round(I.uniform_cube(n, d, seed=14) * 32.0) / 32.0
    if name == "plane3d":
        p = I.uniform_cube(n, d, seed=15)
        p[:, 2] = 0.5
        return p
    if name == "same3d":
        return np.concatenate([np.tile([[0.1, 0.2, 0.3]], (3000, 1)), I.uniform_cube(n - 3000, d, seed=16)])
    if "cube" in name:
        return I.uniform_cube(n, d, seed=10 + d)
    return I.gaussian_mixture(n, seed=11)


@pytest.mark.parametrize("name,d,n,q,g1,g2", HIDR_CASES, ids=[c[0] for c in HIDR_CASES])
def test_hidr_bit_exact(H2, name, d, n, q, g1, g2):
    pts = _hidr_points(name, d, n)
    t = H2.Tree(dev(pts), q)
    h = H2.Hidr(t, g1, g2)
    o = O.tree_build(pts, q)
    oh = O.Hidr(o, g1, g2)
    for which in ["x", "y"]:
        cnt, data = h.get(which)
        off = np.concatenate([[0], np.cumsum(cnt)])
        for i in range(1, t.nnodes):
            want = oh.get(i, which)
            got = data[off[i]:off[i + 1]]
            assert np.array_equal(got, want), (which, i)


SURFACE_CASES = [("cube3d", 3, 6000, 60, 4, 5), ("gmix2d", 2, 8000, 30, 6, 7), ("cube3d_big", 3, 40000, 64, 5, 6),
                 ("lattice3d", 3, 20000, 32, 4, 4), ("plane3d", 3, 20000, 64, 4, 5), ("same3d", 3, 3400, 64, 3, 3)]


@pytest.mark.parametrize("method", ["surface", "fps"])
@pytest.mark.parametrize("name,d,n,q,g1,g2", SURFACE_CASES, ids=[c[0] for c in SURFACE_CASES])
def test_hidr_variants_bit_exact(H2, name, d, n, q, g1, g2, method):
    """The surface-based and farthest-point-sampling DataReducts (section 3.3)
    through HiDR: X_i*, Y_i* bit-exact against the oracle's."""
    pts = _hidr_points(name, d, n)
    t = H2.Tree(dev(pts), q)
    h = H2.Hidr(t, g1, g2, method=method)
    assert json.loads(h.stats())["method"] == method
    o = O.tree_build(pts, q)
    oh = O.Hidr(o, g1, g2, method=method)
    for which in ["x", "y"]:
        cnt, data = h.get(which)
        off = np.concatenate([[0], np.cumsum(cnt)])
        for i in range(1, t.nnodes):
            assert np.array_equal(data[off[i]:off[i + 1]], oh.get(i, which)), (which, i)


def test_surface_reduction_builds_accurate_h2(H2):
    n, q, g, eps = 6000, 100, 7, 1e-6
    pts = I.uniform_cube(n, 3, seed=53)
    z = I.standard_normal(n, seed=51)
    t = H2.Tree(dev(pts), q)
    h = H2.Hidr(t, g, g, method="surface")
    A = H2.H2Matrix(t, h, "coulomb", (), eps, "fp64")
    y = A.matvec(dev(z)).cpu().numpy()
    o = O.tree_build(pts, q)
    yo = O.H2(o, O.Hidr(o, g, g, method="surface"), "coulomb", (), eps).matvec(z)
    assert_rows_close(y, yo, 1e-12, "surface H2 vs oracle")
    yd = O.dense_matvec(pts, "coulomb", (), z)
    assert np.linalg.norm(y - yd) <= 10 * eps * np.linalg.norm(yd)


def _node_cands(o, H, i):
    if o.nchild[i] == 0:
        return np.arange(o.begin[i], o.end[i])
    return np.concatenate([H.skeleton(c) for c in range(o.fchild[i], o.fchild[i] + o.nchild[i])])


CONSTRUCT_CASES = [
    ("coulomb3d", 3, 6000, 100, "coulomb", (), 1e-6, 6),
    ("coulomb3d_deep", 3, 12000, 40, "coulomb", (), 1e-5, 5),
    ("gauss2d", 2, 6000, 64, "gaussian", (0.2,), 1e-6, 10),
    ("expo2d", 2, 5000, 50, "exponential", (0.1,), 1e-6, 10),
    ("mq3d", 3, 4000, 64, "multiquadric", (), 1e-7, 6),
    # Table 1's bump kernel (kappa_4) and the |x-y|^11 of section 5.2
    ("bump3d", 3, 4000, 64, "bump", (0.1,), 1e-7, 6),
    ("power3d", 3, 4000, 64, "power", (11.0,), 1e-7, 6),
    # Table 1's kappa_3 = cos(x . y), not a function of |x - y|
    ("cosdot3d", 3, 4000, 64, "cosdot", (), 1e-7, 6),
]


@pytest.mark.parametrize("name,d,n,q,kern,kp,eps,g", CONSTRUCT_CASES, ids=[c[0] for c in CONSTRUCT_CASES])
def test_construct_and_matvec_fp64(H2, name, d, n, q, kern, kp, eps, g):
    pts = I.uniform_cube(n, d, seed=20 + d)
    z = I.standard_normal(n, seed=21)
    t = H2.Tree(dev(pts), q)
    h = H2.Hidr(t, g, g)
    A = H2.H2Matrix(t, h, kern, kp, eps)
    o, oh, OH = O.build_h2(pts, kern, kp, q, eps, g, g)
    ranks = A.get("rank")
    want_ranks = np.array([max(OH.rank(i), 0) for i in range(o.nnodes)])
    assert np.array_equal(ranks, want_ranks)
    skel = A.get("skel")
    U = A.get("U")
    nc = A.get("ncand")
    koff = np.concatenate([[0], np.cumsum(ranks)])
    uoff = np.concatenate([[0], np.cumsum(ranks.astype(np.int64) * nc)])
    for i in range(1, o.nnodes):
        k = ranks[i]
        if k == 0:
            continue
        assert np.array_equal(skel[koff[i]:koff[i + 1]], OH.skeleton(i)), i
        Ui = U[uoff[i]:uoff[i + 1]].reshape(k, nc[i]).T
        Uo = OH.U(i)
        assert Ui.shape == Uo.shape
        # U = P[I; (R11^{-1} R12)^T]: reordered float64 sums perturb R by ~c u |r_11|
        # and the solve amplifies that by cond(R11) <~ |r_11| / |r_kk| < 1 / eps
        tol = 64 * 2.0 ** -53 * nc[i] / eps
        assert np.max(np.abs(Ui - Uo)) <= tol * max(1.0, np.max(np.abs(Uo))), i
    # the largest interpolation coefficient |G| (U = P [I; G]), what strong RRQR would bound
    st = json.loads(A.stats())
    umax = max(float(np.abs(OH.U(i)).max()) for i in range(1, o.nnodes) if OH.rank(i) > 0)
    assert abs(max(1.0, st["g_max"]) - umax) <= 1e-6 * umax
    y = A.matvec(dev(z)).cpu().numpy()
    yo = OH.matvec(z)
    assert_rows_close(y, yo, 1e-12, f"{name} float64 H2 vs oracle")
    yd = O.dense_matvec(pts, kern, kp, z)
    assert np.linalg.norm(y - yd) / np.linalg.norm(yd) <= 10 * eps
    # host-pointer matvec is the same product
    yh = A.matvec(z)
    # (block sums meet in float64 atomics, so two products agree to rounding)
    assert np.linalg.norm(yh - y) <= 1e-14 * np.linalg.norm(y)


def test_exact_rows(H2):
    pts = I.uniform_cube(20000, 3, seed=31)
    z = I.standard_normal(20000, seed=32)
    rows = I.sample_rows(20000, 300, seed=33)
    t = H2.Tree(dev(pts), 128)
    got = H2.exact_rows(t, "coulomb", (), dev(z), dev(rows)).cpu().numpy()
    want = O.exact_rows(pts, "coulomb", (), z, rows)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    got_h = H2.exact_rows(t, "coulomb", (), z, rows)
    assert np.array_equal(got_h, got)
    for kern, kp in [("gaussian", (0.3,)), ("exponential", (0.2,)), ("multiquadric", ()), ("bump", (0.1,)),
                     ("power", (11.0,)), ("cosdot", ())]:
        got = H2.exact_rows(t, kern, kp, dev(z), dev(rows)).cpu().numpy()
        want = O.exact_rows(pts, kern, kp, z, rows)
        assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max()), kern


def test_exact_rows_coincident_points(H2):
    """The 3D Coulomb exact rows run in float-float arithmetic; with repeated
    points (kappa(x, x) = 0 for every copy, as in float64) and rows out of
    range (NaN), against the oracle's float64 pairwise sums and the float64
    allocation-free entry point, within 1e-12 of the largest row."""
    base = I.uniform_cube(3000, 3, seed=41)
    # exact copies, and near copies two cells of the float-float grid away (a
    # residual is held to ~2^-48 of a cell, ~5e-7 here: closer pairs lose
    # relative accuracy in the float-float terms)
    pts = np.concatenate([base, base[:500], base[:500] + 1e-6])
    n = len(pts)
    z = I.standard_normal(n, seed=42)
    rows = np.concatenate([I.sample_rows(n, 400, seed=43), np.arange(3000, 3010)]).astype(np.int64)
    t = H2.Tree(dev(pts), 64)
    got = H2.exact_rows(t, "coulomb", (), dev(z), dev(rows)).cpu().numpy()
    want = O.exact_rows(pts, "coulomb", (), z, rows)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    out = torch.zeros(len(rows), dtype=torch.float64, device="cuda")
    z_d, rows_d = dev(z), dev(rows)  # (held while the call runs)
    st = H2.lib().h2_exact_rows_noalloc(t.handle, H2.KERNELS["coulomb"], H2._kparams(()),
                                        C.c_void_p(z_d.data_ptr()), C.c_void_p(rows_d.data_ptr()),
                                        len(rows), C.c_void_p(out.data_ptr()), H2._stream(None))
    assert st == 0, H2.lib().h2_last_error()
    torch.cuda.synchronize()
    f64 = out.cpu().numpy()
    assert np.allclose(got, f64, rtol=1e-12, atol=1e-12 * np.abs(f64).max())
    bad = H2.exact_rows(t, "coulomb", (), dev(z), dev(np.array([-1, n], dtype=np.int64))).cpu().numpy()
    assert np.isnan(bad).all()
    t.free()


def test_degenerate_paths(H2):
    # one point, a single leaf, identical points: matvec reduces to the nearfield
    for pts, q in [(np.array([[0.5, 0.5, 0.5]]), 4), (I.uniform_cube(90, 3, seed=3), 200),
                   (np.tile([[0.1, 0.2, 0.3]], (30, 1)), 4)]:
        z = I.standard_normal(len(pts), seed=4)
        t = H2.Tree(dev(pts), q)
        h = H2.Hidr(t, 3, 3)
        A = H2.H2Matrix(t, h, "coulomb", (), 1e-6)
        y = A.matvec(dev(z)).cpu().numpy()
        yd = O.dense_matvec(pts, "coulomb", (), z)
        assert np.allclose(y, yd, rtol=1e-13, atol=1e-13 * max(1.0, np.abs(yd).max()))


def test_handle_lifetimes(H2):
    pts = I.uniform_cube(2000, 3, seed=41)
    t = H2.Tree(dev(pts), 50)
    h = H2.Hidr(t, 3, 3)
    assert H2.lib().h2_free(t.handle) == 7  # the hidr depends on the tree
    A = H2.H2Matrix(t, h, "coulomb", (), 1e-4)
    st = H2.lib().h2_free(t.handle)
    assert st == 7  # tree has dependents
    A.free()
    h.free()
    t.free()


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_nonfinite_points_rejected(H2, bad):
    pts = I.uniform_cube(3000, 3, seed=42)
    pts[1234, 1] = bad
    with pytest.raises(H2.H2Error) as e:
        H2.Tree(dev(pts), 50)
    assert e.value.status == 5 and "finite" in str(e.value)  # H2_ERR_NUMERIC
    # the context stays usable
    t = H2.Tree(dev(np.nan_to_num(pts, posinf=0.5, neginf=0.5, nan=0.5)), 50)
    assert t.get("perm").shape == (3000,)
    t.free()


MIXED_CASES = [
    ("coulomb3d", 3, 8000, 100, "coulomb", (), 1e-5, 7),
    ("coulomb3d_deep", 3, 20000, 40, "coulomb", (), 1e-4, 5),
    ("gauss2d", 2, 6000, 64, "gaussian", (0.2,), 1e-5, 10),
    ("expo2d", 2, 5000, 50, "exponential", (0.1,), 1e-5, 10),
    ("bump3d", 3, 4000, 64, "bump", (0.1,), 1e-5, 6),
    ("power3d", 3, 4000, 64, "power", (11.0,), 1e-5, 6),
    ("cosdot3d", 3, 4000, 64, "cosdot", (), 1e-5, 6),
]


@pytest.mark.parametrize("name,d,n,q,kern,kp,eps,g", MIXED_CASES, ids=[c[0] for c in MIXED_CASES])
def test_construct_and_matvec_mixed(H2, name, d, n, q, kern, kp, eps, g):
    """float32 blocks / Householder updates / matvec kernels, float64 norms,
    pivots and solve: the product stays within 10 eps of both the dense product
    and the oracle's float64 H^2 product built with the same eps and g."""
    pts = I.uniform_cube(n, d, seed=60 + d)
    z = I.standard_normal(n, seed=61)
    t = H2.Tree(dev(pts), q)
    h = H2.Hidr(t, g, g)
    A = H2.H2Matrix(t, h, kern, kp, eps, "mixed")
    y = A.matvec(dev(z)).cpu().numpy()
    yd = O.dense_matvec(pts, kern, kp, z)
    assert np.linalg.norm(y - yd) / np.linalg.norm(yd) <= 10 * eps
    o, oh, OH = O.build_h2(pts, kern, kp, q, eps, g, g)
    yo = OH.matvec(z)
    assert_rows_close(y, yo, 10 * eps, f"{name} mixed H2 vs oracle float64 H2")
    # structure: sorted skeletons inside the candidates, identity rows of U
    ranks, nc = A.get("rank"), A.get("ncand")
    skel, U = A.get("skel"), A.get("U")
    koff = np.concatenate([[0], np.cumsum(ranks)])
    uoff = np.concatenate([[0], np.cumsum(ranks.astype(np.int64) * nc)])
    for i in range(1, t.nnodes):
        k = ranks[i]
        if k == 0:
            continue
        sk = skel[koff[i]:koff[i + 1]]
        assert np.all(np.diff(sk) > 0)
        if o.nchild[i] == 0:
            cand = np.arange(o.begin[i], o.end[i])
        else:
            cand = np.concatenate([skel[koff[c]:koff[c + 1]] for c in range(o.fchild[i], o.fchild[i] + o.nchild[i])])
        rows = np.searchsorted(cand, sk)
        assert np.array_equal(cand[rows], sk)
        Ui = U[uoff[i]:uoff[i + 1]].reshape(k, nc[i]).T
        assert np.array_equal(Ui[rows], np.eye(k))


MULTI_CASES = [
    ("fp64_coulomb3d", 3, 6000, 64, "coulomb", (), 1e-7, 6, "fp64"),
    ("mixed_coulomb3d", 3, 8000, 100, "coulomb", (), 1e-5, 7, "mixed"),
    ("mixed_gauss2d", 2, 6000, 64, "gaussian", (0.2,), 1e-5, 10, "mixed"),
    ("fp64_bump3d", 3, 5000, 64, "bump", (0.1,), 1e-7, 6, "fp64"),
    ("mixed_power3d", 3, 5000, 64, "power", (11.0,), 1e-5, 6, "mixed"),
    ("mixed_cosdot3d", 3, 5000, 64, "cosdot", (), 1e-5, 6, "mixed"),
]


@pytest.mark.parametrize("name,d,n,q,kern,kp,eps,g,prec", MULTI_CASES, ids=[c[0] for c in MULTI_CASES])
def test_matvec_multi_rhs(H2, name, d, n, q, kern, kp, eps, g, prec):
    """Several right-hand sides at once (launches of 16, 4 and 1 columns for
    21 columns): each column is the single-vector product of the same matrix;
    float32 vectors give the same product to float32 rounding; the host path
    with a leading dimension above n leaves the gaps between columns alone."""
    pts = I.uniform_cube(n, d, seed=70 + d)
    nrhs = 21
    Z = I.standard_normal(n * nrhs, seed=71).reshape(n, nrhs)
    t = H2.Tree(dev(pts), q)
    h = H2.Hidr(t, g, g)
    A = H2.H2Matrix(t, h, kern, kp, eps, prec)
    Y = A.matvec(dev(Z)).cpu().numpy()
    assert Y.shape == (n, nrhs)
    tol = 1e-12 if prec == "fp64" else 1e-6
    for j in [0, 5, 15, 16, 19, 20]:
        yj = A.matvec(dev(np.ascontiguousarray(Z[:, j]))).cpu().numpy()
        assert np.linalg.norm(Y[:, j] - yj) <= tol * np.linalg.norm(yj), j
    # the oracle's float64 H^2 product and the dense product, column by column
    o, oh, OH = O.build_h2(pts, kern, kp, q, eps, g, g)
    for j in [0, 20]:
        yo = OH.matvec(Z[:, j])
        lim = 1e-12 if prec == "fp64" else 10 * eps
        assert_rows_close(Y[:, j], yo, lim, f"{name} column {j} vs oracle")
        yd = O.dense_matvec(pts, kern, kp, Z[:, j])
        assert np.linalg.norm(Y[:, j] - yd) <= 10 * eps * np.linalg.norm(yd), j
    # float32 vectors in and out
    Y32 = A.matvec(dev(Z.astype(np.float32))).cpu().numpy()
    assert Y32.dtype == np.float32
    assert np.linalg.norm(Y32 - Y) <= 1e-5 * np.linalg.norm(Y)
    # host buffers with ld = n + 7: gaps between columns untouched
    ld = n + 7
    xh = np.zeros(ld * nrhs)
    yh = np.full(ld * nrhs, -7.25)
    for j in range(nrhs):
        xh[j * ld:j * ld + n] = Z[:, j]
    assert H2.lib().h2_matvec(A.handle, xh.ctypes.data_as(C.c_void_p), yh.ctypes.data_as(C.c_void_p), nrhs,
                              H2.DTYPE_F64, ld, 0, None) == 0
    for j in range(nrhs):
        assert np.linalg.norm(yh[j * ld:j * ld + n] - Y[:, j]) <= 1e-14 * np.linalg.norm(Y[:, j]), j
        assert np.all(yh[j * ld + n:(j + 1) * ld] == -7.25), j
    # argument checks
    assert H2.lib().h2_matvec(A.handle, xh.ctypes.data_as(C.c_void_p), yh.ctypes.data_as(C.c_void_p), 0,
                              H2.DTYPE_F64, ld, 0, None) == 1
    assert H2.lib().h2_matvec(A.handle, xh.ctypes.data_as(C.c_void_p), yh.ctypes.data_as(C.c_void_p), 2,
                              H2.DTYPE_F64, n - 1, 0, None) == 1
    assert H2.lib().h2_matvec(A.handle, xh.ctypes.data_as(C.c_void_p), xh.ctypes.data_as(C.c_void_p), 2,
                              H2.DTYPE_F64, ld, 0, None) == 1


def test_construct_batched_equals_one_by_one(H2):
    """h2_construct_batched: independent problems of uneven sizes (cube and
    sphere, three kernels, both forms, several leaf sizes, one tree and HiDR
    shared by three kernels) give exactly the matrices of one-by-one
    h2_construct calls (same kernels and reduction orders: bit-identical ranks,
    skeletons and U; products equal to rounding, since block sums meet in
    float64 atomics); a bad problem fails the whole call."""
    rng = np.random.default_rng(90)
    probs, keep = [], []
    shared_t = H2.Tree(dev(I.uniform_cube(9000, 3, seed=91)), 64)
    shared_h = H2.Hidr(shared_t, 5, 5)
    keep += [shared_t, shared_h]
    for kern, kp in [("coulomb", ()), ("gaussian", (0.5,)), ("multiquadric", ())]:
        probs.append((shared_t, shared_h, kern, kp, 1e-5, "mixed"))
    for a in range(9):
        n = int(np.exp(rng.uniform(np.log(2000), np.log(30000))))
        pts = I.uniform_cube(n, 3, seed=100 + a) if a % 2 == 0 else I.sphere_surface(n, seed=100 + a)
        q = [64, 128, 256][a % 3]
        kern, kp = [("coulomb", ()), ("gaussian", (0.5,)), ("multiquadric", ())][a % 3]
        t = H2.Tree(dev(pts), q)
        h = H2.Hidr(t, 5, 5)
        keep += [t, h]
        probs.append((t, h, kern, kp, [1e-5, 1e-7][a % 2], ["mixed", "fp64"][a % 2]))
    mats = H2.construct_batched(probs)
    assert len(mats) == len(probs)
    for (t, h, kern, kp, eps, prec), B in zip(probs, mats):
        A = H2.H2Matrix(t, h, kern, kp, eps, prec)
        for f in ["rank", "ncand", "skel", "U"]:
            assert np.array_equal(A.get(f), B.get(f)), (kern, prec, f)
        z = dev(I.standard_normal(t.n, seed=92))
        ya, yb = A.matvec(z), B.matvec(z)
        assert torch.linalg.norm(ya - yb) <= 1e-14 * torch.linalg.norm(ya), (kern, prec)
        A.free()
    for B in mats:
        B.free()
    # a hidr built on another tree: the call fails and returns no matrix
    bad = [probs[3], (probs[4][0], probs[5][1]) + probs[4][2:]]
    with pytest.raises(H2.H2Error) as e:
        H2.construct_batched(bad)
    assert e.value.status == 1 and "problem 1" in str(e.value)
    for x in reversed(keep):
        x.free()


def test_bounded_g_exchanges(H2):
    """Eq. (3)'s bound ||G||_max <= f by exchanges after the QR: float64
    ranks, skeletons, U and the number of exchanges equal the oracle's with
    the same f; every U entry within f; both forms within 10 eps of the dense
    product; an f that is neither 0 nor above 1 is rejected."""
    n, q, eps, g, f = 6000, 100, 1e-6, 7, 1.1
    pts = I.uniform_cube(n, 3, seed=53)
    z = I.standard_normal(n, seed=51)
    t = H2.Tree(dev(pts), q)
    h = H2.Hidr(t, g, g)
    A = H2.H2Matrix(t, h, "coulomb", (), eps, "fp64", g_bound=f)
    o, oh, OH = O.build_h2(pts, "coulomb", (), q, eps, g, g, g_bound=f)
    st = json.loads(A.stats())
    assert st["exchanges"] == OH.exchanges() > 0
    ranks, nc = A.get("rank"), A.get("ncand")
    skel, U = A.get("skel"), A.get("U")
    assert np.array_equal(ranks, np.array([max(OH.rank(i), 0) for i in range(o.nnodes)]))
    koff = np.concatenate([[0], np.cumsum(ranks)])
    uoff = np.concatenate([[0], np.cumsum(ranks.astype(np.int64) * nc)])
    for i in range(1, o.nnodes):
        k = ranks[i]
        if k == 0:
            continue
        assert np.array_equal(skel[koff[i]:koff[i + 1]], OH.skeleton(i)), i
        Ui = U[uoff[i]:uoff[i + 1]].reshape(k, nc[i]).T
        assert np.max(np.abs(Ui - OH.U(i))) <= 64 * 2.0 ** -53 * nc[i] / eps * max(1.0, np.abs(OH.U(i)).max()), i
    assert st["g_max"] <= f
    yd = O.dense_matvec(pts, "coulomb", (), z)
    y = A.matvec(dev(z)).cpu().numpy()
    assert np.linalg.norm(y - yd) <= 10 * eps * np.linalg.norm(yd)
    Am = H2.H2Matrix(t, h, "coulomb", (), 1e-5, "mixed", g_bound=f)
    stm = json.loads(Am.stats())
    assert stm["exchanges"] > 0 and stm["g_max"] <= f
    ym = Am.matvec(dev(z)).cpu().numpy()
    assert np.linalg.norm(ym - yd) <= 10 * 1e-5 * np.linalg.norm(yd)
    for bad in (0.5, 1.0, float("nan"), -2.0):
        with pytest.raises(RuntimeError):
            H2.H2Matrix(t, h, "coulomb", (), eps, "fp64", g_bound=bad)
    Am.free()
    A.free()


def test_autotune_leaf(H2):
    """The leaf-size autotuner returns the candidate with the least measured
    time, from device or host points, and every candidate's time."""
    pts = I.uniform_cube(100000, 3, seed=90)
    best, times = H2.autotune_leaf(dev(pts), (64, 128, 256), g=6, id_tol=1e-5, precision="mixed")
    assert set(times) == {64, 128, 256} and all(v > 0 for v in times.values())
    assert best == min(times, key=lambda q: (times[q], [64, 128, 256].index(q)))
    best_h, times_h = H2.autotune_leaf(pts[:20000], (32, 256), g=5, kernel="gaussian", kparams=(0.5,),
                                       precision="fp64", reps=1)
    assert best_h in (32, 256) and set(times_h) == {32, 256}


@pytest.mark.parametrize("prec,dtype", [("fp64", "float64"), ("mixed", "float32")])
def test_matvec_graph(H2, prec, dtype):
    """A product recorded as a CUDA graph (h2_matvec_graph_create) replays
    y = K~ x for the vector x holds at launch time; its matrix cannot be
    freed while the graph lives."""
    n, q, g, eps = 6000, 64, 6, 1e-6
    pts = I.uniform_cube(n, 3, seed=95)
    t = H2.Tree(dev(pts), q)
    h = H2.Hidr(t, g, g)
    A = H2.H2Matrix(t, h, "coulomb", (), eps, prec)
    tdt = getattr(torch, dtype)
    x = dev(I.standard_normal(n, seed=96)).to(tdt)
    y = torch.zeros(n, dtype=tdt, device="cuda")
    G = A.capture_matvec(x, y)
    for seed in (97, 98):
        z = dev(I.standard_normal(n, seed=seed)).to(tdt)
        x.copy_(z)
        G.launch()
        torch.cuda.synchronize()
        want = A.matvec(z).double().cpu().numpy()
        got = y.double().cpu().numpy()
        tol = 1e-14 if prec == "fp64" else 1e-6
        assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want), seed
    with pytest.raises(H2.H2Error) as e:
        A.free()
    assert e.value.status == 7  # H2_ERR_STATE
    G.free()
    A.free()


def test_tree_and_hidr_batched_equal_one_by_one(H2):
    """h2_tree_build_batched and h2_hidr_reduce_batched: independent problems
    of uneven sizes (cube and sphere, several leaf sizes and grids, with and
    without the interaction-list reduction) give exactly the trees and HiDR
    sets of one-by-one calls; a bad problem fails the whole call and names it."""
    rng = np.random.default_rng(93)
    pts, qs, gs = [], [], []
    for a in range(10):
        n = int(np.exp(rng.uniform(np.log(1500), np.log(25000))))
        pts.append(I.uniform_cube(n, 3, seed=200 + a) if a % 2 == 0 else I.sphere_surface(n, seed=200 + a))
        qs.append([64, 128, 256][a % 3])
        gs.append([4, 5, 6][a % 3])
    trees = H2.tree_build_batched([dev(p) for p in pts], qs, tau=(1, 2))
    for a, t in enumerate(trees):
        o = H2.Tree(dev(pts[a]), qs[a], tau=(1, 2))
        for f in ["perm", "near_ptr", "near_idx", "far_ptr", "far_idx", "lptr"]:
            assert np.array_equal(t.get(f), o.get(f)), (a, f)
        o.free()
    for ilr in (False, True):
        hs = H2.hidr_reduce_batched(trees, gs, gs, il_reduce=ilr)
        for a, (t, h) in enumerate(zip(trees, hs)):
            o = H2.Hidr(t, gs[a], gs[a], il_reduce=ilr)
            for which in ("x", "y"):
                (c1, d1), (c2, d2) = h.get(which), o.get(which)
                assert np.array_equal(c1, c2) and np.array_equal(d1, d2), (a, which, ilr)
            o.free()
        for h in hs:
            h.free()
    # host point sets through the same call
    th = H2.tree_build_batched(pts[:3], 64)
    for a, t in enumerate(th):
        assert np.array_equal(t.get("perm"), H2.Tree(pts[a], 64).get("perm"))
        t.free()
    # a bad leaf size in problem 2: no tree is returned and the message names it
    with pytest.raises(H2.H2Error) as e:
        H2.tree_build_batched([dev(p) for p in pts[:4]], [64, 64, 0, 64])
    assert e.value.status == 1 and "problem 2" in str(e.value)
    with pytest.raises(H2.H2Error) as e:
        H2.hidr_reduce_batched(trees[:3], [4, 4, 4], [4, 0, 4])
    assert e.value.status == 1 and "problem 1" in str(e.value)
    for t in trees:
        t.free()
