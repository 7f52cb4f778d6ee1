"""Pins for the oracle's DataReduct, HiDR, getBasis/ID, construction and matvec.

What pins what (each against something other than the oracle itself):
  * DataReduct (section 3.3): nearest neighbours from scipy's cKDTree (a library
    special case), the subset / size rules, ties to the smaller label;
  * HiDR (Algorithm 1, Theorem 3.1): subset and size invariants, Y_i* inside
    the farfield found by brute force, and the no-reduction case where X_i* = X_i
    and Y_i* is the whole farfield; with the interaction-list reduction, Y_i*
    equals the union of the two scipy reductions it is defined by;
  * getBasis (eqs. (3)-(5)): LAPACK geqp3 pivots and R diagonal through scipy,
    exact rank on products of random factors, U[Xhat,:] = I;
  * matvec: the hand-computed dense product, math.fsum for the exact sums,
    equality with the dense product when nothing is truncated, and the
    relative error <= 10 eps when it is;
  * nestedness Xhat_p subset of the union of the children's Xhat (Algorithm 2)."""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg
from scipy.spatial import cKDTree

from oracle import h2_oracle as O
from paper_2206_01885_gb300 import inputs as I


# ----------------------------------------------------------------- DataReduct
@pytest.mark.parametrize("d,ns,g,seed", [(3, 500, 4, 1), (2, 300, 5, 2), (3, 2000, 7, 3), (1, 50, 9, 4)])
def test_datareduct_matches_kdtree(d, ns, g, seed):
    rng = np.random.default_rng(seed)
    X = rng.random((ns, d)) * rng.uniform(0.5, 3.0, size=d) + rng.normal(size=d)
    labels = np.arange(ns, dtype=np.int64)
    got = O.datareduct(X, labels, g)
    l, u = X.min(0), X.max(0)
    axes = [l[k] + (np.arange(g) + 0.5) * ((u[k] - l[k]) / g) for k in range(d)]
    Q = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, d)
    _, nn = cKDTree(X).query(Q)
    want = np.unique(nn)
    assert np.array_equal(got, want)
    assert len(got) <= g ** d


def test_datareduct_small_set_is_identity_and_sorted():
    X = np.random.default_rng(5).random((40, 3))
    labels = np.array([30, 2, 17, 5], dtype=np.int64)
    assert list(O.datareduct(X, labels, 2)) == [2, 5, 17, 30]


def test_datareduct_tie_goes_to_smaller_label():
    # points 3 and 1 coincide; the grid point nearest to them must pick 1
    X = np.array([[0.0, 0.0], [0.5, 0.5], [1.0, 1.0], [0.5, 0.5], [0.0, 1.0], [1.0, 0.0]])
    got = O.datareduct(X, np.arange(6, dtype=np.int64), 1)  # one grid point at (0.5, 0.5)
    assert list(got) == [1]


# ----------------------------------------------------------------------- HiDR
def _farfield_points(t, i):
    """all Morton positions in X_j for j far from i or from an ancestor of i"""
    pts = set()
    a = i
    while a >= 0:
        for j in t.far(a):
            pts.update(range(int(t.begin[j]), int(t.end[j])))
        a = int(t.parent[a]) if a > 0 else -1
    return pts


@pytest.mark.parametrize("d,n,q,g,method", [(3, 3000, 30, 3, "volume"), (2, 2500, 20, 4, "volume"),
                                            (3, 3000, 30, 3, "surface"), (2, 2500, 20, 4, "surface"),
                                            (3, 3000, 30, 3, "fps"), (2, 2500, 20, 4, "fps")])
def test_hidr_invariants(d, n, q, g, method):
    pts = I.uniform_cube(n, d, seed=7 + d)
    t = O.tree_build(pts, q)
    h = O.Hidr(t, g, g, method=method)
    r = g ** d
    for i in range(1, t.nnodes):
        xs = h.get(i, "x")
        assert len(xs) <= r and np.all(np.diff(xs) > 0)
        assert np.all((xs >= t.begin[i]) & (xs < t.end[i]))  # X_i* subset of X_i
        if t.nchild[i]:
            S = np.concatenate([h.get(c, "x") for c in range(t.fchild[i], t.fchild[i] + t.nchild[i])])
            assert len(S) <= (2 ** d) * r  # Theorem 3.1: |S_i| = O(1)
            assert set(xs) <= set(S)
        ys = h.get(i, "y")
        assert len(ys) <= r
        far = _farfield_points(t, i)
        assert set(ys.tolist()) <= far
        assert (len(ys) == 0) == (len(far) == 0)


def _kdtree_reduce(X, labels, g):
    """DataReduct(S, g^d) by its definition, through scipy: S itself when it has
    at most g^d points, else the nearest point of S to each cell-centred point
    of the g^d grid over S's bounding box."""
    labels = np.asarray(labels, dtype=np.int64)
    d = X.shape[1]
    if len(labels) <= g ** d:
        return np.unique(labels)
    P = X[labels]
    l, u = P.min(0), P.max(0)
    axes = [l[k] + (np.arange(g) + 0.5) * ((u[k] - l[k]) / g) for k in range(d)]
    Q = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, d)
    _, nn = cKDTree(P).query(Q)
    return np.unique(labels[nn])


@pytest.mark.parametrize("d,n,q,g", [(3, 3000, 30, 3), (2, 2500, 20, 4), (3, 6000, 40, 4)])
def test_hidr_il_reduce_adds_the_interaction_list_reduction(d, n, q, g):
    # Y_i* = DataReduct(T_i) u DataReduct(union of X_j*, j in IL(i)), T_i = Y_p* u that union
    pts = I.uniform_cube(n, d, seed=7 + d)
    t = O.tree_build(pts, q)
    h0 = O.Hidr(t, g, g)
    h = O.Hidr(t, g, g, il_reduce=True)
    grew = 0
    empty = np.zeros(0, dtype=np.int64)
    for i in range(1, t.nnodes):
        assert np.array_equal(h.get(i, "x"), h0.get(i, "x"))
        far = t.far(i)
        il = np.concatenate([h.get(int(j), "x") for j in far]) if len(far) else empty
        T = np.concatenate([h.get(int(t.parent[i]), "y") if t.parent[i] > 0 else empty, il])
        want = np.union1d(_kdtree_reduce(t.x, T, g) if len(T) else empty,
                          _kdtree_reduce(t.x, il, g) if len(il) else empty)
        ys = h.get(i, "y")
        assert np.array_equal(ys, want), i
        assert len(ys) <= 2 * g ** d
        assert set(ys.tolist()) <= _farfield_points(t, i)
        grew += len(ys) > len(_kdtree_reduce(t.x, T, g) if len(T) else empty)
    assert grew > 0


def test_hidr_no_reduction_gives_full_sets():
    pts = I.uniform_cube(1500, 3, seed=21)
    t = O.tree_build(pts, 25)
    h = O.Hidr(t, 1000, 1000)  # g^d larger than any set
    for i in range(1, t.nnodes):
        assert np.array_equal(h.get(i, "x"), np.arange(t.begin[i], t.end[i]))
        assert set(h.get(i, "y").tolist()) == _farfield_points(t, i)


# ------------------------------------------------------------------ getBasis
def _graded(m, c, seed, decay=0.7):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, c)) @ np.diag(decay ** np.arange(c)) @ scipy.linalg.qr(rng.standard_normal((c, c)))[0]
    return A


@pytest.mark.parametrize("m,c,seed", [(40, 25, 1), (25, 40, 2), (60, 60, 3), (7, 3, 4)])
def test_id_pivots_match_lapack_geqp3(m, c, seed):
    A = np.random.default_rng(seed).standard_normal((m, c)) * np.linspace(1.0, 3.0, c)
    k, piv, T = O.interp_decomp(A, 0.0)
    Q, R, P = scipy.linalg.qr(A, pivoting=True, mode="economic")
    assert k == min(m, c)
    assert np.array_equal(piv[:k], P[:k])


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-10])
def test_id_truncation_rule_against_lapack_R(eps):
    A = _graded(50, 40, 11)
    k, piv, T = O.interp_decomp(A, eps)
    Q, R, P = scipy.linalg.qr(A, pivoting=True, mode="economic")
    dg = np.abs(np.diag(R))
    # first j with |r_jj| <= eps |r_11|
    want = int(np.argmax(dg <= eps * dg[0])) if np.any(dg <= eps * dg[0]) else len(dg)
    assert k == want
    assert np.array_equal(piv[:k], P[:k])
    # the ID reproduces the non-skeleton columns within the truncation level
    err = np.linalg.norm(A[:, piv[k:]] - A[:, piv[:k]] @ T, 2)
    assert err <= 10 * eps * np.linalg.norm(A, 2) * np.sqrt(A.shape[1])


def test_id_exact_rank():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((30, 7)) @ rng.standard_normal((7, 45))
    k, piv, T = O.interp_decomp(A, 1e-10)
    assert k == 7
    assert np.allclose(A[:, piv[k:]], A[:, piv[:k]] @ T, rtol=0, atol=1e-11 * np.abs(A).max())


def test_id_zero_and_full_rank():
    k, piv, T = O.interp_decomp(np.zeros((5, 4)), 1e-8)
    assert k == 0
    A = np.random.default_rng(4).standard_normal((12, 9))
    k, piv, T = O.interp_decomp(A, 0.0)
    assert k == 9 and T.shape == (9, 0)


# --------------------------------------------------------------- H^2 matvec
def test_dense_golden(golden_dir):
    gold = json.load(open(os.path.join(golden_dir, "kernel_3pt.json")))
    pts = np.array(gold["points"])
    z = np.array(gold["z"])
    env = {"exp": math.exp, "sqrt": math.sqrt, "cos": math.cos}
    for name, kern, kp in [("coulomb", "coulomb", ()), ("gaussian_h1", "gaussian", (1.0,)),
                           ("exponential_l1", "exponential", (1.0,)), ("multiquadric", "multiquadric", ()),
                           ("bump_a0.1", "bump", (0.1,)), ("bump_a0.25", "bump", (0.25,)),
                           ("power_p11", "power", (11.0,)), ("cosdot", "cosdot", ())]:
        want = np.array([eval(e, env) for e in gold[name]])
        got = O.dense_matvec(pts, kern, kp, z)
        assert np.allclose(got, want, rtol=1e-15, atol=0), name


def test_exact_rows_summation_against_fsum():
    pts = I.uniform_cube(3000, 3, seed=31)
    z = I.standard_normal(3000, seed=32)
    rows = np.array([0, 17, 2999])
    got = O.exact_rows(pts, "coulomb", (), z, rows)
    for a, r in enumerate(rows):
        d = np.sqrt(((pts - pts[r]) ** 2).sum(1))
        terms = [(1.0 / dd) * zz if dd > 0 else 0.0 for dd, zz in zip(d, z)]
        assert abs(got[a] - math.fsum(terms)) <= 1e-13 * math.fsum(abs(v) for v in terms)


@pytest.mark.parametrize("d,n,q,kern,kp", [(3, 1200, 40, "coulomb", ()), (2, 1500, 30, "gaussian", (0.2,)),
                                           (3, 1000, 50, "multiquadric", ()), (3, 1000, 50, "bump", (0.1,)),
                                           (3, 900, 50, "power", (11.0,)), (3, 1000, 50, "cosdot", ())])
def test_h2_exact_without_reduction_or_truncation(d, n, q, kern, kp):
    pts = I.uniform_cube(n, d, seed=41)
    z = I.standard_normal(n, seed=42)
    t, h, H = O.build_h2(pts, kern, kp, q, 1e-15, 10 ** 6, 10 ** 6)
    y = H.matvec(z)
    yd = O.dense_matvec(pts, kern, kp, z)
    assert np.linalg.norm(y - yd) / np.linalg.norm(yd) < 1e-10


@pytest.mark.parametrize("d,n,q,kern,kp,eps,g", [
    (3, 6000, 100, "coulomb", (), 1e-4, 5),
    (3, 6000, 100, "coulomb", (), 1e-6, 7),
    (2, 5000, 64, "exponential", (0.1,), 1e-6, 12),
    (3, 4000, 64, "gaussian", (0.5,), 1e-5, 7),
    (3, 4000, 64, "bump", (0.1,), 1e-6, 6),
    (3, 4000, 64, "power", (11.0,), 1e-6, 6),
    (3, 4000, 64, "cosdot", (), 1e-6, 6),
])
def test_h2_matvec_error_within_10eps(d, n, q, kern, kp, eps, g):
    pts = I.uniform_cube(n, d, seed=50 + d)
    z = I.standard_normal(n, seed=51)
    t, h, H = O.build_h2(pts, kern, kp, q, eps, g, g)
    y = H.matvec(z)
    yd = O.dense_matvec(pts, kern, kp, z)
    err = np.linalg.norm(y - yd) / np.linalg.norm(yd)
    assert err <= 10 * eps, err
    # it must actually compress: some far pairs and ranks below the candidates
    assert len(t.far_idx) > 0
    assert any(0 < H.rank(i) < H.ncand(i) for i in range(t.nnodes))


def test_h2_with_il_reduce_within_10eps():
    pts = I.uniform_cube(4000, 3, seed=53)
    z = I.standard_normal(4000, seed=51)
    t, h, H = O.build_h2(pts, "coulomb", (), 64, 1e-6, 5, 5, il_reduce=True)
    assert max(len(h.get(i, "y")) for i in range(1, t.nnodes)) > 5 ** 3  # rows beyond one grid
    yd = O.dense_matvec(pts, "coulomb", (), z)
    err = np.linalg.norm(H.matvec(z) - yd) / np.linalg.norm(yd)
    assert err <= 1e-5, err


def test_nested_skeletons_and_identity_rows():
    pts = I.uniform_cube(6000, 3, seed=61)
    t, h, H = O.build_h2(pts, "coulomb", (), 60, 1e-6, 6, 6)
    for i in range(1, t.nnodes):
        k = H.rank(i)
        if k <= 0:
            continue
        sk = H.skeleton(i)
        assert np.all(np.diff(sk) > 0)
        if t.nchild[i]:
            union = np.concatenate([H.skeleton(c) for c in range(t.fchild[i], t.fchild[i] + t.nchild[i])])
            assert set(sk.tolist()) <= set(union.tolist())  # Xhat_p subset of Xbar_p
            cand = union
        else:
            cand = np.arange(t.begin[i], t.end[i])
        U = H.U(i)
        assert U.shape == (len(cand), k)
        rows = np.searchsorted(cand, sk)
        assert np.array_equal(U[rows], np.eye(k))
        assert k <= min(len(h.get(i, "y")), len(cand))  # eq. (5)


def test_calibration_picks_smallest_g():
    z1, z2 = I.calibration_sets(3, 8, n1=256, n2=1024)
    g = O.calibrate(3, "coulomb", (), 1e-4, z1, z2, gmax=12)
    assert 1 < g <= 12
    e_g, _, _ = O.calib_error(3, "coulomb", (), 1e-6, z1, z2, g)
    e_prev, _, _ = O.calib_error(3, "coulomb", (), 1e-6, z1, z2, g - 1)
    assert e_g < 1e-6 <= e_prev


@pytest.mark.parametrize("d,min_sq", [(2, 5), (3, 8)])
def test_calibration_on_exact_rank_kernels(d, min_sq):
    # |x - y|^p has rank 1 for p = 0 and rank d + 2 for p = 2 (|x|^2 - 2 x.y + |y|^2):
    # the ID must reveal exactly that rank, one representor (g = 1) reproduces the
    # constant kernel, and the 2^d bins of g = 2 hold at least d + 2 points in general
    # position, so g = 2 reproduces the squared distance to rounding while g = 1 cannot.
    z1, z2 = I.calibration_sets(d, min_sq, n1=256, n2=1024)
    e, k, _ = O.calib_error(d, "power", (0.0,), 1e-8, z1, z2, 1)
    assert k == 1 and e < 1e-14
    assert O.calibrate(d, "power", (0.0,), 1e-6, z1, z2, gmax=12) == 1
    e1, k1, _ = O.calib_error(d, "power", (2.0,), 1e-8, z1, z2, 1)
    e2, k2, _ = O.calib_error(d, "power", (2.0,), 1e-8, z1, z2, 2)
    assert k1 == 1 and e1 > 0.1
    assert k2 == d + 2 and e2 < 1e-14
    assert O.calibrate(d, "power", (2.0,), 1e-6, z1, z2, gmax=12) == 2


def test_id_tie_goes_to_first_column():
    # equal column norms everywhere: the pivot order must be 0, 1, 2, ...
    k, piv, T = O.interp_decomp(np.eye(5), 0.0)
    assert k == 5 and list(piv) == [0, 1, 2, 3, 4]
    A = np.array([[1.0, 0.0, 1.0], [0.0, 1.0, 0.0]])  # columns 0 and 2 identical
    k, piv, T = O.interp_decomp(A, 1e-12)
    assert k == 2 and list(piv[:2]) == [0, 1]
    assert np.allclose(T[:, 0], [1.0, 0.0])


def test_id_reflector_is_stable_for_nearly_aligned_columns():
    # columns almost parallel to e_1: alpha - beta must not cancel
    rng = np.random.default_rng(9)
    D = np.diag(np.linspace(1.0, 0.5, 6)) + 1e-9 * rng.standard_normal((6, 6))
    A = np.hstack([D, 1e-3 * rng.standard_normal((6, 2))])
    k, piv, T = O.interp_decomp(A, 0.0)
    assert k == 6 and np.all(np.isfinite(T))
    assert np.allclose(A[:, piv[6:]], A[:, piv[:6]] @ T, rtol=0, atol=1e-13)


# ----------------------------------------- eq. (3)'s bound on ||G||_max
def _kahan_rank_k(k, c, extra, m, seed):
    """Q [R11 R12] with R11 the k x k Kahan matrix (all columns of norm 1, so
    column pivoting keeps their order; a relative 1e-7 taper fixes it) and the
    extra columns continuing its pattern: exact rank k, and R11^{-1} R12 grows
    like (1 + c)^k, the classic case where column pivoting leaves |G| large."""
    s = np.sqrt(1 - c * c)
    R = np.zeros((k, k + extra))
    for i in range(k):
        R[i, i] = s ** i
        R[i, i + 1:] = -c * s ** i
    R = R * (1 + 1e-7 * np.arange(k + extra, 0, -1))[None, :]
    Q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((m, m)))
    return Q[:, :k] @ R


def test_id_bound_exchanges_reach_the_bound_and_keep_the_id_exact():
    A = _kahan_rank_k(6, 0.6, 2, 9, 0)
    k, piv, T = O.interp_decomp(A, 1e-12)
    assert k == 6 and list(piv) == list(range(8)) and np.abs(T).max() > 6
    vol0 = abs(np.linalg.det(A[:, piv[:k]].T @ A[:, piv[:k]]))
    nex, piv2, T2 = O.id_bound(k, piv, T, 2.0)
    assert nex >= 1 and np.abs(T2).max() <= 2.0
    assert sorted(piv2) == list(range(8))
    # exact rank: the exchanged T is the least-squares ID of the new skeleton, exact
    S, Rr = piv2[:k], piv2[k:]
    G = np.linalg.lstsq(A[:, S], A[:, Rr], rcond=None)[0]
    assert np.abs(G - T2).max() <= 1e-12
    assert np.abs(A[:, S] @ T2 - A[:, Rr]).max() <= 1e-13
    # each exchange multiplies the skeleton's volume by |g| > f
    vol = abs(np.linalg.det(A[:, S].T @ A[:, S]))
    assert vol >= vol0 * 4.0 ** nex * (1 - 1e-9)


def test_id_bound_leaves_a_bounded_id_alone():
    A = np.random.default_rng(5).standard_normal((12, 9))
    k, piv, T = O.interp_decomp(A, 1e-3)
    f = max(1.0, float(np.abs(T).max())) * 1.01 if T.size else 1.0
    nex, piv2, T2 = O.id_bound(k, piv, T, f)
    assert nex == 0 and np.array_equal(piv2, piv) and np.array_equal(T2, T)


def test_h2_with_bounded_g():
    pts = I.uniform_cube(6000, 3, seed=53)
    z = I.standard_normal(6000, seed=51)
    yd = O.dense_matvec(pts, "coulomb", (), z)
    t, h, H = O.build_h2(pts, "coulomb", (), 100, 1e-6, 7, 7, g_bound=1.1)
    assert H.exchanges() > 0
    umax = max(float(np.abs(H.U(i)).max()) for i in range(1, t.nnodes) if H.rank(i) > 0)
    assert umax <= 1.1
    assert np.linalg.norm(H.matvec(z) - yd) <= 10 * 1e-6 * np.linalg.norm(yd)


# ------------------------------------------ surface-based DataReduct (section 3.3)
def _surface_dirs(d, ne):
    """unit directions of the reading: the Fibonacci lattice (3D), equal angles (2D)"""
    out = []
    for j in range(ne):
        if d == 3:
            z = 1.0 - (2.0 * j + 1.0) / ne
            rho = math.sqrt(1.0 - z * z)
            phi = j * (math.pi * (3.0 - math.sqrt(5.0)))
            out.append((rho * math.cos(phi), rho * math.sin(phi), z))
        else:
            th = 2.0 * math.pi * (j + 0.5) / ne
            out.append((math.cos(th), math.sin(th)))
    return np.array(out)


@pytest.mark.parametrize("d,g", [(3, 4), (2, 9)])
def test_surface_datareduct_finds_points_on_its_ellipsoids(d, g):
    """S = the corners of a box (fixing the bounding box [l, u] and so the
    ellipsoids: centre (l + u) / 2, semi-axes gamma (u - l)), the points of the
    gamma = 0.3 ellipsoid (inside the box; the 0.6 and 1.2 ones reach outside
    it) and random interior points: every reference point on the gamma = 0.3
    ellipsoid finds itself (distance 0)."""
    lo, hi = np.array([0.0, -1.0, 2.0][:d]), np.array([1.0, 1.5, 2.5][:d])
    corners = np.array(np.meshgrid(*[[a, b] for a, b in zip(lo, hi)], indexing="ij")).reshape(d, -1).T
    ne = g ** d // 3
    u = _surface_dirs(d, ne)
    c, w = (lo + hi) * 0.5, hi - lo
    on = [c + (0.3 * w) * u]
    rnd = lo + (hi - lo) * np.random.default_rng(4).random((400, d))
    X = np.concatenate([corners] + on + [rnd])
    labels = np.arange(len(X))
    got = O.datareduct(X, labels, g, "surface")
    assert np.all(np.diff(got) > 0) and len(got) <= 3 * ne
    want = set(range(len(corners), len(corners) + ne))
    assert want <= set(got.tolist())
    # the other two ellipsoids pick further points of S
    assert len(set(got.tolist()) - want) >= 1


def test_surface_datareduct_small_set_is_identity():
    X = I.uniform_cube(20, 3, seed=8)
    assert np.array_equal(O.datareduct(X, np.arange(20)[::-1].copy(), 3, "surface"), np.arange(20))


# ------------------------------------------ farthest point sampling (section 3.3)
def test_fps_worked_example():
    """Points 0, 1, 2, 3, 10 on a line (labels in that order), g^2 = 4 picks:
    0 (smallest label); 10 (farthest from {0}); 3 (squared distances 1, 4, 9 to
    {0, 10}); then 1 and 2 tie at squared distance 1 and the smaller label, 1,
    wins."""
    X = np.array([[0.0, 0.0], [1.0, 0.0], [2.0, 0.0], [3.0, 0.0], [10.0, 0.0]])
    got = O.datareduct(X, np.array([4, 2, 0, 3, 1]), 2, "fps")
    assert got.tolist() == [0, 1, 3, 4]


@pytest.mark.parametrize("d,n,g", [(3, 700, 4), (2, 500, 6)])
def test_fps_covering_radius_at_most_separation(d, n, g):
    """FPS picks each point at the largest distance to the set so far, so every
    point left out is no farther from the picked set than any two picked points
    are from each other."""
    X = I.uniform_cube(n, d, seed=17 + d)
    got = O.datareduct(X, np.arange(n), g, "fps")
    assert len(got) == g ** d and got[0] == 0 and np.all(np.diff(got) > 0)
    P = X[got]
    rest = np.setdiff1d(np.arange(n), got)
    cover = np.sqrt(((X[rest][:, None, :] - P[None, :, :]) ** 2).sum(-1)).min(1).max()
    D = np.sqrt(((P[:, None, :] - P[None, :, :]) ** 2).sum(-1))
    np.fill_diagonal(D, np.inf)
    assert cover <= D.min() * (1 + 1e-12)
