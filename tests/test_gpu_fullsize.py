"""Full-size parity at the benchmark configurations, in the launch configuration
bench.py times:

  cube1m  1,048,576 uniform points in [0,1]^3 (seed 2), leaf size 256,
          Coulomb, eq. (1) with tau = 1/2, HiDR with the interaction-list
          reduction; float64 eps = 1e-9, g = 8 and mixed eps = 3e-6, g = 6;
          the metric's bounds on 1000 sampled rows against exact sums:
          <= 1e-8 (float64) and <= 1e-5 (mixed);
  gmix2m  2,097,152 points of the 16-component Gaussian mixture in [0,1]^2
          (seed 3), leaf size 128, Gaussian kernel exp(-r^2/0.04), g = 20,
          eps = 1e-10 (float64) and 1e-6 (mixed, same grid): within 10 eps;
  sphere8m  8,388,608 points on the unit sphere (seed 5), leaf size 256,
          Coulomb, tau = 1/2, interaction-list reduction, g = 6, mixed
          eps = 1e-6, 16 float32 right-hand sides: within 10 eps.

The oracle cannot build the whole H^2 matrix at these sizes in seconds, so the
checks are: the tree and near/far lists in full (bit-exact); X_i* for every
node (bit-exact, the oracle's bottom-up pass is cheap); Y_i* for sampled nodes
(the oracle computes their ancestor chains); ranks, skeletons and U for
sampled leaves and parents (float64, same tolerance as the small cases); exact
rows against the oracle's; both forms' products on the sampled rows against
the oracle's exact sums; for the sphere, every one of the 16 columns against
its own single-vector product and the exact rows of two columns."""
import numpy as np
import pytest

from oracle import h2_oracle as O
from paper_2206_01885_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CONFIGS = {
    "cube1m": dict(make=lambda: I.uniform_cube(1 << 20, 3, seed=2), q=256, kern="coulomb", kp=(), tau=(1, 2),
                   il_reduce=True, eps=1e-9, g=8, eps_m=3e-6, g_m=6, err64=1e-8, errm=1e-5),
    "gmix2m": dict(make=lambda: I.gaussian_mixture(1 << 21, seed=3), q=128, kern="gaussian", kp=(0.2,),
                   tau=(7, 10), il_reduce=False, eps=1e-10, g=20, eps_m=1e-6, g_m=20, err64=1e-9, errm=1e-5),
}


@pytest.fixture(scope="module", params=list(CONFIGS))
def setup(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_01885_gb300 import build as B
    B.build()
    from paper_2206_01885_gb300 import h2
    cfg = CONFIGS[request.param]
    pts = cfg["make"]()
    P = torch.from_numpy(pts).cuda()
    t = h2.Tree(P, cfg["q"], tau=cfg["tau"])
    hd = h2.Hidr(t, cfg["g"], cfg["g"], il_reduce=cfg["il_reduce"])
    A = h2.H2Matrix(t, hd, cfg["kern"], cfg["kp"], cfg["eps"])
    ot = O.tree_build(pts, cfg["q"], cfg["tau"])
    yield h2, pts, P, t, hd, A, ot, cfg
    A.free()
    hd.free()
    t.free()


def test_fullsize_tree_and_lists(setup):
    h2, pts, P, t, hd, A, ot, cfg = setup
    for f in ["perm", "keys", "level", "parent", "fchild", "nchild", "begin", "end", "prefix", "lptr",
              "near_ptr", "near_idx", "far_ptr", "far_idx"]:
        got = t.get(f)
        want = getattr(ot, f.replace("keys", "key"))
        assert np.array_equal(got, want.astype(got.dtype)), f


def _sample_nodes(ot, rng):
    leaves = np.flatnonzero(ot.nchild == 0)
    deep = leaves[ot.level[leaves] == ot.nlevels - 1]
    shallow = leaves[ot.level[leaves] < ot.nlevels - 1]
    parents = np.flatnonzero((ot.nchild > 0) & (ot.level == ot.nlevels - 2))
    return (rng.choice(deep, 6, replace=False), rng.choice(shallow, 4, replace=False),
            rng.choice(parents, 2, replace=False))


def test_fullsize_hidr_and_bases(setup):
    h2, pts, P, t, hd, A, ot, cfg = setup
    rng = np.random.default_rng(2024)
    deep, shallow, parents = _sample_nodes(ot, rng)
    build = np.zeros(ot.nnodes, dtype=bool)
    build[np.concatenate([deep, shallow, parents])] = True
    need = O.closure_down(ot, build)
    G = cfg["g"]
    oh = O.Hidr(ot, G, G, need_y=need, il_reduce=cfg["il_reduce"])  # X* everywhere, Y* on need and ancestors
    xc, xd = hd.get("x")
    yc, yd = hd.get("y")
    xo, yo = np.concatenate([[0], np.cumsum(xc)]), np.concatenate([[0], np.cumsum(yc)])
    for i in range(1, ot.nnodes):
        assert np.array_equal(xd[xo[i]:xo[i + 1]], oh.get(i, "x")), ("X*", i)
    checked = 0
    for i in range(1, ot.nnodes):
        want = oh.get(i, "y")
        if want is None:
            continue
        assert np.array_equal(yd[yo[i]:yo[i + 1]], want), ("Y*", i)
        checked += 1
    assert checked >= len(need.nonzero()[0])
    EPS = cfg["eps"]
    OH = O.H2(ot, oh, cfg["kern"], cfg["kp"], EPS, need=build)
    ranks, nc = A.get("rank"), A.get("ncand")
    skel, U = A.get("skel"), A.get("U")
    ko = np.concatenate([[0], np.cumsum(ranks)])
    uo = np.concatenate([[0], np.cumsum(ranks.astype(np.int64) * nc)])
    for i in np.flatnonzero(build):
        k = ranks[i]
        assert k == OH.rank(i), i
        assert np.array_equal(skel[ko[i]:ko[i + 1]], OH.skeleton(i)), i
        Ui = U[uo[i]:uo[i + 1]].reshape(k, nc[i]).T
        tol = 64 * 2.0 ** -53 * nc[i] / EPS
        assert np.max(np.abs(Ui - OH.U(i))) <= tol * max(1.0, np.abs(OH.U(i)).max()), i


def test_fullsize_exact_rows_and_forms(setup):
    """The sampled-row error the bench reports, for both forms, against the
    oracle's exact float64 sums (bench.py's right-hand side and rows)."""
    h2, pts, P, t, hd, A, ot, cfg = setup
    n, kern, kp = len(pts), cfg["kern"], cfg["kp"]
    z = I.standard_normal(n, seed=9)
    rows = I.sample_rows(n, 1000, seed=11)
    Z, R = torch.from_numpy(z).cuda(), torch.from_numpy(rows).cuda()
    ex = h2.exact_rows(t, kern, kp, Z, R).cpu().numpy()
    want = O.exact_rows(pts, kern, kp, z, rows)
    assert np.allclose(ex, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    # the float64 form: the metric's bound
    y64 = A.matvec(Z).cpu().numpy()
    err64 = np.linalg.norm(y64[rows] - want) / np.linalg.norm(want)
    print(f"sampled relative error, float64 form: {err64:.3e}")
    assert err64 <= cfg["err64"]
    # the mixed form with its own grid and tolerance, against the same exact sums
    hm = hd if cfg["g_m"] == cfg["g"] else h2.Hidr(t, cfg["g_m"], cfg["g_m"], il_reduce=cfg["il_reduce"])
    Am = h2.H2Matrix(t, hm, kern, kp, cfg["eps_m"], "mixed")
    ym = Am.matvec(Z).cpu().numpy()
    errm = np.linalg.norm(ym[rows] - want) / np.linalg.norm(want)
    print(f"sampled relative error, mixed form: {errm:.3e}")
    assert errm <= cfg["errm"]
    Am.free()
    if hm is not hd:
        hm.free()


def test_fullsize_sphere_16_rhs():
    """8,388,608 points on the unit sphere, 16 float32 right-hand sides, mixed
    form at eps = 1e-6, tau = 1/2, HiDR with the interaction-list reduction,
    g = 6: tree and lists bit-exact; each column of the 16-column product
    equals that column's own product; two columns against exact float64 rows,
    within 10 eps."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_01885_gb300 import build as B
    B.build()
    from paper_2206_01885_gb300 import h2
    n, q, g, eps = 1 << 23, 256, 6, 1e-6
    pts = I.sphere_surface(n, seed=5)
    t = h2.Tree(torch.from_numpy(pts).cuda(), q, tau=(1, 2))
    ot = O.tree_build(pts, q, (1, 2))
    for f in ["perm", "level", "begin", "end", "near_ptr", "near_idx", "far_ptr", "far_idx"]:
        got = t.get(f)
        assert np.array_equal(got, getattr(ot, f).astype(got.dtype)), f
    del ot
    hd = h2.Hidr(t, g, g, il_reduce=True)
    A = h2.H2Matrix(t, hd, "coulomb", (), eps, "mixed")
    rng = np.random.default_rng(55)
    Zh = rng.standard_normal((n, 16)).astype(np.float32)
    Z = torch.from_numpy(Zh).cuda()
    Y = A.matvec(Z)
    assert Y.shape == (n, 16) and Y.dtype == torch.float32
    Y = Y.cpu().numpy()
    for j in range(16):
        yj = A.matvec(Z[:, j].contiguous()).cpu().numpy()
        assert np.linalg.norm(Y[:, j] - yj) <= 1e-6 * np.linalg.norm(yj), j
    rows = I.sample_rows(n, 100, seed=56)
    for j in [0, 15]:
        zj = Zh[:, j].astype(np.float64)
        want = O.exact_rows(pts, "coulomb", (), zj, rows)
        got = h2.exact_rows(t, "coulomb", (), torch.from_numpy(zj).cuda(), torch.from_numpy(rows).cuda())
        assert np.allclose(got.cpu().numpy(), want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
        err = np.linalg.norm(Y[rows, j] - want) / np.linalg.norm(want)
        print(f"sampled relative error, column {j}: {err:.3e}")
        assert err <= 10 * eps
    A.free()
    hd.free()
    t.free()
