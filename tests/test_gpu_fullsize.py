"""Full-size parity at the benchmark configuration: 1,048,576 uniform points in
[0,1]^3 (seed 2), leaf size 256, g = 9, Coulomb, eps = 1e-8, the launch
configuration bench.py times.

The oracle cannot build the whole H^2 matrix at this size in seconds, so the
checks are: the tree and near/far lists in full (bit-exact); X_i* for every
node (bit-exact, the oracle's bottom-up pass is cheap); Y_i* for sampled nodes
(the oracle computes their ancestor chains); ranks, skeletons and U for
sampled leaves and level-4 parents (float64, same tolerance as the small
cases); exact rows against the oracle's; and the mixed form against the float64
form built with the same tolerance and grid."""
import numpy as np
import pytest

from oracle import h2_oracle as O
from paper_2206_01885_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N, Q, G, EPS = 1 << 20, 256, 9, 1e-8


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_01885_gb300 import build as B
    B.build()
    from paper_2206_01885_gb300 import h2
    pts = I.uniform_cube(N, 3, seed=2)
    P = torch.from_numpy(pts).cuda()
    t = h2.Tree(P, Q)
    hd = h2.Hidr(t, G, G)
    A = h2.H2Matrix(t, hd, "coulomb", (), EPS)
    ot = O.tree_build(pts, Q)
    return h2, pts, P, t, hd, A, ot


def test_fullsize_tree_and_lists(setup):
    h2, pts, P, t, hd, A, ot = setup
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
    h2, pts, P, t, hd, A, ot = setup
    rng = np.random.default_rng(2024)
    deep, shallow, parents = _sample_nodes(ot, rng)
    build = np.zeros(ot.nnodes, dtype=bool)
    build[np.concatenate([deep, shallow, parents])] = True
    need = O.closure_down(ot, build)
    oh = O.Hidr(ot, G, G, need_y=need)  # X* everywhere, Y* on need and its ancestors
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
    OH = O.H2(ot, oh, "coulomb", (), EPS, need=build)
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
    h2, pts, P, t, hd, A, ot = setup
    z = I.standard_normal(N, seed=9)
    rows = I.sample_rows(N, 200, seed=11)
    Z, R = torch.from_numpy(z).cuda(), torch.from_numpy(rows).cuda()
    ex = h2.exact_rows(t, "coulomb", (), Z, R).cpu().numpy()
    want = O.exact_rows(pts, "coulomb", (), z, rows)
    assert np.allclose(ex, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    # the float64 product on the sampled rows: the error the bench reports
    y64 = A.matvec(Z).cpu().numpy()
    err64 = np.linalg.norm(y64[rows] - want) / np.linalg.norm(want)
    assert err64 < 1e-4
    # mixed form at the same tolerance and grid: within 10 eps of the float64 form
    eps_m = 1e-5
    A64 = h2.H2Matrix(t, hd, "coulomb", (), eps_m, "fp64")
    Am = h2.H2Matrix(t, hd, "coulomb", (), eps_m, "mixed")
    ya, yb = A64.matvec(Z).cpu().numpy(), Am.matvec(Z).cpu().numpy()
    assert np.linalg.norm(yb - ya) / np.linalg.norm(ya) <= 10 * eps_m
