"""The float64 form's Coulomb products in float-float arithmetic.

In the float64 form the on-the-fly coupling and nearfield products of the 3D
Coulomb kernel run on the float32 units with values carried as hi + lo pairs
(h2_construct_opts.fp64_products = 0, the default).  Row by row they agree with
the same matrix's float64-arithmetic products (fp64_products = 1) within 1e-13
of max|y| and with the oracle's float64 H^2 product within 1e-12; a leaf's own
block (kappa(x, x) = 0) and single-leaf trees follow the dense product; a
captured product replays the same arithmetic."""
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


CASES = [
    ("cube", lambda: I.uniform_cube(6000, 3, seed=41), 64, 1e-7, 6, (7, 10), False),
    ("cube_deep", lambda: I.uniform_cube(20000, 3, seed=42), 32, 1e-9, 6, (1, 2), True),
    ("spheres3", lambda: I.three_spheres(15000, seed=43), 64, 1e-8, 7, (7, 10), False),
    # coordinates far from the origin: the offsets from the cell centres carry the digits
    ("shifted", lambda: I.uniform_cube(8000, 3, seed=44) * 1e-3 + 1000.0, 64, 1e-8, 6, (1, 2), True),
]


@pytest.mark.parametrize("name,make,q,eps,g,tau,ilr", CASES, ids=[c[0] for c in CASES])
def test_float_float_products(H2, name, make, q, eps, g, tau, ilr):
    pts = make()
    n = len(pts)
    z = I.standard_normal(n, seed=45)
    t = H2.Tree(dev(pts), q, tau=tau)
    hd = H2.Hidr(t, g, g, il_reduce=ilr)
    Adf = H2.H2Matrix(t, hd, "coulomb", (), eps, "fp64")
    A64 = H2.H2Matrix(t, hd, "coulomb", (), eps, "fp64", fp64_products=True)
    assert json.loads(Adf.stats())["fp64_products"] is False
    assert json.loads(A64.stats())["fp64_products"] is True
    Z = dev(z)
    ydf = Adf.matvec(Z).cpu().numpy()
    y64 = A64.matvec(Z).cpu().numpy()
    assert_rows_close(ydf, y64, 1e-13, f"{name}: float-float vs float64 products")
    o = O.tree_build(pts, q, tau)
    yo = O.H2(o, O.Hidr(o, g, g, il_reduce=ilr), "coulomb", (), eps).matvec(z)
    assert_rows_close(ydf, yo, 1e-12, f"{name}: float-float products vs the oracle's H^2 product")
    # a captured product replays the same kernels
    y = torch.empty_like(Z)
    G = Adf.capture_matvec(Z, y)
    y.zero_()
    G.launch()
    torch.cuda.synchronize()
    assert_rows_close(y.cpu().numpy(), ydf, 1e-14, "replay")
    G.free()
    for h in (Adf, A64, hd, t):
        h.free()


@pytest.mark.parametrize("n,q", [(100, 500), (300, 40)])
def test_float_float_small_trees_equal_the_dense_product(H2, n, q):
    """A single leaf (only its own block, kappa(x, x) = 0) and a small tree
    with no reduction and no truncation: the product equals the dense one
    (1e-10, the oracle's own bound for this case) and the float64-arithmetic
    product (1e-13)."""
    pts = I.uniform_cube(n, 3, seed=46)
    z = I.standard_normal(n, seed=47)
    t = H2.Tree(dev(pts), q)
    hd = H2.Hidr(t, 25, 25)  # 25^3 > n: no reduction
    A = H2.H2Matrix(t, hd, "coulomb", (), 0.0, "fp64")
    B = H2.H2Matrix(t, hd, "coulomb", (), 0.0, "fp64", fp64_products=True)
    y = A.matvec(dev(z)).cpu().numpy()
    assert_rows_close(y, B.matvec(dev(z)).cpu().numpy(), 1e-13, "float64 products")
    assert_rows_close(y, O.dense_matvec(pts, "coulomb", (), z), 1e-10, "dense")
    for h in (A, B, hd, t):
        h.free()


@pytest.mark.parametrize("kern,kp,eps", [("coulomb", (), 1e-9), ("gaussian", (0.3,), 1e-8), ("multiquadric", (), 1e-8)])
def test_float_float_qr_equals_float64_qr(H2, kern, kp, eps):
    """The float64 form's QR in float-float arithmetic (the default) and in
    float64 arithmetic (fp64_qr): equal ranks and skeletons, U within
    64 u' c / eps with u' = 2^-46 (the float pairs' rounding in place of
    float64's), and the oracle's H^2 product within 1e-12 row by row."""
    n, q, g = 8000, 64, 6
    pts = I.uniform_cube(n, 3, seed=48)
    z = I.standard_normal(n, seed=49)
    t = H2.Tree(dev(pts), q, tau=(1, 2))
    hd = H2.Hidr(t, g, g, il_reduce=True)
    A = H2.H2Matrix(t, hd, kern, kp, eps, "fp64")
    B = H2.H2Matrix(t, hd, kern, kp, eps, "fp64", fp64_qr=True)
    assert json.loads(A.stats())["fp64_qr"] is False and json.loads(B.stats())["fp64_qr"] is True
    ka, kb = A.get("rank"), B.get("rank")
    assert np.array_equal(ka, kb)
    assert np.array_equal(A.get("skel"), B.get("skel"))
    nc = A.get("ncand")
    Ua, Ub = A.get("U"), B.get("U")
    off = np.concatenate([[0], np.cumsum(ka.astype(np.int64) * nc)])
    for i in range(t.nnodes):
        if ka[i] == 0:
            continue
        ua, ub = Ua[off[i]:off[i + 1]], Ub[off[i]:off[i + 1]]
        tol = 64 * 2.0 ** -46 * nc[i] / eps
        assert np.max(np.abs(ua - ub)) <= tol * max(1.0, np.abs(ub).max()), i
    o = O.tree_build(pts, q, (1, 2))
    yo = O.H2(o, O.Hidr(o, g, g, il_reduce=True), kern, kp, eps).matvec(z)
    assert_rows_close(A.matvec(dev(z)).cpu().numpy(), yo, 1e-12, f"{kern}: float-float QR vs the oracle")
    for h in (A, B, hd, t):
        h.free()
