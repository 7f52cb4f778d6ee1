"""Widening beyond the hot-path table, to the same parity bar.

- One HiDR for every kernel (section 6.1.3): the reduced sets X_i*, Y_i* depend
  only on the points, so one tree and one HiDR serve Coulomb, Gaussians of
  bandwidth 10^k (k = -2..2), exponential, multiquadric, Table 1's bump
  kernel and cos(x . y), and the |x-y|^11 of section 5.2; each
  float64 product equals the oracle's H^2 product on the same reduction
  (1e-12) and the dense product within 10 eps.
- The paper's three-sphere dataset (section 6.1.1): three unit spheres with
  centres on a unit equilateral triangle; tree, lists and HiDR bit-exact,
  products as above, in both forms."""
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


KERNELS = [("coulomb", ()), ("gaussian", (0.01,)), ("gaussian", (0.1,)), ("gaussian", (1.0,)),
           ("gaussian", (10.0,)), ("gaussian", (100.0,)), ("exponential", (0.2,)), ("multiquadric", ()),
           ("bump", (0.1,)), ("power", (11.0,)), ("cosdot", ())]


def test_one_hidr_for_every_kernel(H2):
    n, q, g, eps = 10000, 64, 6, 1e-6
    pts = I.uniform_cube(n, 3, seed=80)
    z = I.standard_normal(n, seed=81)
    t = H2.Tree(dev(pts), q)
    hd = H2.Hidr(t, g, g)
    o = O.tree_build(pts, q)
    oh = O.Hidr(o, g, g)
    mats = H2.construct_batched([(t, hd, k, kp, eps, "fp64") for k, kp in KERNELS])
    Z = dev(z)
    for (kern, kp), A in zip(KERNELS, mats):
        y = A.matvec(Z).cpu().numpy()
        yo = O.H2(o, oh, kern, kp, eps).matvec(z)
        assert_rows_close(y, yo, 1e-12, f"{kern}{kp} vs oracle")
        yd = O.dense_matvec(pts, kern, kp, z)
        assert np.linalg.norm(y - yd) <= 10 * eps * np.linalg.norm(yd), (kern, kp)
        A.free()
    hd.free()
    t.free()


@pytest.mark.parametrize("prec,eps,g", [("fp64", 1e-8, 8), ("mixed", 1e-5, 6)])
def test_three_spheres(H2, prec, eps, g):
    n, q = 30000, 64
    pts = I.three_spheres(n, seed=82)
    z = I.standard_normal(n, seed=83)
    t = H2.Tree(dev(pts), q)
    o = O.tree_build(pts, q)
    for f in ["perm", "level", "parent", "begin", "end", "near_ptr", "near_idx", "far_ptr", "far_idx"]:
        got = t.get(f)
        assert np.array_equal(got, getattr(o, f).astype(got.dtype)), f
    hd = H2.Hidr(t, g, g)
    oh = O.Hidr(o, g, g)
    for which in ["x", "y"]:
        cnt, data = hd.get(which)
        off = np.concatenate([[0], np.cumsum(cnt)])
        for i in range(1, t.nnodes):
            assert np.array_equal(data[off[i]:off[i + 1]], oh.get(i, which)), (which, i)
    A = H2.H2Matrix(t, hd, "coulomb", (), eps, prec)
    y = A.matvec(dev(z)).cpu().numpy()
    yo = O.H2(o, oh, "coulomb", (), eps if prec == "fp64" else eps).matvec(z)
    tol = 1e-12 if prec == "fp64" else 10 * eps
    assert_rows_close(y, yo, tol, f"three spheres {prec} vs oracle")
    yd = O.dense_matvec(pts, "coulomb", (), z)
    assert np.linalg.norm(y - yd) <= 10 * eps * np.linalg.norm(yd)
    A.free()
    hd.free()
    t.free()
