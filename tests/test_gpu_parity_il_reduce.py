"""GPU parity of HiDR with the interaction-list reduction (H2_HIDR_IL_REDUCE):
Y_i* = DataReduct(T_i, g2^d) u DataReduct(union of X_j*, j in IL(i), g2^d).

X_i*, Y_i* bit-exact against the oracle's Hidr(il_reduce=True) on the HiDR
parity cases (every DataReduct variant); the float64 H^2 matvec within 1e-12
of the oracle's and within 10 eps of the dense product; the mixed form within
10 eps of the oracle's float64 product; g2^d above 4096 refused."""
import json

import numpy as np
import pytest

from oracle import h2_oracle as O
from paper_2206_01885_gb300 import inputs as I
from rowcheck import assert_rows_close

from test_gpu_parity import HIDR_CASES, SURFACE_CASES, _hidr_points, dev

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


IL_CASES = [c + ("volume",) for c in HIDR_CASES if c[4] ** c[1] <= 4096 and c[5] ** c[1] <= 4096] + \
           [c + (m,) for c in SURFACE_CASES for m in ("surface", "fps")]


@pytest.mark.parametrize("name,d,n,q,g1,g2,method", IL_CASES, ids=[f"{c[0]}-{c[6]}" for c in IL_CASES])
def test_hidr_il_reduce_bit_exact(H2, name, d, n, q, g1, g2, method):
    pts = _hidr_points(name, d, n)
    t = H2.Tree(dev(pts), q)
    h = H2.Hidr(t, g1, g2, method=method, il_reduce=True)
    st = json.loads(h.stats())
    assert st["il_reduce"] is True and st["method"] == method
    o = O.tree_build(pts, q)
    oh = O.Hidr(o, g1, g2, method=method, il_reduce=True)
    for which in ["x", "y"]:
        cnt, data = h.get(which)
        off = np.concatenate([[0], np.cumsum(cnt)])
        for i in range(1, t.nnodes):
            assert np.array_equal(data[off[i]:off[i + 1]], oh.get(i, which)), (which, i)


def test_il_reduce_refuses_large_grids(H2):
    pts = I.uniform_cube(2000, 2, seed=3)
    t = H2.Tree(dev(pts), 64)
    with pytest.raises(H2.H2Error) as e:
        H2.Hidr(t, 4, 65, il_reduce=True)  # 65^2 = 4225 > 4096
    assert e.value.status == 1
    H2.Hidr(t, 4, 64, il_reduce=True)  # 64^2 = 4096 is accepted


@pytest.mark.parametrize("prec,eps,g", [("fp64", 1e-6, 5), ("mixed", 1e-5, 5)])
def test_il_reduce_h2_matvec(H2, prec, eps, g):
    n, q = 12000, 64
    pts = I.uniform_cube(n, 3, seed=53)
    z = I.standard_normal(n, seed=51)
    t = H2.Tree(dev(pts), q)
    h = H2.Hidr(t, g, g, il_reduce=True)
    A = H2.H2Matrix(t, h, "coulomb", (), eps, prec)
    y = A.matvec(dev(z)).cpu().numpy()
    o = O.tree_build(pts, q)
    yo = O.H2(o, O.Hidr(o, g, g, il_reduce=True), "coulomb", (), eps).matvec(z)
    assert_rows_close(y, yo, 1e-12 if prec == "fp64" else 10 * eps, f"{prec} H2 with IL reduction vs oracle")
    yd = O.dense_matvec(pts, "coulomb", (), z)
    assert np.linalg.norm(y - yd) <= 10 * eps * np.linalg.norm(yd)
