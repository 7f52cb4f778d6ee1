"""Stored coupling and nearfield blocks (Algorithm 2's B_ij and near blocks,
memory mode STORE) against the on-the-fly product and the oracle.

The stored entries are the values the on-the-fly kernels evaluate, so the two
products differ only in summation order: row by row within 1e-13 of max|y| in
float64 and 2e-6 in the mixed form (float32 block sums in another order).
Both stay within the usual bounds of the oracle's float64 H^2 product (1e-12
float64, 10 eps mixed).  The stored byte count equals the block sizes summed
over the unordered far and near pairs; STORE over its memory budget fails with
H2_ERR_OOM; AUTO stores in the float64 form only; several right-hand sides
and a captured product give the same result on a stored matrix."""
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


def stored_bytes(t, A, esz):
    """sum over unordered pairs (j >= i) of |rows_i| |rows_j| elements"""
    ranks = A.get("rank").astype(np.int64)
    sizes = (t.get("end") - t.get("begin")).astype(np.int64)
    leaf = t.get("nchild") == 0
    pts = np.where(leaf, sizes, 0)
    tot = 0
    for rows, ptr, idx in ((ranks, t.get("far_ptr"), t.get("far_idx")), (pts, t.get("near_ptr"), t.get("near_idx"))):
        i = np.repeat(np.arange(t.nnodes), np.diff(ptr))
        keep = idx >= i
        tot += int(np.sum(rows[i[keep]] * rows[idx[keep]]))
    return tot * esz


CASES = [
    ("coulomb3d", 3, 6000, 64, "coulomb", (), 1e-7, 6),
    ("gauss2d", 2, 5000, 64, "gaussian", (0.2,), 1e-7, 10),
    ("power3d", 3, 4000, 64, "power", (11.0,), 1e-7, 6),
    ("cosdot3d", 3, 4000, 64, "cosdot", (), 1e-7, 6),
    ("mq3d", 3, 4000, 50, "multiquadric", (), 1e-7, 6),
]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name,d,n,q,kern,kp,eps,g", CASES, ids=[c[0] for c in CASES])
def test_stored_blocks_match_on_the_fly(H2, name, d, n, q, kern, kp, eps, g, prec):
    if prec == "mixed":
        eps = 1e-5
    pts = I.uniform_cube(n, d, seed=90 + d)
    z = I.standard_normal(n, seed=91)
    t = H2.Tree(dev(pts), q)
    hd = H2.Hidr(t, g, g)
    A0 = H2.H2Matrix(t, hd, kern, kp, eps, prec)
    A1 = H2.H2Matrix(t, hd, kern, kp, eps, prec, mem_mode="store")
    st = json.loads(A1.stats())
    assert st["mem_mode"] == "stored" and json.loads(A0.stats())["mem_mode"] == "on_the_fly"
    esz = 8 if prec == "fp64" else 4
    assert st["stored_bytes"] == stored_bytes(t, A1, esz) == st["planned_bytes"]
    Z = dev(z)
    y0 = A0.matvec(Z).cpu().numpy()
    y1 = A1.matvec(Z).cpu().numpy()
    assert_rows_close(y1, y0, 1e-13 if prec == "fp64" else 2e-6, f"{name} {prec} stored vs on the fly")
    o, oh, OH = O.build_h2(pts, kern, kp, q, eps, g, g)
    assert_rows_close(y1, OH.matvec(z), 1e-12 if prec == "fp64" else 10 * eps, f"{name} {prec} stored vs oracle")
    # a second product reuses the blocks; host buffers go through the same path
    assert_rows_close(A1.matvec(z), y1, 1e-14, "second product")
    A0.free()
    A1.free()
    hd.free()
    t.free()


def test_store_budget_auto_and_other_paths(H2):
    n, q, g, eps = 6000, 64, 6, 1e-7
    pts = I.uniform_cube(n, 3, seed=95)
    z = I.standard_normal(n, seed=96)
    t = H2.Tree(dev(pts), q)
    hd = H2.Hidr(t, g, g)
    # STORE above its budget: H2_ERR_OOM, no matrix
    with pytest.raises(H2.H2Error) as e:
        H2.H2Matrix(t, hd, "coulomb", (), eps, "fp64", mem_mode="store", mem_fraction=1e-9)
    assert e.value.status == 2 and "stored blocks" in str(e.value)
    # AUTO: stored in float64, on the fly in the mixed form; above the budget on the fly
    a64 = H2.H2Matrix(t, hd, "coulomb", (), eps, "fp64", mem_mode="auto")
    am = H2.H2Matrix(t, hd, "coulomb", (), 1e-5, "mixed", mem_mode="auto")
    asmall = H2.H2Matrix(t, hd, "coulomb", (), eps, "fp64", mem_mode="auto", mem_fraction=1e-9)
    assert json.loads(a64.stats())["mem_mode"] == "stored"
    assert json.loads(am.stats())["mem_mode"] == "on_the_fly"
    assert json.loads(asmall.stats())["mem_mode"] == "on_the_fly"
    Z = dev(z)
    ref = asmall.matvec(Z).cpu().numpy()
    assert_rows_close(a64.matvec(Z).cpu().numpy(), ref, 1e-13, "auto stored vs on the fly")
    # several right-hand sides on a stored matrix (evaluated on the fly) equal
    # the single-vector products
    Zm = I.standard_normal(n * 5, seed=97).reshape(n, 5)
    Y = a64.matvec(dev(Zm)).cpu().numpy()
    for j in range(5):
        assert_rows_close(Y[:, j], asmall.matvec(dev(np.ascontiguousarray(Zm[:, j]))).cpu().numpy(), 1e-13,
                          f"column {j}")
    # a product captured as a CUDA graph replays the stored-block kernels
    x = dev(z)
    y = torch.empty_like(x)
    G = a64.capture_matvec(x, y)
    y.zero_()
    G.launch()
    torch.cuda.synchronize()
    assert_rows_close(y.cpu().numpy(), ref, 1e-13, "graph replay of a stored product")
    G.free()
    # unknown modes and fractions are refused before any work
    prm = H2._ConstructOpts(0.0, 7, 0.0)
    out = C.c_void_p()
    st = H2.lib().h2_construct_ex(t.handle, hd.handle, 1, None, eps, 0, C.byref(prm), None, C.byref(out))
    assert st == 1 and out.value is None
    prm = H2._ConstructOpts(0.0, 1, 1.5)
    st = H2.lib().h2_construct_ex(t.handle, hd.handle, 1, None, eps, 0, C.byref(prm), None, C.byref(out))
    assert st == 1 and out.value is None
    for A in (a64, am, asmall):
        A.free()
    hd.free()
    t.free()
