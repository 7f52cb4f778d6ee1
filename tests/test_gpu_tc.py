"""The mixed form's several-right-hand-side nearfield on the tensor cores.

With h2_construct_opts.tensor_core_products = 1, sixteen columns at a time run
through tcgen05.mma (kind tf32, kernel values and weights split as hi + lo,
three products per 32-source chunk, float32 accumulation folded per chunk);
remaining columns stay on the CUDA cores.  Row by row the product equals the
all-CUDA-core product (the default) within 2e-6 of max|y| (two
float32-accurate evaluations of the same sums) and the oracle's float64 H^2
product within 10 eps, for 16, 21 (16 + 5) and 32 columns, 2D and 3D, and
kernels of every form (1/r, exp(-r^2/h^2), cos(x . y))."""
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
    ("coulomb3d", 3, 9000, 100, "coulomb", (), 1e-5, 7, 16),
    ("coulomb3d_21", 3, 6000, 200, "coulomb", (), 1e-5, 6, 21),
    ("gauss2d_32", 2, 7000, 128, "gaussian", (0.2,), 1e-5, 10, 32),
    ("cosdot3d", 3, 5000, 64, "cosdot", (), 1e-5, 6, 16),
    ("sphere_q256", 3, 12000, 256, "coulomb", (), 1e-5, 6, 16),
]


@pytest.mark.parametrize("name,d,n,q,kern,kp,eps,g,R", CASES, ids=[c[0] for c in CASES])
def test_tensor_core_nearfield(H2, name, d, n, q, kern, kp, eps, g, R):
    pts = I.sphere_surface(n, seed=120) if name.startswith("sphere") else I.uniform_cube(n, d, seed=120 + d)
    Z = I.standard_normal(n * R, seed=121).reshape(n, R).astype(np.float32)
    t = H2.Tree(dev(pts), q)
    hd = H2.Hidr(t, g, g)
    Atc = H2.H2Matrix(t, hd, kern, kp, eps, "mixed", tensor_core_products=True)
    Acc = H2.H2Matrix(t, hd, kern, kp, eps, "mixed")
    Ytc = Atc.matvec(dev(Z)).cpu().numpy().astype(np.float64)
    Ycc = Acc.matvec(dev(Z)).cpu().numpy().astype(np.float64)
    o, oh, OH = O.build_h2(pts, kern, kp, q, eps, g, g)
    for j in range(R):
        assert_rows_close(Ytc[:, j], Ycc[:, j], 2e-6, f"{name} column {j}: tensor cores vs CUDA cores")
    for j in (0, R - 1):
        assert_rows_close(Ytc[:, j], OH.matvec(Z[:, j].astype(np.float64)), 10 * eps,
                          f"{name} column {j} vs the oracle")
    # the host-buffer path synchronises and checks the kernel's wait status
    Yh = Atc.matvec(Z)
    assert np.allclose(Yh, Ytc, rtol=0, atol=1e-6 * np.abs(Ytc).max())
    for h in (Atc, Acc, hd, t):
        h.free()
