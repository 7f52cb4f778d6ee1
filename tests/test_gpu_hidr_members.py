"""HiDR's top-down search over members against the copy-and-bin form.

The default volume DataReduct of the top-down sets reads each X_j* in place
(chunk and member boxes, the members entered in the reference grid's cells);
H2_HIDR_COPY_SETS copies every set out and bins it entry by entry.  Both
compute, for every grid point, the float64-nearest point of the same set with
ties to the smaller label, so X_i* and Y_i* must be identical element by
element, and a second run identical to the first (the member search's
visiting order depends on atomics; its result must not).  The cases cover both
of its forms: members in every cell they overlap, and, where the member-cell
pairs exceed the list's capacity (coarse levels, large member boxes), members
in their centre cell with widened bounds; 2D and 3D, flat and clustered sets,
with and without the interaction-list reduction.  The oracle comparison of the
same sets is in test_gpu_parity.py and test_gpu_parity_il_reduce.py."""
import numpy as np
import pytest

from paper_2206_01885_gb300 import inputs as I

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


def flat3d(n, seed):
    p = I.uniform_cube(n, 3, seed=seed)
    p[:, 2] = 0.25  # one coordinate constant: a flat axis in every box
    return p


CASES = [
    ("cube3d_q64_g4", lambda: I.uniform_cube(23000, 3, seed=206), 64, 4, (1, 2)),
    ("cube3d_q256_g6", lambda: I.uniform_cube(40000, 3, seed=11), 256, 6, (1, 2)),
    ("cube3d_q128_g8", lambda: I.uniform_cube(60000, 3, seed=12), 128, 8, (1, 2)),
    ("sphere_q128_g5", lambda: I.sphere_surface(30000, seed=13), 128, 5, (1, 2)),
    ("spheres3_q64_g6", lambda: I.three_spheres(30000, seed=14), 64, 6, (7, 10)),
    ("gmix2d_q64_g16", lambda: I.gaussian_mixture(40000, seed=15, d=2), 64, 16, (1, 2)),
    ("cube2d_q32_g12", lambda: I.uniform_cube(20000, 2, seed=16), 32, 12, (7, 10)),
    ("flat3d_q64_g6", lambda: flat3d(15000, 17), 64, 6, (1, 2)),
]


@pytest.mark.parametrize("name,make,q,g,tau", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("ilr", [False, True], ids=["alg1", "ilr"])
def test_member_search_equals_copy(H2, name, make, q, g, tau, ilr):
    pts = make()
    t = H2.Tree(dev(pts), q, tau=tau)
    runs = []
    for copy in (False, False, True):
        hd = H2.Hidr(t, g, g, il_reduce=ilr, copy_sets=copy)
        runs.append((hd.get("x"), hd.get("y")))
        hd.free()
    (xc, xd), (yc, yd) = runs[2]
    for k, what in ((0, "member search"), (1, "member search, second run")):
        (mxc, mxd), (myc, myd) = runs[k]
        assert np.array_equal(mxc, xc) and np.array_equal(mxd, xd), f"{name}: X* of the {what}"
        if not (np.array_equal(myc, yc) and np.array_equal(myd, yd)):
            oa = np.concatenate([[0], np.cumsum(myc)])
            ob = np.concatenate([[0], np.cumsum(yc)])
            bad = next(i for i in range(len(yc))
                       if not np.array_equal(myd[oa[i]:oa[i + 1]], yd[ob[i]:ob[i + 1]]))
            pytest.fail(f"{name}: Y* of the {what} differs first at node {bad}: "
                        f"{myc[bad]} against {yc[bad]} labels")
    t.free()
