"""bench.py's workload plumbing on the CPU: every workload names the fields the
GPU and oracle legs read, the point and right-hand-side generators give the
shapes and types the legs expect, and fixed-g workloads skip the calibration."""
import numpy as np

import bench


def test_workloads_are_complete():
    for name, wl in bench.WORKLOADS.items():
        for key in ("n", "d", "kernel", "kparams", "q", "eps", "prec", "seed", "rows"):
            assert key in wl, (name, key)
        assert wl["prec"] in ("fp64", "mixed")
        if "compare" in wl:
            assert wl["compare"] in bench.WORKLOADS
        tau = wl.get("tau", (7, 10))
        assert 0 < tau[0] / tau[1] <= 0.7  # the paper's range for eq. (1)


def test_generators_small():
    for name, wl in bench.WORKLOADS.items():
        n = 1000
        pts = bench.workload_points(wl, n, wl["seed"])
        assert pts.shape == (n, wl["d"]) and pts.dtype == np.float64, name
        zm, z = bench.workload_rhs(wl, n, wl["seed"] + 7)
        R = wl.get("rhs", 1)
        if R == 1:
            assert zm.shape == (n,) and zm.dtype == np.float64 and zm is z
        else:
            assert zm.shape == (n, R) and zm.dtype == np.float32
            assert z.shape == (n,) and z.dtype == np.float64 and np.array_equal(z, zm[:, 0].astype(np.float64))


def test_fixed_g_skips_the_calibration():
    assert bench.oracle_g(bench.WORKLOADS["gmix2m_fp64"]) == 20
    assert bench.oracle_g(bench.WORKLOADS["sphere8m_mixed16"]) == 6
