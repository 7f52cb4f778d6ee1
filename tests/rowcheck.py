"""Element-by-element comparison of two products.

Every row must satisfy |got_i - want_i| <= tol * max_j |want_j|, so a few bad
rows cannot hide inside a relative 2-norm; the 2-norm bound
||got - want|| <= tol ||want|| is checked beside it.  A failure names the worst
row."""
import numpy as np


def assert_rows_close(got, want, tol, what=""):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    assert got.shape == want.shape, (what, got.shape, want.shape)
    diff = np.abs(got - want)
    scale = float(np.max(np.abs(want))) if want.size else 0.0
    i = int(np.argmax(diff)) if diff.size else 0
    worst = float(diff.flat[i]) if diff.size else 0.0
    assert worst <= tol * scale, (
        f"{what}: row {i}: |got - want| = {worst:.3e} > {tol:.1e} * max|want| = {tol * scale:.3e} "
        f"(got {float(got.flat[i]):.17g}, want {float(want.flat[i]):.17g}; elementwise ratio {worst / scale:.3e})")
    nd, nw = float(np.linalg.norm(got - want)), float(np.linalg.norm(want))
    assert nd <= tol * nw, f"{what}: ||got - want|| = {nd:.3e} > {tol:.1e} * ||want|| = {tol * nw:.3e}"
