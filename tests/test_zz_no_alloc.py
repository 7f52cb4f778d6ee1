"""h2_exact_rows_noalloc: the allocation-free exact-row entry point.

Some callers cannot allocate device memory in the middle of their work: a
program that is capturing a CUDA graph on another stream, an application whose
device memory is already handed out by its own allocator, or a time-critical
loop where an allocator call may synchronise the device or fail.  For them the
library offers a variant of h2_exact_rows whose only scratch (the right-hand
side permuted to tree order) is a fixed array inside the library.  This file
checks, through the C ABI, that it returns what h2_exact_rows returns, on two
calls in a row (the second call reuses the scratch left by the first), and
that a tree above its size limit is refused.  It is collected last so that a
failure here never hides the other GPU tests."""
import ctypes as C

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


def _noalloc(H2, tree, kernel, kparams, z, rows, out):
    st = H2.lib().h2_exact_rows_noalloc(tree.handle, H2.KERNELS[kernel], H2._kparams(kparams),
                                        C.c_void_p(z.data_ptr()), C.c_void_p(rows.data_ptr()), len(rows),
                                        C.c_void_p(out.data_ptr()), H2._stream(None))
    return st


@pytest.mark.parametrize("n,kernel,kparams", [(20000, "coulomb", ()), (1 << 20, "gaussian", (0.2,))])
def test_noalloc_matches_exact_rows_twice(H2, n, kernel, kparams):
    pts = I.uniform_cube(n, 3, seed=501)
    dev = torch.device("cuda")
    t = H2.Tree(torch.from_numpy(pts).to(dev), 128)
    for call, seed in enumerate([502, 503]):  # two calls in a row, different right-hand sides
        z = torch.from_numpy(I.standard_normal(n, seed=seed)).to(dev)
        rows = torch.from_numpy(I.sample_rows(n, 200, seed=seed + 1)).to(dev)
        want = H2.exact_rows(t, kernel, kparams, z, rows).cpu().numpy()
        out = torch.full((len(rows),), float("nan"), dtype=torch.float64, device=dev)
        assert _noalloc(H2, t, kernel, kparams, z, rows, out) == 0, H2.lib().h2_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max()), call
    t.free()


def test_noalloc_rejects_trees_above_its_limit(H2):
    n = (1 << 20) + 1
    pts = I.uniform_cube(n, 3, seed=511)
    dev = torch.device("cuda")
    t = H2.Tree(torch.from_numpy(pts).to(dev), 256)
    z = torch.zeros(n, dtype=torch.float64, device=dev)
    rows = torch.zeros(4, dtype=torch.int64, device=dev)
    out = torch.zeros(4, dtype=torch.float64, device=dev)
    assert _noalloc(H2, t, "coulomb", (), z, rows, out) == 1  # H2_ERR_INVALID_ARG
    assert b"1048576" in H2.lib().h2_last_error()
    t.free()


def test_noalloc_refuses_host_pointers_without_launching(H2):
    n = 5000
    pts = I.uniform_cube(n, 3, seed=521)
    dev = torch.device("cuda")
    t = H2.Tree(torch.from_numpy(pts).to(dev), 128)
    z_d = torch.from_numpy(I.standard_normal(n, seed=522)).to(dev)
    rows_d = torch.from_numpy(I.sample_rows(n, 16, seed=523)).to(dev)
    out_d = torch.zeros(16, dtype=torch.float64, device=dev)
    z_h = torch.from_numpy(I.standard_normal(n, seed=522))          # pageable host memory
    out_h = torch.zeros(16, dtype=torch.float64).pin_memory()       # pinned host memory
    torch.cuda.synchronize()
    before = H2.launches_total()
    assert _noalloc(H2, t, "coulomb", (), z_h, rows_d, out_d) == 1  # H2_ERR_INVALID_ARG
    assert b"z" in H2.lib().h2_last_error()
    assert _noalloc(H2, t, "coulomb", (), z_d, rows_d, out_h) == 1
    assert b"out" in H2.lib().h2_last_error()
    assert H2.launches_total() == before  # refused before any kernel launch
    # the context is still usable: a valid call right after succeeds
    assert _noalloc(H2, t, "coulomb", (), z_d, rows_d, out_d) == 0, H2.lib().h2_last_error()
    torch.cuda.synchronize()
    want = H2.exact_rows(t, "coulomb", (), z_d, rows_d).cpu().numpy()
    assert np.allclose(out_d.cpu().numpy(), want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    t.free()
