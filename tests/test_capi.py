"""The C ABI library builds, loads and exports every entry point declared in
include/h2.h; argument checks that precede any device work return their
documented status without a GPU."""
import ctypes as C
import os
import re

import pytest

from paper_2206_01885_gb300 import build as B
from paper_2206_01885_gb300 import h2

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return h2.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "h2.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(h2_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(L, name), name


def test_invalid_arguments_are_rejected_without_device_work(L):
    prm = h2._Params(64, 7, 10)
    out = C.c_void_p()
    st = L.h2_tree_build(None, 10, 3, 0, C.byref(prm), None, C.byref(out))
    assert st == 1 and out.value is None
    assert b"pts" in L.h2_last_error()
    pts = (C.c_double * 30)()
    assert L.h2_tree_build(pts, 10, 4, 0, C.byref(prm), None, C.byref(out)) == 1  # dim
    assert L.h2_tree_build(pts, 0, 3, 0, C.byref(prm), None, C.byref(out)) == 1   # n
    bad = h2._Params(0, 7, 10)
    assert L.h2_tree_build(pts, 10, 3, 0, C.byref(bad), None, C.byref(out)) == 1  # leaf size
    bad = h2._Params(4, 7, 0)
    assert L.h2_tree_build(pts, 10, 3, 0, C.byref(bad), None, C.byref(out)) == 1  # tau
    assert L.h2_free(None) == 0
    bogus = (C.c_uint32 * 4)(1, 2, 3, 4)
    assert L.h2_free(bogus) == 1
    assert L.h2_hidr_reduce(bogus, 3, 3, None, C.byref(out)) == 1
    assert L.h2_hidr_reduce_ex(bogus, 3, 3, 0x400, None, C.byref(out)) == 1  # unknown flag
    assert b"flag" in L.h2_last_error()
    assert L.h2_hidr_reduce_ex(bogus, 3, 3, 3 | h2.HIDR_IL_REDUCE, None, C.byref(out)) == 1  # unknown method
    assert L.h2_hidr_reduce_ex(bogus, 3, 3, h2.HIDR_IL_REDUCE, None, C.byref(out)) == 1  # bogus tree
    assert L.h2_matvec(bogus, pts, pts, 1, 0, 10, 0, None) == 1
    assert L.h2_construct_batched(0, None, None, None, None, None, None, None, None) == 0
    assert L.h2_construct_batched(-1, None, None, None, None, None, None, None, None) == 1
    assert L.h2_construct_batched(2, None, None, None, None, None, None, None, None) == 1
    g = C.c_int(0)
    assert L.h2_calibrate(3, 99, None, 1e-6, pts, 5, pts, 5, 8, None, C.byref(g), None) == 1  # kernel id
    for kid in (5, 6):  # bump and power need a positive kparams[0]
        assert L.h2_calibrate(3, kid, None, 1e-6, pts, 5, pts, 5, 8, None, C.byref(g), None) == 1
        neg = (C.c_double * 4)(-1.0, 0.0, 0.0, 0.0)
        assert L.h2_calibrate(3, kid, neg, 1e-6, pts, 5, pts, 5, 8, None, C.byref(g), None) == 1
        assert b"kparams" in L.h2_last_error()
    b = C.c_int(0)
    assert L.h2_autotune_leaf(pts, 10, 3, 0, None, 0, 7, 1, None, 1e-5, 1, 1, None, C.byref(b), None) == 1
    cands = (C.c_int * 2)(64, 0)
    assert L.h2_autotune_leaf(pts, 10, 3, 0, cands, 2, 7, 1, None, 1e-5, 1, 1, None, C.byref(b), None) == 1
    assert b"leaf" in L.h2_last_error()
    gh = C.c_void_p()
    assert L.h2_matvec_graph_create(bogus, pts, pts, 1, 0, 10, None, C.byref(gh)) == 1 and gh.value is None
    assert L.h2_matvec_graph_launch(bogus, None) == 1
    buf = C.create_string_buffer(64)
    assert L.h2_get_stats(bogus, buf, 64) == 1
