"""Pins for the oracle's tree and interaction lists (section 2.1, eq. (1)).

Each check compares the oracle with something other than itself: the paper's
1D worked example, a hand-computed quantisation, real-space geometry computed
here from the node boxes, and brute-force coverage of all point pairs."""
import json
import os

import numpy as np
import pytest

from oracle import h2_oracle as O
from paper_2206_01885_gb300 import inputs as I


def test_quantisation_golden():
    # 2D, lo = (0,0), side = 1, B = 31: (0.5, 0.25) -> cells (2^30, 2^29)
    # -> key bits 2*30 + 0 and 2*29 + 1; (1, 1) clamps to 2^31 - 1 in both.
    pts = np.array([[0.0, 0.0], [1.0, 1.0], [0.5, 0.25]])
    t = O.tree_build(pts, leaf_size=4)
    assert t.B == 31 and t.side == 1.0
    keys = dict(zip(t.perm.tolist(), t.key.tolist()))
    assert keys[0] == 0
    assert keys[2] == (1 << 60) | (1 << 59)
    assert keys[1] == (1 << 62) - 1


def test_duplicates_single_leaf():
    pts = np.tile(np.array([[0.3, 0.2, 0.1]]), (50, 1))
    t = O.tree_build(pts, leaf_size=4)
    assert t.nnodes == 1 and t.side == 0.0
    assert list(t.near(0)) == [0]


def _node_box(t, i):
    """real-space box of node i: lo + [c, c+1) * e * side / 2^B per dim"""
    level = int(t.level[i])
    e = 2.0 ** (t.B - level)
    c = np.zeros(t.d)
    pre = int(t.prefix[i])
    for b in range(level):
        for k in range(t.d):
            c[k] += ((pre >> (t.d * b + k)) & 1) << b
    unit = t.side / 2.0 ** t.B
    lo = t.lo + c * e * unit
    return lo, lo + e * unit


@pytest.mark.parametrize("d,n,q", [(2, 3000, 25), (3, 4000, 40), (1, 500, 7)])
def test_tree_invariants(d, n, q):
    pts = I.uniform_cube(n, d, seed=100 + d)
    t = O.tree_build(pts, q)
    # perm is a permutation, keys sorted, coordinates gathered
    assert np.array_equal(np.sort(t.perm), np.arange(n))
    assert np.all(np.diff(t.key.astype(np.float64)) >= 0)
    assert np.array_equal(t.x, pts[t.perm])
    # levels contiguous, parents precede children, children inside parent
    for l in range(t.nlevels):
        assert np.all(t.level[t.lptr[l]:t.lptr[l + 1]] == l)
    leaf_pts = 0
    for i in range(t.nnodes):
        if t.nchild[i] == 0:
            assert t.end[i] - t.begin[i] <= q
            assert t.end[i] > t.begin[i]
            leaf_pts += t.end[i] - t.begin[i]
        else:
            ch = range(t.fchild[i], t.fchild[i] + t.nchild[i])
            assert t.begin[t.fchild[i]] == t.begin[i]
            assert t.end[t.fchild[i] + t.nchild[i] - 1] == t.end[i]
            for a, b in zip(list(ch)[:-1], list(ch)[1:]):
                assert t.end[a] == t.begin[b]
            for c in ch:
                assert t.parent[c] == i and t.level[c] == t.level[i] + 1
            assert t.end[i] - t.begin[i] > q
    assert leaf_pts == n
    # every point lies in its leaf's real-space box (tolerance: rounding)
    for i in range(t.nnodes):
        if t.nchild[i]:
            continue
        lo, hi = _node_box(t, i)
        xs = t.x[t.begin[i]:t.end[i]]
        tol = 1e-12 * max(t.side, 1.0)
        assert np.all(xs >= lo - tol) and np.all(xs <= hi + tol)


def test_il_1d_worked_example(golden_dir):
    gold = json.load(open(os.path.join(golden_dir, "il_1d_example.json")))
    pts = ((np.arange(16) + 0.5) / 16.0)[:, None]
    for tau in [(1, 2), (6, 10), (7, 10), (9, 10)]:
        t = O.tree_build(pts, leaf_size=1, tau=tau)
        assert t.nlevels == 5 and list(np.diff(t.lptr)) == [1, 2, 4, 8, 16]
        for node, il in gold["interaction_lists"].items():
            mine = sorted(int(j) + 1 for j in t.far(int(node) - 1))  # paper numbers from 1
            assert mine == il, (tau, node, mine)


@pytest.mark.parametrize("d,n,q,seed", [(2, 900, 12, 1), (3, 700, 10, 2), (3, 500, 60, 3)])
def test_lists_cover_every_pair_once(d, n, q, seed):
    pts = I.uniform_cube(n, d, seed=seed)
    if seed == 3:  # clustered, adaptive tree with leaves on several levels
        pts = I.gaussian_mixture(n, seed=seed, ncomp=3, d=d)
    t = O.tree_build(pts, q)
    cover = np.zeros((n, n), dtype=np.int32)
    tau = 0.7
    for i in range(t.nnodes):
        bi = slice(t.begin[i], t.end[i])
        for j in t.far(i):
            bj = slice(t.begin[j], t.end[j])
            cover[bi, bj] += 1
            # eq. (1) checked in floating point from the real-space cell boxes
            lo_i, hi_i = _node_box(t, i)
            lo_j, hi_j = _node_box(t, j)
            lhs = np.linalg.norm(hi_i - lo_i) + np.linalg.norm(hi_j - lo_j)
            rhs = 2 * tau * np.linalg.norm((lo_i + hi_i) / 2 - (lo_j + hi_j) / 2)
            assert lhs <= rhs * (1 + 1e-12)
            assert i in t.far(j)  # symmetric
        for j in t.near(i):
            assert t.nchild[i] == 0 and t.nchild[j] == 0
            lo_i, hi_i = _node_box(t, i)
            lo_j, hi_j = _node_box(t, j)
            lhs = np.linalg.norm(hi_i - lo_i) + np.linalg.norm(hi_j - lo_j)
            rhs = 2 * tau * np.linalg.norm((lo_i + hi_i) / 2 - (lo_j + hi_j) / 2)
            assert lhs > rhs * (1 - 1e-12)
            cover[bi, slice(t.begin[j], t.end[j])] += 1
            assert i in t.near(j)
    assert np.all(cover == 1)


def test_same_level_stencil_3d():
    # at tau = 0.7 in 3D, same-level cells are admissible iff |v|^2 >= 8, so a
    # cell deep inside a uniform grid has 81 near neighbours (offsets with
    # |v|^2 <= 6); checked with the real-space form of eq. (1) below
    offs = [(a, b, c) for a in range(-3, 4) for b in range(-3, 4) for c in range(-3, 4)]
    near = [v for v in offs if not (2 * np.sqrt(3) <= 2 * 0.7 * np.linalg.norm(v))]
    assert len(near) == 81
    g = 16
    centers = (np.stack(np.meshgrid(*[np.arange(g)] * 3, indexing="ij"), -1).reshape(-1, 3) + 0.5) / g
    pts = np.concatenate([centers, [[0.0, 0.0, 0.0], [1.0, 1.0, 1.0]]])
    t = O.tree_build(pts, leaf_size=1)
    l4 = [i for i in range(t.lptr[4], t.lptr[5])]
    # pick the leaf containing the centre cell (8,8,8)
    target = None
    for i in l4:
        lo, hi = _node_box(t, i)
        if np.all(lo <= 8.5 / 16) and np.all(hi > 8.5 / 16):
            target = i
    assert target is not None
    nb = [j for j in t.near(target) if t.level[j] == 4]
    assert len(nb) == 81
