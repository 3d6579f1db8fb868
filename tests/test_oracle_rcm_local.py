"""Pins of the oracle's local-edge RCM (a reordering variant for small-world
patterns, after the paper's remark that RCM's benefit depends on the pattern,
Sec. 4.1, Fig. 5): the ordering is the RCM of the edges that lie on a
triangle or a 4-cycle (edges between two vertices whose degree product
exceeds 4096 are kept untested).  Pinned by a hand-worked example, by
brute-force detection of short cycles on small graphs, by the grid-plus-
shortcuts case where the local edges are exactly the grid edges, and by the
degree-product rule on stars."""
import json
import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import GOLDEN
from workloads import generators as G


@pytest.fixture(scope="module", autouse=True)
def built():
    O.build()


def matrix_from_pairs(n, pairs, seed=0):
    keys = np.unique(np.array([max(a, b) * n + min(a, b) for a, b in pairs], dtype=np.int64))
    return W.from_keys(n, keys, "uniform", seed)


def test_hand_worked_triangle_with_pendant():
    g = json.load(open(os.path.join(GOLDEN, "rcm_local_hand_4.json")))
    A = matrix_from_pairs(g["n"], g["edges"])
    assert O.rcm(A, guard=False, local=True)[0].tolist() == g["expected_perm_new_to_old"]
    assert O.rcm(A, guard=False)[0].tolist() == g["expected_plain_rcm"]


def brute_local_edges(A):
    """Local edges by definition, with an explicit adjacency matrix."""
    n = A.n
    M = np.zeros((n, n), dtype=bool)
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    M[rows, A.col] = True
    M[A.col, rows] = True
    deg = M.sum(1)
    keep = []
    for u, v in zip(rows, A.col):
        if deg[u] * deg[v] > 4096:
            keep.append((u, v))
            continue
        nu = [a for a in np.nonzero(M[u])[0] if a != v]
        nv = [b for b in np.nonzero(M[v])[0] if b != u]
        tri = any(M[a, v] for a in nu)
        quad = any(M[a, b] for a in nu for b in nv if a != b)
        if tri or quad:
            keep.append((u, v))
    return keep


@pytest.mark.parametrize("seed", range(6))
def test_matches_brute_force_short_cycle_detection(seed):
    rng = np.random.default_rng(seed)
    n = 40
    pairs = set()
    for _ in range(70):
        a, b = rng.integers(0, n, 2)
        if a != b:
            pairs.add((int(max(a, b)), int(min(a, b))))
    A = matrix_from_pairs(n, sorted(pairs), seed)
    keep = brute_local_edges(A)
    K = matrix_from_pairs(n, keep, seed) if keep else W.from_keys(n, np.zeros(0, np.int64), "uniform", seed)
    assert np.array_equal(O.rcm(A, guard=False, local=True)[0], O.rcm(K, guard=False)[0])


@pytest.mark.parametrize("dims,extra", [((30, 20), 0.02), ((12, 10, 8), 0.01)])
def test_grid_plus_shortcuts(dims, extra):
    """Every grid edge lies on a 4-cycle and is kept; random shortcuts lie on
    no short cycle unless they happen to close one with grid edges (a few
    do).  The ordering is the RCM of the kept edges, and over the grid edges
    its bandwidth is no wider than plain RCM's, which the shortcuts steer."""
    seed = 31
    A = W.grid_plus_random(dims, extra, "normal", seed)
    n = A.n
    u, v = G.grid_edges(dims)
    gk = G._relabel(n, G._pairs_to_lower_keys(n, u, v), seed)
    keep = brute_local_edges(A)
    kk = np.array(sorted(int(a) * n + int(b) for a, b in keep), dtype=np.int64)
    assert np.setdiff1d(gk, kk).size == 0                      # every grid edge kept
    assert np.setdiff1d(kk, gk).size <= 0.005 * A.nnz          # few shortcuts survive
    perm = O.rcm(A, guard=False, local=True)[0]
    assert np.array_equal(perm, O.rcm(matrix_from_pairs(n, keep, seed), guard=False)[0])
    Gm = W.from_keys(n, gk, "normal", seed)
    assert O.bandwidth(Gm, perm) <= O.bandwidth(Gm, O.rcm(A, guard=False)[0])


def test_degree_product_rule_on_stars():
    big = matrix_from_pairs(5001, [(i, 0) for i in range(1, 5001)])      # 5000 x 1 > 4096: kept
    assert np.array_equal(O.rcm(big, guard=False, local=True)[0], O.rcm(big, guard=False)[0])
    small = matrix_from_pairs(101, [(i, 0) for i in range(1, 101)])      # 100 x 1: tested, on no cycle
    assert O.rcm(small, guard=False, local=True)[0].tolist() == list(range(100, -1, -1))


def test_guard_and_bandwidths_use_all_edges():
    A = W.grid_plus_random((20, 20), 0.05, "uniform", 4)
    perm, b0, b1 = O.rcm(A, guard=True, local=True)
    assert b0 == O.bandwidth(A) and b1 == O.bandwidth(A, perm) and b1 <= b0
