"""Pins of the oracle's RCM (Sec. 1 and Sec. 3.1.2) against a hand-worked
example, graph-theory facts (path and grid bandwidths), brute-force minimum
bandwidth, and an independent checker of the Cuthill-McKee visiting rules."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import GOLDEN


def _graph(n, edges):
    keys = np.array(sorted(max(a, b) * n + min(a, b) for a, b in edges), dtype=np.int64)
    return W.from_keys(n, keys, "uniform", 0)


def _adj(A):
    n = A.n
    nb = [[] for _ in range(n)]
    for i in range(n):
        for k in range(A.rowptr[i], A.rowptr[i + 1]):
            nb[i].append(int(A.col[k]))
            nb[int(A.col[k])].append(i)
    return nb


def check_cuthill_mckee(A, perm):
    """Independent verifier (not a re-run of the construction): the reversed
    perm must (a) be a permutation, (b) start a new component only once the
    previous ones are closed (no listed vertex has an unlisted neighbour), at
    the unlisted vertex of least (degree, index), (c) list every other vertex
    after its parent -- its earliest-listed neighbour -- with parents in
    non-decreasing position, and (d) list siblings by (degree, index)."""
    n = A.n
    cm = np.asarray(perm)[::-1]
    assert sorted(cm.tolist()) == list(range(n))
    nb = _adj(A)
    deg = [len(x) for x in nb]
    pos = np.empty(n, dtype=np.int64)
    pos[cm] = np.arange(n)
    order = sorted(range(n), key=lambda u: (deg[u], u))
    placed = np.zeros(n, dtype=bool)
    ptr = 0
    reach = -1
    prev_parent_pos = -1
    prev_key = None
    for k, v in enumerate(cm):
        earlier = [pos[u] for u in nb[v] if pos[u] < k]
        if not earlier:
            assert reach < k, f"component started at {k} while an earlier one was open"
            while placed[order[ptr]]:
                ptr += 1
            assert order[ptr] == v, f"start vertex at {k} is not the least (degree, index)"
            prev_parent_pos = -1
            prev_key = None
        else:
            p = min(earlier)
            assert p >= prev_parent_pos, f"parent order broken at {k}"
            key = (deg[v], int(v))
            if p == prev_parent_pos:
                assert key > prev_key, f"siblings not in (degree, index) order at {k}"
            prev_parent_pos = p
            prev_key = key
        placed[v] = True
        if nb[v]:
            reach = max(reach, max(pos[u] for u in nb[v]))
    return True


def test_hand_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "rcm_hand_9.json")))
    A = _graph(g["n"], g["edges"])
    perm, b0, b1 = O.rcm(A)
    assert perm.tolist() == g["expected_perm_new_to_old"]
    assert (b0, b1) == (g["bandwidth_before"], g["bandwidth_after"])
    assert check_cuthill_mckee(A, perm)


@pytest.mark.parametrize("n,seed", [(2, 1), (10, 2), (257, 3)])
def test_path_under_random_permutation(n, seed):
    p = np.random.default_rng(seed).permutation(n)
    A = _graph(n, [(p[i], p[i + 1]) for i in range(n - 1)])
    perm, b0, b1 = O.rcm(A)
    assert b1 == 1
    assert O.bandwidth(A, perm) == 1
    check_cuthill_mckee(A, perm)


@pytest.mark.parametrize("dims", [(7, 4), (20, 13), (200, 100)])
def test_grid_bandwidth(dims):
    """The a x b grid graph has bandwidth exactly min(a, b) (a classical
    result), so no ordering beats it; a corner-started BFS order reaches at
    most min(a, b) + 1."""
    A = W.grid(dims, "uniform", W.SEED_BASE, permute=True)
    perm, b0, b1 = O.rcm(A)
    assert min(dims) <= b1 <= min(dims) + 1
    assert b1 <= b0
    check_cuthill_mckee(A, perm)


def test_config0_bandwidth():
    A, _, _ = W.config0()
    perm, b0, b1 = O.rcm(A)
    assert b1 == 101 and b0 > 10000
    check_cuthill_mckee(A, perm)


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_minimum_bandwidth(seed):
    """For n <= 8, min over all n! orderings is a lower bound of the RCM bandwidth."""
    n = 7 if seed % 2 else 8
    A = W.random_skew(n, 0.35, 100 + seed)
    perm, b0, b1 = O.rcm(A)
    best = min(O.bandwidth(A, np.array(p, dtype=np.int32)) for p in itertools.permutations(range(n)))
    assert best <= b1 <= b0
    perm_ng, _, b1_ng = O.rcm(A, guard=False)
    check_cuthill_mckee(A, perm_ng)
    assert best <= b1_ng
    assert perm.tolist() == (list(range(n)) if b1_ng > b0 else perm_ng.tolist())


def test_guard_keeps_identity_for_banded_input():
    """A tridiagonal-plus-corner pattern that is already optimally banded:
    if RCM widened it the guard returns the identity."""
    n = 12
    edges = [(i, i + 1) for i in range(n - 1)] + [(i, i + 2) for i in range(n - 2)]
    A = _graph(n, edges)
    perm, b0, b1 = O.rcm(A)
    assert b0 == 2 and b1 <= 2
    perm_ng, _, b1_ng = O.rcm(A, guard=False)
    if b1_ng > b0:
        assert perm.tolist() == list(range(n))


def test_isolated_vertices_go_last():
    """Isolated vertices have degree 0: they start their own components first
    and, after the reversal, occupy the last positions."""
    n = 10
    A = _graph(n, [(0, 5), (5, 7), (7, 2)])
    perm, _, _ = O.rcm(A)
    iso = {1, 3, 4, 6, 8, 9}
    assert set(perm[-len(iso):].tolist()) == iso
    check_cuthill_mckee(A, perm)


def test_empty_and_single():
    for n in (0, 1):
        A = W.random_skew(n, 0.5, 1)
        perm, b0, b1 = O.rcm(A)
        assert perm.tolist() == list(range(n)) and b0 == b1 == 0
