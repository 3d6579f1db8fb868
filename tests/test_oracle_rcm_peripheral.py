"""Pins of the oracle's pseudo-peripheral RCM start (George-Liu: from the
(degree, index) candidate, move to the smallest (degree, index) vertex of
the last BFS level while that strictly increases the eccentricity): a
hand-worked example, trees (whose pseudo-peripheral vertex is an end of a
diameter, computed here by all-pairs shortest paths), grid corners, and the
Cuthill-McKee order property."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import shortest_path

import oracle as O
import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def built():
    O.build()


def from_edges(n, edges):
    low = sorted({(max(a, b), min(a, b)) for a, b in edges})
    rp = np.zeros(n + 1, dtype=np.int32)
    for i, _ in low:
        rp[i + 1] += 1
    rp = np.cumsum(rp).astype(np.int32)
    col = np.array([j for _, j in low], dtype=np.int32)
    return W.SkewMatrix(n, rp, col, np.ones(len(low)))


def ecc(A, v):
    L = sp.csr_matrix((np.ones(A.col.size), A.col, A.rowptr), shape=(A.n, A.n))
    G = L + L.T
    d = shortest_path(G, unweighted=True, indices=[v])[0]
    return int(d[np.isfinite(d)].max())


def test_hand_worked_spider():
    g = json.load(open(os.path.join(HERE, "golden", "rcm_spider_peripheral.json")))
    A = from_edges(g["n"], g["edges"])
    perm, b0, b1 = O.rcm(A, peripheral=True)
    assert perm.tolist() == g["perm_peripheral"]
    assert (b0, b1) == (g["bw_before"], g["bw_after"])
    perm2, _, _ = O.rcm(A, peripheral=False)
    assert perm2.tolist() == g["perm_min_degree"]


@pytest.mark.parametrize("seed", range(8))
def test_tree_start_is_a_diameter_end(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(20, 120))
    edges = [(i, int(rng.integers(0, i))) for i in range(1, n)]
    A = from_edges(n, edges)
    perm, _, _ = O.rcm(A, guard=False, peripheral=True)
    start = int(perm[-1])   # the first vertex of the Cuthill-McKee order
    L = sp.csr_matrix((np.ones(A.col.size), A.col, A.rowptr), shape=(n, n))
    diam = int(shortest_path(L + L.T, unweighted=True).max())
    assert ecc(A, start) == diam


@pytest.mark.parametrize("shape", [(7, 5), (12, 3), (6, 6)])
def test_grid_start_is_a_corner(shape):
    A = W.grid(shape, "uniform", 1, permute=False)
    perm, _, _ = O.rcm(A, guard=False, peripheral=True)
    start = int(perm[-1])
    a, b = shape
    assert ecc(A, start) == (a - 1) + (b - 1)


@pytest.mark.parametrize("mk", [lambda: W.random_skew(150, 0.03, 2), lambda: W.rmat(8, 600, seed=3),
                                lambda: W.grid((9, 8, 3), "normal", 4)])
def test_permutation_and_level_order(mk):
    """Every component is laid out breadth-first from its start (levels
    non-decreasing along the Cuthill-McKee order), and the result is a
    permutation."""
    A = mk()
    perm, _, _ = O.rcm(A, guard=False, peripheral=True)
    assert np.array_equal(np.sort(perm), np.arange(A.n))
    cm = perm[::-1]
    L = sp.csr_matrix((np.ones(A.col.size), A.col, A.rowptr), shape=(A.n, A.n))
    G = (L + L.T).tocsr()
    pos = np.empty(A.n, dtype=np.int64)
    pos[cm] = np.arange(A.n)
    level = np.full(A.n, -1)
    for q, v in enumerate(cm):
        if level[v] < 0:   # a new component starts here
            d = shortest_path(G, unweighted=True, indices=[v])[0]
            comp = np.isfinite(d)
            level[comp] = d[comp].astype(int)
            members = np.sort(pos[comp])
            assert members[0] == q and members[-1] - members[0] + 1 == comp.sum()
            lv = level[cm[members[0]:members[-1] + 1]]
            assert np.all(np.diff(lv) >= 0)
