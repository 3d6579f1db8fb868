"""Pins of the oracle's operator y = (alpha I + S) x against facts that do not
come from the oracle: the worked example of Eqs. 2-6, skew-symmetry
invariants, unit-vector probing against the input arrays, a closed form on a
path graph, and numpy's dense product."""
import json
import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import GOLDEN


def _from_triplets(n, trip):
    trip = sorted(trip)
    keys = np.array([r * n + c for r, c, _ in trip], dtype=np.int64)
    A = W.from_keys(n, keys, "uniform", 0)
    A.val = np.array([v for _, _, v in trip], dtype=np.float64)
    return A


def test_worked_example_eqs_2_6():
    g = json.load(open(os.path.join(GOLDEN, "worked_example_eq2_6.json")))
    A = _from_triplets(g["n"], [tuple(t) for t in g["stored"]])
    x = np.array(g["x"])
    exp = np.array(g["expected_y"])
    assert np.array_equal(O.spmv_full(A, 0.0, x), exp)
    assert np.array_equal(O.spmv_sss(A, 0.0, x), exp)
    assert np.array_equal(O.dense_apply(A, 0.0, x), exp)
    # the shift adds alpha * x exactly
    assert np.array_equal(O.spmv_full(A, 2.0, x), exp + 2.0 * x)


@pytest.mark.parametrize("n,density,seed", [(1, 0.5, 1), (2, 1.0, 2), (17, 0.3, 3), (200, 0.05, 4), (500, 0.01, 5)])
def test_skew_invariants(n, density, seed):
    A = W.random_skew(n, density, seed)
    x = W.vector("uniform", n, seed)
    F = O.Full(A)
    alpha = 0.75
    y = F.apply(alpha, x)
    sx = F.apply(0.0, x)
    # x^T S x = 0 for skew S, up to rounding of a sum of |x_i s_ij x_j| terms
    scale = float(np.abs(x) @ F.abs_bound(0.0, x))
    assert abs(float(x @ sx)) <= 1e-14 * max(scale, 1e-300) + 1e-300
    # x^T (alpha I + S) x = alpha ||x||^2
    assert abs(float(x @ y) - alpha * float(x @ x)) <= 1e-14 * (scale + alpha * float(x @ x)) + 1e-300
    # (S x) . z = -(S z) . x
    z = W.vector("normal", n, seed + 100)
    sz = F.apply(0.0, z)
    zscale = float(np.abs(z) @ F.abs_bound(0.0, x))
    assert abs(float(sx @ z) + float(sz @ x)) <= 1e-13 * max(zscale, 1e-300) + 1e-300


@pytest.mark.parametrize("n,density,seed", [(9, 0.4, 11), (60, 0.1, 12)])
def test_unit_vector_probing_reconstructs_input(n, density, seed):
    """S e_j is column j of S exactly (each y_i is one product with 1.0);
    rebuilding S this way must give s_ij = l_ij below and -l_ji above the
    diagonal, read straight from the input arrays."""
    A = W.random_skew(n, density, seed)
    F = O.Full(A)
    S = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        S[:, j] = F.apply(0.0, e)
        assert np.array_equal(O.spmv_sss(A, 0.0, e), S[:, j])
    expect = np.zeros((n, n))
    for i in range(n):
        for k in range(A.rowptr[i], A.rowptr[i + 1]):
            expect[i, A.col[k]] = A.val[k]
            expect[A.col[k], i] = -A.val[k]
    assert np.array_equal(S, expect)
    assert np.array_equal(S, -S.T)


def test_path_graph_closed_form():
    """Path 0-1-...-(n-1) with every stored l_{i,i-1} = 1: (S x)_i = x_{i-1} - x_{i+1}."""
    n = 50
    keys = np.array([i * n + (i - 1) for i in range(1, n)], dtype=np.int64)
    A = W.from_keys(n, keys, "uniform", 0)
    A.val = np.ones(n - 1)
    x = W.vector("uniform", n, 7)
    xp = np.concatenate([[0.0], x, [0.0]])
    expect = xp[:-2] - xp[2:]
    assert np.array_equal(O.spmv_full(A, 0.0, x), expect)
    assert np.array_equal(O.spmv_sss(A, 0.0, x), expect)


@pytest.mark.parametrize("n,density,seed", [(300, 0.02, 21), (1000, 0.004, 22)])
def test_against_dense_numpy(n, density, seed):
    A = W.random_skew(n, density, seed)
    x = W.vector("uniform", n, seed)
    alpha = -0.3
    yd = alpha * x + O.dense(A) @ x           # numpy's dense matmul
    F = O.Full(A)
    bound = F.abs_bound(alpha, x)
    for y in (F.apply(alpha, x), O.spmv_sss(A, alpha, x)):
        assert np.all(np.abs(y - yd) <= 1e-14 * bound + 1e-300)


def test_block_apply_matches_columns():
    A = W.random_skew(150, 0.05, 31)
    X = W.vector("uniform", (150, 4), 31)
    F = O.Full(A)
    Y = F.apply_block(0.5, X)
    for c in range(4):
        assert np.array_equal(Y[:, c], F.apply(0.5, X[:, c]))


def test_permutation_identity():
    """P(Ax) = (P A P^T)(P x) with the reordered matrix built by numpy fancy indexing."""
    A = W.random_skew(80, 0.08, 41)
    x = W.vector("uniform", 80, 41)
    perm = np.random.default_rng(5).permutation(80)
    S = O.dense(A)
    Sp = S[np.ix_(perm, perm)]
    lhs = O.spmv_full(A, 0.2, x)[perm]
    rhs = 0.2 * x[perm] + Sp @ x[perm]
    assert np.allclose(lhs, rhs, rtol=0, atol=1e-13)


def test_validate_rejects_bad_input():
    A = W.random_skew(10, 0.5, 1)
    assert O.validate(A) == 0
    bad = W.random_skew(10, 0.5, 1)
    bad.col = bad.col.copy()
    r = int(np.argmax(np.diff(bad.rowptr) >= 2))
    k = bad.rowptr[r]
    bad.col[k], bad.col[k + 1] = bad.col[k + 1], bad.col[k]   # unsorted row
    assert O.validate(bad) != 0
    up = W.random_skew(10, 0.5, 1)
    up.col = up.col.copy()
    up.col[-1] = 9                                             # on/above the diagonal
    assert O.validate(up) != 0
