"""The seeded input generators: every family yields a valid strict-lower
pattern, is deterministic in its seed, and has the structure its docstring
states (sizes of the named workloads, grid degrees, R-MAT counts, the
finite-element-like coupling)."""
import math

import numpy as np
import pytest

import workloads as W


def valid_lower(A):
    rp, col = np.asarray(A.rowptr), np.asarray(A.col)
    assert rp[0] == 0 and rp[-1] == col.size and np.all(np.diff(rp) >= 0)
    rows = np.repeat(np.arange(A.n), np.diff(rp))
    assert np.all(col < rows) and np.all(col >= 0)
    same = rows[1:] == rows[:-1]
    assert np.all(col[1:][same] > col[:-1][same])   # sorted, unique
    assert np.all(np.isfinite(A.val)) and A.val.size == col.size


def full_degrees(A):
    d = np.diff(A.rowptr).astype(np.int64)
    np.add.at(d, A.col, 1)
    return d


@pytest.mark.parametrize("mk", [
    lambda s: W.random_skew(300, 0.02, s),
    lambda s: W.banded_skew(500, 17, 0.4, s),
    lambda s: W.grid((13, 9), "uniform", s),
    lambda s: W.grid((5, 6, 7), "normal", s),
    lambda s: W.grid_plus_random((8, 8, 8), 0.02, "normal", s),
    lambda s: W.rmat(9, 2000, seed=s),
    lambda s: W.fem_grid2d(7, 9, 3, "normal", s),
])
def test_valid_and_deterministic(mk):
    A, B, C = mk(3), mk(3), mk(4)
    valid_lower(A)
    assert np.array_equal(A.rowptr, B.rowptr) and np.array_equal(A.col, B.col) and np.array_equal(A.val, B.val)
    assert not (np.array_equal(A.col, C.col) and np.array_equal(A.val, C.val))


def test_grid_degrees_and_counts():
    A = W.grid((11, 7), "uniform", 1)
    assert A.n == 77 and A.nnz == 10 * 7 + 11 * 6
    d = full_degrees(A)
    assert sorted(np.unique(d).tolist()) == [2, 3, 4]
    assert int(np.sum(d == 4)) == 9 * 5


def test_fem_like_coupling():
    a, b, dofs = 6, 8, 3
    A = W.fem_grid2d(a, b, dofs, "normal", 2, permute=False)
    assert A.n == a * b * dofs
    node_pairs = a * (b - 1) + (a - 1) * b + 2 * (a - 1) * (b - 1)   # 9-point stencil, each pair once
    assert A.nnz == a * b * dofs * (dofs - 1) // 2 + node_pairs * dofs * dofs
    d = full_degrees(A)
    # an interior unknown couples to all unknowns of 9 nodes but itself
    interior = [((i * b) + j) * dofs + k for i in range(1, a - 1) for j in range(1, b - 1) for k in range(dofs)]
    assert np.all(d[interior] == 9 * dofs - 1)
    corner = np.arange(dofs)
    assert np.all(d[corner] == 4 * dofs - 1)
    valid_lower(W.fem_grid2d(a, b, dofs, "normal", 2))


def test_rmat_exact_count_no_self_loops():
    A = W.rmat(10, 3000, seed=5)
    assert A.n == 1024 and A.nnz == 3000
    valid_lower(A)


def test_named_small_config_and_batch_shapes():
    A, alpha, x = W.config0()
    assert (A.n, A.nnz, alpha, x.shape) == (20000, 39700, 0.0, (20000,))
    shapes = W.config4_shapes()
    assert len(shapes) == 64
    for shp in shapes:
        n = int(np.prod(shp))
        assert len(shp) in (2, 3)
        assert 0.8e4 <= n <= 5.6e5   # rounding of the grid sides around [1e4, 5e5]
    ns = [int(np.prod(s)) for s in shapes]
    # log-uniform: the geometric mean sits near sqrt(1e4 * 5e5)
    gm = math.exp(np.mean(np.log(ns)))
    assert 2.5e4 < gm < 2.5e5
