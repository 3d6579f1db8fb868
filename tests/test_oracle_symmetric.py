"""Pins of the oracle's symmetric variant (mirror sign +1: S = L + L^T, the
case the paper says its method also covers -- abstract, Sec. 5).  Each pin
comes from outside the oracle: the input arrays themselves, a closed form,
an invariant, scipy.sparse, or the skew variant's own pins."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import workloads as W


@pytest.fixture(scope="module", autouse=True)
def built():
    O.build()


MATS = [
    lambda: W.random_skew(60, 0.1, 1, "normal"),
    lambda: W.grid((7, 6), "uniform", 2),
    lambda: W.banded_skew(80, 9, 0.5, 3),
    lambda: W.rmat(7, 300, seed=4),
]


def lower_csr(A):
    return sp.csr_matrix((A.val, A.col, A.rowptr), shape=(A.n, A.n))


@pytest.mark.parametrize("mk", MATS)
def test_unit_probing_gives_the_stored_entries_on_both_sides(mk):
    A = mk()
    F = O.Full(A, +1.0)
    L = lower_csr(A).toarray()
    for j in range(A.n):
        e = np.zeros(A.n)
        e[j] = 1.0
        col = F.apply(0.0, e)
        # rows below j carry l_ij, rows above j carry l_ji: exactly the inputs
        assert np.array_equal(col[j + 1:], L[j + 1:, j])
        assert np.array_equal(col[:j], L[j, :j])
        assert col[j] == 0.0


@pytest.mark.parametrize("mk", MATS)
def test_symmetric_plus_skew_is_twice_the_lower_triangle(mk):
    A = mk()
    x = W.vector("normal", A.n, 5)
    ys = O.Full(A, +1.0).apply(0.0, x)
    yk = O.Full(A, -1.0).apply(0.0, x)
    ref = 2.0 * (lower_csr(A) @ x)
    bound = 2.0 * (abs(lower_csr(A)) @ np.abs(x)) + (abs(lower_csr(A)).T @ np.abs(x))
    assert np.all(np.abs((ys + yk) - ref) <= 1e-14 * bound + 1e-300)


@pytest.mark.parametrize("mk", MATS)
def test_quadratic_form_closed_form(mk):
    A = mk()
    x = W.vector("uniform", A.n, 6)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    q = 2.0 * np.sum(A.val * x[rows] * x[A.col])
    y = O.Full(A, +1.0).apply(0.0, x)
    assert abs(float(x @ y) - q) <= 1e-12 * (2.0 * np.sum(np.abs(A.val * x[rows] * x[A.col])) + 1e-300)


def test_chain_closed_form():
    """l_{i,i-1} = -1 on a chain, alpha = 2: the second-difference matrix,
    whose product with the ones vector is (1, 0, ..., 0, 1)."""
    n = 50
    rp = np.concatenate([[0], np.arange(n)]).astype(np.int32)
    col = np.arange(n - 1, dtype=np.int32)
    A = W.SkewMatrix(n, rp, col, -np.ones(n - 1))
    y = O.Full(A, +1.0).apply(2.0, np.ones(n))
    ref = np.zeros(n)
    ref[0] = ref[-1] = 1.0
    assert np.array_equal(y, ref)
    assert np.array_equal(O.spmv_sss(A, 2.0, np.ones(n), +1.0), ref)


@pytest.mark.parametrize("mk", MATS)
def test_sss_and_dense_agree_with_full(mk):
    A = mk()
    x = W.vector("normal", A.n, 7)
    yf = O.Full(A, +1.0).apply(0.3, x)
    ys = O.spmv_sss(A, 0.3, x, +1.0)
    yd = 0.3 * x + O.dense(A, +1.0) @ x
    S = O.dense(A, +1.0)
    assert np.array_equal(S, S.T)
    bound = 0.3 * np.abs(x) + np.abs(S) @ np.abs(x)
    assert np.all(np.abs(yf - ys) <= 1e-14 * bound + 1e-300)
    assert np.all(np.abs(yf - yd) <= 1e-14 * bound + 1e-300)


@pytest.mark.parametrize("mk", MATS)
def test_split_reconstructs_the_permuted_symmetric_matrix(mk):
    A = mk()
    perm = np.random.default_rng(8).permutation(A.n).astype(np.int32)
    s = O.split(A, perm, 32, 32, mirror=+1.0)
    S = O.dense(A, +1.0)
    P = S[np.ix_(perm, perm)]
    B = sp.csr_matrix((s["val"], s["col"], s["rowptr"]), shape=(A.n, A.n)).toarray()
    assert np.array_equal(B, np.tril(P, -1))
