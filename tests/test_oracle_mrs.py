"""Pins of the oracle's MRS iteration (Sec. 1: one product and one inner
product per iteration) against a 2x2 closed form, finite termination on
block-diagonal input, dense least squares over the Krylov space (the
defining minimal-residual property), monotone residuals and numpy.linalg.solve."""
import numpy as np
import pytest

import oracle as O
import workloads as W


def _dense_S(A):
    return O.dense(A)


def test_2x2_closed_form():
    """S = [[0, -a], [a, 0]]: (alpha I + S)^{-1} b = (alpha I - S) b / (alpha^2 + a^2)."""
    a, alpha = 1.7, 0.3
    A = W.from_keys(2, np.array([1 * 2 + 0], dtype=np.int64), "uniform", 0)
    A.val = np.array([a])
    b = np.array([0.25, -2.0])
    S = np.array([[0.0, -a], [a, 0.0]])
    exact = (alpha * b - S @ b) / (alpha ** 2 + a ** 2)
    F = O.Full(A)
    x, info = O.mrs(lambda v: F.apply(0.0, v), 2, alpha, b, rtol=1e-15)
    assert info["iters"] <= 2
    assert np.allclose(x, exact, rtol=1e-14, atol=1e-15)


def test_block_diagonal_terminates_at_two():
    """S = diag of identical 2x2 blocks: A has two eigenvalues, so the Krylov
    space stops growing at dimension 2 and MRS is exact at iteration 2."""
    m, a, alpha = 25, 0.9, 0.6
    n = 2 * m
    keys = np.array([(2 * k + 1) * n + 2 * k for k in range(m)], dtype=np.int64)
    A = W.from_keys(n, keys, "uniform", 0)
    A.val = np.full(m, a)
    b = W.vector("uniform", n, 3)
    F = O.Full(A)
    x, info = O.mrs(lambda v: F.apply(0.0, v), n, alpha, b, rtol=1e-14)
    assert info["iters"] == 2
    exact = np.linalg.solve(alpha * np.eye(n) + O.dense(A), b)
    assert np.allclose(x, exact, rtol=0, atol=1e-13)


@pytest.mark.parametrize("n,alpha,seed", [(40, 0.5, 1), (41, 0.05, 2)])
def test_iterates_minimize_residual_over_krylov_space(n, alpha, seed):
    """x_k = argmin ||b - A x|| over x0 + K_k(S, r0), computed by numpy QR +
    least squares on an explicitly built Krylov basis."""
    A = W.random_skew(n, 0.15, seed, "normal")
    S = O.dense(A)
    Am = alpha * np.eye(n) + S
    b = W.vector("uniform", n, seed)
    F = O.Full(A)
    x0 = np.zeros(n)
    for k in range(1, 9):
        xk, info = O.mrs(lambda v: F.apply(0.0, v), n, alpha, b, x0=x0, rtol=0.0, maxit=k)
        assert info["iters"] == k
        K = np.empty((n, k))
        v = b.copy()
        for c in range(k):
            K[:, c] = v
            v = S @ v
        Q, _ = np.linalg.qr(K)
        y, *_ = np.linalg.lstsq(Am @ Q, b, rcond=None)
        xls = Q @ y
        assert np.linalg.norm(xk - xls) <= 1e-10 * max(1.0, np.linalg.norm(xls))


def test_monotone_residual_and_solution():
    n, alpha = 300, 0.2
    A = W.random_skew(n, 0.03, 9, "normal")
    b = W.vector("uniform", n, 9)
    F = O.Full(A)
    true_res = lambda x: float(np.linalg.norm(b - F.apply(alpha, x)))
    x, info = O.mrs(lambda v: F.apply(0.0, v), n, alpha, b, rtol=1e-12, history=True, true_residual=true_res)
    h = np.array(info["hist"])
    assert np.all(np.diff(h) <= 1e-12 * h[0])
    assert true_res(x) <= 1e-12 * np.linalg.norm(b) * 1.0001
    exact = np.linalg.solve(alpha * np.eye(n) + O.dense(A), b)
    assert np.linalg.norm(x - exact) <= 1e-9 * np.linalg.norm(exact)


def test_recursive_estimate_tracks_true_residual():
    n, alpha = 200, 1.0
    A = W.random_skew(n, 0.05, 4, "normal")
    b = W.vector("uniform", n, 4)
    F = O.Full(A)
    for k in (3, 10, 25):
        x, info = O.mrs(lambda v: F.apply(0.0, v), n, alpha, b, rtol=0.0, maxit=k)
        tr = np.linalg.norm(b - F.apply(alpha, x))
        assert abs(info["est"] - tr) <= 1e-10 * np.linalg.norm(b)


def test_alpha_zero_rejected():
    A = W.random_skew(4, 0.5, 1)
    with pytest.raises(ValueError):
        O.mrs(lambda v: v, 4, 0.0, np.ones(4))
