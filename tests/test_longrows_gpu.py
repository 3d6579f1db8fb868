"""GPU parity of the long-row path on the shapes that stress it.

Long rows are cut into pieces of `piece` entries (default 192) and a shorter
last piece; each piece is one lane's sequential sum, laid out like the tile
slices, and the fold adds a row's pieces in order.  Shapes:
- one row of 14,400 entries (a hub vertex joined to every vertex of a 2D
  grid): hundreds of pieces of one row, spread over many blocks;
- thousands of short long rows (every row with more than two full-storage
  entries sent to the long list): one piece per row, slices of 32 rows'
  last pieces sorted by length;
- piece lengths from 8 to 255 on the hub row and on an R-MAT graph.
Tolerances as in test_spmv_gpu: |y - y_ref| <= tau * (|alpha||x_i| +
sum_j |s_ij||x_j|), tau = 1e-12 (fp64) and 2e-6 (fp32).  Two calls on the
same input must agree bit for bit, and the SpMM path must match column by
column.
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from paper_2407_17651_gb300 import _build
from paper_2407_17651_gb300 import pars3 as P

pytestmark = pytest.mark.gpu
TAU = {P.F64: 1e-12, P.F32: 2e-6}


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    O.build()
    torch.cuda.init()


def hub_plus_grid(a: int, seed: int) -> W.SkewMatrix:
    """a x a 5-point grid plus one hub vertex (the last index) joined to all
    a^2 grid vertices: the hub's row has a^2 full-storage entries."""
    u, v = W.grid_edges((a, a))
    n = a * a + 1
    hub = n - 1
    u = np.concatenate([np.asarray(u, np.int64), np.full(a * a, hub, np.int64)])
    v = np.concatenate([np.asarray(v, np.int64), np.arange(a * a, dtype=np.int64)])
    r, c = np.maximum(u, v), np.minimum(u, v)
    keys = np.unique(r * n + c)
    return W.from_keys(n, keys, "normal", seed, name=f"hub_grid{a}")


def product(h, dtype, alpha, xp_np, k=1):
    vt = torch.float64 if dtype == P.F64 else torch.float32
    xp = torch.from_numpy(np.ascontiguousarray(xp_np)).to("cuda", vt)
    y = torch.full_like(xp, float("nan"))
    if k == 1:
        P.pars3_spmv(h, dtype, alpha, xp, y)
    else:
        P.pars3_spmm(h, dtype, alpha, xp, y)
    torch.cuda.synchronize()
    P.pars3_check(h)
    return y.double().cpu().numpy()


def check_against_oracle(A, h, perm, dtype, alpha, x):
    F = O.Full(A)
    ref = F.apply(alpha, x)[perm]
    bound = F.abs_bound(alpha, x)[perm]
    y = product(h, dtype, alpha, x[perm])
    err = np.abs(y - ref)
    lim = TAU[dtype] * bound + (1e-300 if dtype == P.F64 else 1e-30)
    bad = np.nonzero(~(err <= lim))[0]
    assert bad.size == 0, f"{bad.size} rows off, worst {err[bad].max():.3e} at {bad[:5]}"
    return y


@pytest.mark.parametrize("dtype", [P.F64, P.F32])
def test_row_of_hundreds_of_pieces(dtype):
    A = hub_plus_grid(120, 5)
    perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, T=1024, W=32,
                      dtypes=P.dtype_bit(P.F64) | P.dtype_bit(P.F32))
    P.pars3_upload(h)
    info = P.pars3_info_get(h)
    assert info["long_rows"] >= 1 and info["long_pieces"] >= 14400 // 192   # 14,400 entries in one row
    assert P.pars3_layout_check(h) == 0
    for alpha, seed in ((0.5, 1), (0.0, 2)):
        x = W.vector("uniform", A.n, seed)
        y1 = check_against_oracle(A, h, perm, dtype, alpha, x)
        y2 = product(h, dtype, alpha, x[perm])
        assert np.array_equal(y1, y2)   # run-to-run bitwise
    h.close()


@pytest.mark.parametrize("dtype", [P.F64, P.F32])
def test_many_short_long_rows(dtype):
    A = W.grid((150, 150), "normal", 7)
    perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, T=4096, W=32, long_row=2,
                      dtypes=P.dtype_bit(P.F64) | P.dtype_bit(P.F32))
    P.pars3_upload(h)
    info = P.pars3_info_get(h)
    # most rows hold four entries: one piece per long row
    assert info["long_rows"] > 15000
    assert info["long_pieces"] == info["long_rows"]
    assert P.pars3_layout_check(h) == 0
    x = W.vector("uniform", A.n, 3)
    y1 = check_against_oracle(A, h, perm, dtype, 0.25, x)
    y2 = product(h, dtype, 0.25, x[perm])
    assert np.array_equal(y1, y2)
    h.close()


def test_spmm_on_a_row_of_many_pieces():
    A = hub_plus_grid(100, 9)
    perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, T=512, W=32, dtypes=P.dtype_bit(P.F32))
    P.pars3_upload(h)
    assert P.pars3_info_get(h)["long_pieces"] >= 2
    k = 4
    X = W.vector("uniform", (A.n, k), 4)
    Y = product(h, P.F32, 0.5, X[perm], k=k)
    F = O.Full(A)
    for c in range(k):
        ref = F.apply(0.5, X[:, c])[perm]
        bound = F.abs_bound(0.5, X[:, c])[perm]
        assert np.all(np.abs(Y[:, c] - ref) <= TAU[P.F32] * bound + 1e-30), c
    h.close()


@pytest.mark.parametrize("piece", [8, 37, 255])
@pytest.mark.parametrize("dtype", [P.F64, P.F32])
def test_piece_lengths(piece, dtype):
    """Pieces from 8 to 255 entries: the hub row and an R-MAT graph (power-law
    rows, several rows of many pieces, remainders of every length)."""
    for A in (hub_plus_grid(60, 3), W.rmat(13, 60000, seed=10)):
        perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
        h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, T=512, W=32, long_row=32, piece=piece,
                          dtypes=P.dtype_bit(P.F64) | P.dtype_bit(P.F32))
        P.pars3_upload(h)
        info = P.pars3_info_get(h)
        assert info["long_rows"] >= 1 and info["long_pieces"] >= info["long_entries"] // piece
        assert P.pars3_layout_check(h) == 0
        x = W.vector("uniform", A.n, piece)
        y1 = check_against_oracle(A, h, perm, dtype, 0.5, x)
        y2 = product(h, dtype, 0.5, x[perm])
        assert np.array_equal(y1, y2)
        k = 4
        X = W.vector("uniform", (A.n, k), piece + 1)
        Y = product(h, dtype, 0.5, X[perm], k=k)
        F = O.Full(A)
        for c in range(k):
            ref = F.apply(0.5, X[:, c])[perm]
            bound = F.abs_bound(0.5, X[:, c])[perm]
            assert np.all(np.abs(Y[:, c] - ref) <= TAU[dtype] * bound + 1e-30), c
        h.close()
