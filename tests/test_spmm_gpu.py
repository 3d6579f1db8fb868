"""GPU parity of pars3_spmm (k right-hand sides, row-major) against the FP64
oracle's block product, entry by entry with the tolerance of the single
product (tau * (|alpha||X_ic| + sum_j |s_ij||X_jc|))."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from paper_2407_17651_gb300 import _build
from paper_2407_17651_gb300 import pars3 as P

pytestmark = pytest.mark.gpu
TAU = {P.F64: 1e-12, P.F32: 2e-6, P.BF16: 2e-6}


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    O.build()
    torch.cuda.init()


def bf16_round(v):
    f = np.asarray(v, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def check_block(A, h, perm, dtype, alpha, X):
    if dtype == P.BF16:
        F = O.Full(W.SkewMatrix(A.n, A.rowptr, A.col, bf16_round(A.val)))
        Xr = X.astype(np.float32).astype(np.float64)
    else:
        F = O.Full(A)
        Xr = X
    ref = F.apply_block(alpha, Xr)
    bound = F.abs_bound_block(alpha, Xr)
    vt = torch.float64 if dtype == P.F64 else torch.float32
    Xp = torch.from_numpy(np.ascontiguousarray(X[perm])).to("cuda", vt)
    Y = torch.full_like(Xp, float("nan"))
    P.pars3_spmm(h, dtype, alpha, Xp, Y)
    torch.cuda.synchronize()
    P.pars3_check(h)
    y = Y.double().cpu().numpy()
    err = np.abs(y - ref[perm])
    lim = TAU[dtype] * bound[perm] + (1e-300 if dtype == P.F64 else 1e-30)
    bad = np.argwhere(~(err <= lim))
    assert bad.shape[0] == 0, f"{bad.shape[0]} entries off, first {bad[:3]}"
    return y


CASES = [
    ("band", lambda: W.banded_skew(3000, 40, 0.3, 5), {"T": 256, "W": 64}),
    ("grid2d", lambda: W.grid((90, 70), "uniform", 7), {"T": 1024, "W": 128}),
    ("grid3d", lambda: W.grid((22, 21, 20), "normal", 8), {"T": 1024, "W": 512}),
    ("grid+rand", lambda: W.grid_plus_random((20, 20, 20), 0.01, "normal", 9), {"T": 512, "W": 32}),
    ("rmat_long", lambda: W.rmat(12, 30000, seed=10), {"T": 256, "W": 256, "long_row": 40}),
]


@pytest.mark.parametrize("name,gen,kw", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("dtype", [P.F64, P.F32, P.BF16], ids=["f64", "f32", "bf16"])
@pytest.mark.parametrize("k", [1, 3, 4, 16, 32])
def test_spmm_parity(name, gen, kw, dtype, k):
    A = gen()
    perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, dtypes=7, **kw)
    P.pars3_upload(h)
    X = W.vector("uniform", (A.n, k), 40 + k)
    check_block(A, h, perm, dtype, -0.6, X)


def test_spmm_columns_equal_spmv_and_deterministic():
    A = W.grid_plus_random((16, 16, 16), 0.02, "normal", 3)
    perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, T=1024, W=256)
    P.pars3_upload(h)
    X = W.vector("uniform", (A.n, 4), 5)[perm]
    Xt = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    Y1 = torch.empty_like(Xt)
    Y2 = torch.empty_like(Xt)
    P.pars3_spmm(h, P.F64, 0.3, Xt, Y1)
    P.pars3_spmm(h, P.F64, 0.3, Xt, Y2)
    torch.cuda.synchronize()
    assert torch.equal(Y1, Y2)
    F = O.Full(A)
    for c in range(4):
        x = np.empty(A.n)
        x[perm] = X[:, c]
        ref = F.apply(0.3, x)[perm]
        assert np.all(np.abs(Y1[:, c].cpu().numpy() - ref) <= 1e-12 * F.abs_bound(0.3, x)[perm] + 1e-300)


def test_spmm_rejects_bad_k():
    A = W.random_skew(100, 0.05, 1)
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val)
    P.pars3_upload(h)
    X = torch.zeros((A.n, 33), dtype=torch.float64, device="cuda")
    Y = torch.zeros_like(X)
    with pytest.raises(P.Pars3Error) as e:
        P.pars3_spmm(h, P.F64, 1.0, X, Y)
    assert e.value.code == P.EINVAL


@pytest.mark.parametrize("dtype", [P.F64, P.F32], ids=["f64", "f32"])
def test_spmm_unaligned_blocks_use_scalar_lanes(dtype):
    """X, Y not 16-byte aligned: the product falls back to one column per
    lane and gives the same bits as the 16-byte-lane product."""
    A = W.grid_plus_random((14, 15, 16), 0.01, "normal", 21)
    perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, T=512, W=64, dtypes=7)
    P.pars3_upload(h)
    k = 8
    vt = torch.float64 if dtype == P.F64 else torch.float32
    X = torch.from_numpy(W.vector("uniform", (A.n, k), 22)[perm]).to("cuda", vt)
    Y = torch.empty_like(X)
    P.pars3_spmm(h, dtype, 0.7, X, Y)
    buf_x = torch.empty(A.n * k + 1, dtype=vt, device="cuda")
    buf_y = torch.empty(A.n * k + 1, dtype=vt, device="cuda")
    Xu = buf_x[1:].view(A.n, k)
    Yu = buf_y[1:].view(A.n, k)
    Xu.copy_(X)
    assert Xu.data_ptr() % 16 != 0
    P.pars3_spmm(h, dtype, 0.7, Xu, Yu)
    torch.cuda.synchronize()
    assert torch.equal(Y, Yu)
