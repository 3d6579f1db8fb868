"""GPU parity of the symmetric variant (PARS3_SPLIT_SYMMETRIC: S = L + L^T,
the case the paper says its method also covers -- abstract, Sec. 5) against
the oracle with mirror sign +1: products in fp64 / fp32 / bf16 over the
half path, halo rows, full-storage rows and long rows; SpMM; a batch that
mixes symmetric and skew handles; MRS rejects a symmetric handle."""
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


def oracle_full(A, dtype):
    if dtype == P.BF16:
        return O.Full(W.SkewMatrix(A.n, A.rowptr, A.col, bf16_round(A.val)), +1.0)
    return O.Full(A, +1.0)


CASES = [
    ("band_half", lambda: W.banded_skew(4000, 40, 0.3, 5), {"T": 256, "W": 64}),
    ("grid2d", lambda: W.grid((90, 70), "uniform", 7), {"T": 1024, "W": 128}),
    ("grid+rand", lambda: W.grid_plus_random((20, 20, 20), 0.01, "normal", 9), {"T": 512, "W": 32}),
    ("rmat_long", lambda: W.rmat(12, 30000, seed=10), {"T": 256, "W": 256, "long_row": 40}),
]


@pytest.mark.parametrize("name,gen,kw", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("dtype", [P.F64, P.F32, P.BF16], ids=["f64", "f32", "bf16"])
def test_symmetric_spmv_parity(name, gen, kw, dtype):
    A = gen()
    perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, dtypes=7, symmetric=True, **kw)
    P.pars3_upload(h)
    x = W.vector("uniform", A.n, 31)
    xr = x.astype(np.float32).astype(np.float64) if dtype == P.BF16 else x
    F = oracle_full(A, dtype)
    ref = F.apply(0.4, xr)[perm]
    bound = F.abs_bound(0.4, xr)[perm]
    vt = torch.float64 if dtype == P.F64 else torch.float32
    xp = torch.from_numpy(np.ascontiguousarray(x[perm])).to("cuda", vt)
    y = torch.full_like(xp, float("nan"))
    P.pars3_spmv(h, dtype, 0.4, xp, y)
    torch.cuda.synchronize()
    P.pars3_check(h)
    err = np.abs(y.double().cpu().numpy() - ref)
    assert np.all(err <= TAU[dtype] * bound + 1e-30), int(np.sum(~(err <= TAU[dtype] * bound + 1e-30)))


def test_symmetric_unit_probing_is_symmetric():
    A = W.banded_skew(300, 20, 0.4, 3, "normal")
    perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, T=64, W=32, symmetric=True)
    P.pars3_upload(h)
    S = np.zeros((A.n, A.n))
    e = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(e)
    for j in range(A.n):
        e.zero_()
        e[j] = 1.0
        P.pars3_spmv(h, P.F64, 0.0, e, y)
        S[:, j] = y.cpu().numpy()
    assert np.array_equal(S, S.T)
    D = O.dense(A, +1.0)
    assert np.array_equal(S, D[np.ix_(perm, perm)])


def test_symmetric_spmm_and_mixed_batch():
    mats = [(W.grid((40, 30), "normal", 41), {"T": 256, "W": 64}, True),
            (W.grid((12, 11, 10), "normal", 42), {"T": 512, "W": 128}, False),
            (W.rmat(11, 12000, seed=43, value_kind="normal"), {"T": 256, "W": 64, "long_row": 40}, True)]
    hs, perms, Xs, Ys, Fs = [], [], [], [], []
    k = 4
    for A, kw, sym in mats:
        perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
        h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, dtypes=7, symmetric=sym, **kw)
        P.pars3_upload(h)
        X = W.vector("uniform", (A.n, k), 44)
        hs.append(h)
        perms.append(perm)
        Fs.append((O.Full(A, +1.0 if sym else -1.0), X))
        Xs.append(torch.from_numpy(np.ascontiguousarray(X[perm])).cuda())
        Ys.append(torch.empty_like(Xs[-1]))
    P.pars3_spmm_batched(hs, P.F64, [0.5] * 3, Xs, Ys)
    torch.cuda.synchronize()
    for (F, X), perm, h, Xd, Y in zip(Fs, perms, hs, Xs, Ys):
        ref = F.apply_block(0.5, X)[perm]
        bound = F.abs_bound_block(0.5, X)[perm]
        assert np.all(np.abs(Y.cpu().numpy() - ref) <= 1e-12 * bound + 1e-300)
        Y1 = torch.empty_like(Y)
        P.pars3_spmm(h, P.F64, 0.5, Xd, Y1)
        torch.cuda.synchronize()
        assert torch.equal(Y, Y1)


def test_mrs_rejects_symmetric_handle():
    A = W.random_skew(200, 0.05, 5)
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, T=64, W=32, symmetric=True)
    P.pars3_upload(h)
    b = torch.ones(A.n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(P.Pars3Error) as e:
        P.pars3_mrs(h, 1.0, b, x)
    assert e.value.code == P.EUNSUPPORTED
