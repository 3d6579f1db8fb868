"""Parity at the full sizes of the named workloads, in the launch
configuration bench.py times (cut points from the autotuner, and the
(2048, 32) cut the headline usually gets): every output entry is compared
with the fp64 oracle (its plain full-storage product of the unreordered
matrix runs in well under a second at these sizes), with the product
tolerance tau * (|alpha||x_i| + sum_j |s_ij||x_j|)."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from paper_2407_17651_gb300 import _build
from paper_2407_17651_gb300 import pars3 as P

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
TAU = {P.F64: 1e-12, P.F32: 2e-6, P.BF16: 2e-6}
ALL = P.dtype_bit(P.F64) | P.dtype_bit(P.F32) | P.dtype_bit(P.BF16)


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


def compare(A, perm, h, dtype, alpha, X, F=None):
    """X in the original numbering (n or n x k); every entry checked."""
    if dtype == P.BF16:
        F = O.Full(W.SkewMatrix(A.n, A.rowptr, A.col, bf16_round(A.val)))
        Xr = X.astype(np.float32).astype(np.float64)
    else:
        F = F or O.Full(A)
        Xr = X
    vt = torch.float64 if dtype == P.F64 else torch.float32
    Xd = torch.from_numpy(np.ascontiguousarray(X[perm])).to("cuda", vt)
    Yd = torch.full_like(Xd, float("nan"))
    if X.ndim == 1:
        P.pars3_spmv(h, dtype, alpha, Xd, Yd)
        ref, bound = F.apply(alpha, Xr), F.abs_bound(alpha, Xr)
    else:
        P.pars3_spmm(h, dtype, alpha, Xd, Yd)
        ref, bound = F.apply_block(alpha, Xr), F.abs_bound_block(alpha, Xr)
    torch.cuda.synchronize()
    P.pars3_check(h)
    y = np.empty_like(ref)
    y[perm] = Yd.double().cpu().numpy()
    bad = ~(np.abs(y - ref) <= TAU[dtype] * bound + (1e-300 if dtype == P.F64 else 1e-30))
    assert not bad.any(), f"{int(bad.sum())} entries off, first at {np.argwhere(bad)[:3].tolist()}"


@pytest.fixture(scope="module")
def cfg1():
    A, alpha, x = W.config1()
    perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
    return A, alpha, x, perm, O.Full(A)


@pytest.mark.parametrize("dtype", [P.F64, P.F32, P.BF16], ids=["f64", "f32", "bf16"])
def test_cfg1_headline_cut(cfg1, dtype):
    A, alpha, x, perm, F = cfg1
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, T=2048, W=32, dtypes=ALL)
    P.pars3_upload(h)
    compare(A, perm, h, dtype, alpha, x, F)


def test_cfg1_autotuned_cut_and_k32(cfg1):
    A, alpha, x, perm, F = cfg1
    for dtype, k in ((P.F64, 1), (P.F32, 32)):
        t = P.pars3_autotune(A.n, A.rowptr, A.col, A.val, perm, dtype=dtype, k=k, dtypes=ALL)
        h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, **P.split_kwargs(t))
        P.pars3_upload(h)
        X = x if k == 1 else W.vector("uniform", (A.n, k), 91)
        compare(A, perm, h, dtype, alpha, X, F)


def test_cfg2_autotuned(cfg1):
    A, alpha, x = W.config2()
    perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
    F = O.Full(A)
    for dtype in (P.F64, P.F32):
        t = P.pars3_autotune(A.n, A.rowptr, A.col, A.val, perm, dtype=dtype, k=1, dtypes=ALL)
        h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, **P.split_kwargs(t))
        P.pars3_upload(h)
        info = P.pars3_info_get(h)
        assert info["long_rows"] > 0   # the power-law rows are summed in pieces
        compare(A, perm, h, dtype, alpha, x, F)
        h.close()


@pytest.mark.parametrize("dtype,k", [(P.F32, 32), (P.F64, 4)], ids=["f32k32", "f64k4"])
def test_cfg4_batched_autotuned(dtype, k):
    shapes = W.config4_shapes()
    mats, perms, hs = [], [], []
    for m, shp in enumerate(shapes):
        A = W.config4_matrix(m, shp)
        perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
        t = P.pars3_autotune(A.n, A.rowptr, A.col, A.val, perm, dtype=P.F32, k=4,
                             dtypes=P.dtype_bit(P.F64) | P.dtype_bit(P.F32))
        h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, **P.split_kwargs(t))
        P.pars3_upload(h)
        mats.append(A)
        perms.append(perm)
        hs.append(h)
    vt = torch.float64 if dtype == P.F64 else torch.float32
    Xs = [W.config4_rhs(A.n, k, m) for m, A in enumerate(mats)]
    Xd = [torch.from_numpy(np.ascontiguousarray(X[p])).to("cuda", vt) for X, p in zip(Xs, perms)]
    Yd = [torch.full_like(X, float("nan")) for X in Xd]
    P.pars3_spmm_batched(hs, dtype, [1.0] * len(hs), Xd, Yd, capture=True)
    torch.cuda.synchronize()
    for A, p, X, Y in zip(mats, perms, Xs, Yd):
        F = O.Full(A)
        ref, bound = F.apply_block(1.0, X), F.abs_bound_block(1.0, X)   # fp64 oracle on the original X
        y = np.empty_like(ref)
        y[p] = Y.double().cpu().numpy()
        assert np.all(np.abs(y - ref) <= TAU[dtype] * bound + 1e-30)


@pytest.mark.parametrize("dtype,k", [(P.F32, 4), (P.F64, 4), (P.F32, 32)], ids=["f32k4", "f64k4", "f32k32"])
def test_cfg2_spmm_long_rows(dtype, k):
    """The multi-vector product on the R-MAT matrix: its power-law rows are
    summed in k-wide pieces (long_row = 32, pieces of 255, the autotuner's
    usual choice there); every entry of Y against the fp64 oracle on the
    original X."""
    A, alpha, x = W.config2()
    perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, T=2048, W=32, long_row=32, piece=255, long_slices=16,
                      dtypes=P.dtype_bit(dtype))
    P.pars3_upload(h)
    info = P.pars3_info_get(h)
    assert info["long_rows"] > 100000 and info["long_pieces"] > info["long_rows"]
    X = W.vector("uniform", (A.n, k), 77)
    compare(A, perm, h, dtype, 0.5, X, O.Full(A))
    h.close()
