"""GPU parity of pars3_spmm_batched: many uneven products in one persistent
launch.  Each batched result must equal the single-matrix call on the same
handle bit for bit (the work units and the fold run the same device code in
the same order) and match the FP64 oracle within the product tolerance;
graph replay must follow new contents of the same buffers."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from paper_2407_17651_gb300 import _build
from paper_2407_17651_gb300 import pars3 as P

pytestmark = pytest.mark.gpu
ALL = P.dtype_bit(P.F64) | P.dtype_bit(P.F32) | P.dtype_bit(P.BF16)
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


def batch_members():
    """Uneven grids like the batched workload (2D and 3D), one R-MAT member
    with long rows and halo targets, one matrix smaller than a tile; each with
    its own tile geometry so that the shared-memory plans differ."""
    mats = [
        (W.grid((61, 47), "normal", 11), {"T": 256, "W": 64}),
        (W.grid((13, 12, 14), "normal", 12), {"T": 512, "W": 256}),
        (W.rmat(11, 14000, seed=13, value_kind="normal"), {"T": 256, "W": 128, "long_row": 40}),
        (W.grid((9, 7), "uniform", 14), {"T": 1024, "W": 32}),
        (W.grid((40, 40, 6), "normal", 15), {"T": 1024, "W": 1024}),
    ]
    out = []
    for A, kw in mats:
        perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
        h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, dtypes=ALL, **kw)
        P.pars3_upload(h)
        out.append((A, perm, h))
    return out


@pytest.fixture(scope="module")
def members():
    return batch_members()


def operands(members, dtype, k, seed):
    vt = torch.float64 if dtype == P.F64 else torch.float32
    Xs, Ys, Xn = [], [], []
    for m, (A, perm, h) in enumerate(members):
        shape = (A.n,) if k == 1 else (A.n, k)
        X = W.vector("uniform", shape, seed + m)
        Xn.append(X)
        Xs.append(torch.from_numpy(np.ascontiguousarray(X[perm])).to("cuda", vt))
        Ys.append(torch.full_like(Xs[-1], float("nan")))
    return Xs, Ys, Xn


def oracle_check(A, perm, dtype, alpha, X, y):
    if dtype == P.BF16:
        F = O.Full(W.SkewMatrix(A.n, A.rowptr, A.col, bf16_round(A.val)))
        Xr = X.astype(np.float32).astype(np.float64)
    else:
        F = O.Full(A)
        Xr = X
    X2 = Xr.reshape(A.n, -1)
    ref = F.apply_block(alpha, X2)[perm]
    bound = F.abs_bound_block(alpha, X2)[perm]
    err = np.abs(y.reshape(A.n, -1) - ref)
    lim = TAU[dtype] * bound + (1e-300 if dtype == P.F64 else 1e-30)
    assert np.all(err <= lim), int(np.sum(~(err <= lim)))


@pytest.mark.parametrize("dtype", [P.F64, P.F32, P.BF16], ids=["f64", "f32", "bf16"])
@pytest.mark.parametrize("k", [1, 4, 16, 32])
@pytest.mark.parametrize("capture", [False, True], ids=["launch", "graph"])
def test_batched_equals_single_and_oracle(members, dtype, k, capture):
    alphas = [0.5, -1.0, 0.25, 2.0, 0.0][: len(members)]
    Xs, Ys, Xn = operands(members, dtype, k, 100 + k)
    P.pars3_spmm_batched([h for _, _, h in members], dtype, alphas, Xs, Ys, capture=capture)
    torch.cuda.synchronize()
    for m, (A, perm, h) in enumerate(members):
        P.pars3_check(h)
        Y1 = torch.full_like(Xs[m], float("nan"))
        P.pars3_spmm(h, dtype, alphas[m], Xs[m], Y1)
        torch.cuda.synchronize()
        assert torch.equal(Ys[m], Y1), f"member {m} differs from the single call"
        oracle_check(A, perm, dtype, alphas[m], Xn[m], Ys[m].double().cpu().numpy())


def test_batched_with_heavy_long_rows_equals_single():
    """A member with rows of at least 64 pieces (folded by warps): the batched
    result equals the single-matrix call bit for bit and the oracle."""
    u, v = W.grid_edges((60, 60))
    n = 3601
    hub = n - 1
    u = np.concatenate([np.asarray(u, np.int64), np.full(3600, hub, np.int64)])
    v = np.concatenate([np.asarray(v, np.int64), np.arange(3600, dtype=np.int64)])
    A = W.from_keys(n, np.unique(np.maximum(u, v) * n + np.minimum(u, v)), "normal", 6)
    B = W.grid((50, 40), "normal", 7)
    mem = []
    for M, kw in ((A, dict(T=512, W=32, long_row=32, piece=8)), (B, dict(T=256, W=64))):
        perm = P.pars3_reorder(M.n, M.rowptr, M.col)[0]
        h = P.pars3_split(M.n, M.rowptr, M.col, M.val, perm, dtypes=ALL, **kw)
        P.pars3_upload(h)
        mem.append((M, perm, h))
    for dtype in (P.F64, P.F32):
        for k in (1, 4):
            Xs, Ys, Xn = operands(mem, dtype, k, 300 + k)
            P.pars3_spmm_batched([h for _, _, h in mem], dtype, [0.5, 1.0], Xs, Ys, capture=False)
            torch.cuda.synchronize()
            for m, (M, perm, h) in enumerate(mem):
                Y1 = torch.full_like(Xs[m], float("nan"))
                P.pars3_spmm(h, dtype, [0.5, 1.0][m], Xs[m], Y1)
                torch.cuda.synchronize()
                assert torch.equal(Ys[m], Y1), (dtype, k, m)
                oracle_check(M, perm, dtype, [0.5, 1.0][m], Xn[m], Ys[m].double().cpu().numpy())


def test_graph_replay_follows_buffer_contents(members):
    hs = [h for _, _, h in members]
    alphas = [1.0] * len(members)
    Xs, Ys, _ = operands(members, P.F64, 4, 7)
    P.pars3_spmm_batched(hs, P.F64, alphas, Xs, Ys, capture=True)
    torch.cuda.synchronize()
    first = [Y.clone() for Y in Ys]
    for X in Xs:
        X.mul_(-2.0)
    P.pars3_spmm_batched(hs, P.F64, alphas, Xs, Ys, capture=True)   # replay
    torch.cuda.synchronize()
    for Y, Y0 in zip(Ys, first):
        assert torch.equal(Y, -2.0 * Y0)   # exact: scaling by a power of two
    # new alphas rebuild the argument table
    P.pars3_spmm_batched(hs, P.F64, [0.0] * len(hs), Xs, Ys, capture=True)
    torch.cuda.synchronize()
    for (A, perm, h), X, Y in zip(members, Xs, Ys):
        Y1 = torch.empty_like(Y)
        P.pars3_spmm(h, P.F64, 0.0, X, Y1)
        torch.cuda.synchronize()
        assert torch.equal(Y, Y1)


def test_batched_deterministic_and_single_member(members):
    A, perm, h = members[2]
    Xs, Ys, Xn = operands([members[2]], P.F32, 8, 3)
    P.pars3_spmm_batched([h], P.F32, [0.7], Xs, Ys)
    Y0 = Ys[0].clone()
    for _ in range(3):
        P.pars3_spmm_batched([h], P.F32, [0.7], Xs, Ys)
        torch.cuda.synchronize()
        assert torch.equal(Ys[0], Y0)
    oracle_check(A, perm, P.F32, 0.7, Xn[0], Y0.double().cpu().numpy())


def test_batched_with_an_empty_member(members):
    E = W.SkewMatrix(0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    he = P.pars3_split(0, E.rowptr, E.col, E.val, dtypes=ALL)
    P.pars3_upload(he)
    A, perm, h = members[0]
    x = torch.from_numpy(W.vector("uniform", A.n, 9)).cuda()
    y = torch.empty_like(x)
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    P.pars3_spmm_batched([he, h], P.F64, [1.0, 0.3], [e, x], [e.clone(), y])
    y1 = torch.empty_like(x)
    P.pars3_spmv(h, P.F64, 0.3, x, y1)
    torch.cuda.synchronize()
    assert torch.equal(y, y1)


def test_batched_errors(members):
    hs = [h for _, _, h in members]
    Xs, Ys, _ = operands(members, P.F64, 4, 1)
    assert P.lib().pars3_spmm_batched(None, 0, P.F64, None, 4, None, None, 0, None) == P.EINVAL
    X33 = torch.zeros((members[0][0].n, 33), dtype=torch.float64, device="cuda")
    with pytest.raises(P.Pars3Error) as e:   # k = 33 columns
        P.pars3_spmm_batched(hs[:1], P.F64, [1.0], [X33], [torch.zeros_like(X33)])
    assert e.value.code == P.EINVAL
    with pytest.raises(ValueError):   # Y of another shape: caught by the binding
        P.pars3_spmm_batched(hs[:1], P.F64, [1.0], [X33], [Ys[0]])
    with pytest.raises(P.Pars3Error) as e:   # in place
        P.pars3_spmm_batched(hs[:1], P.F64, [1.0], Xs[:1], Xs[:1])
    assert e.value.code == P.EINVAL
    A = members[0][0]
    h64 = P.pars3_split(A.n, A.rowptr, A.col, A.val, members[0][1], dtypes=P.dtype_bit(P.F64))
    P.pars3_upload(h64)
    with pytest.raises(P.Pars3Error) as e:
        P.pars3_spmm_batched([h64], P.F32, [1.0], [Xs[0].float()], [Ys[0].float()])
    assert e.value.code == P.EUNSUPPORTED
    h_new = P.pars3_split(A.n, A.rowptr, A.col, A.val, members[0][1], dtypes=ALL)
    with pytest.raises(P.Pars3Error) as e:
        P.pars3_spmm_batched([h_new], P.F64, [1.0], [Xs[0]], [Ys[0]])
    assert e.value.code == P.ESTATE
