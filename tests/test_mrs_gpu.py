"""GPU parity of pars3_mrs (Sec. 1: MRS for (alpha I + S) x = b) against the
FP64 oracle: the first k iterates match the oracle's MRS iterates; the final
true residual, recomputed by the oracle in fp64, meets the target for plain
fp64 MRS and for fp32 / bf16-value inner solves inside fp64 refinement; the
solution matches numpy.linalg.solve on small problems."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from paper_2407_17651_gb300 import _build
from paper_2407_17651_gb300 import pars3 as P

pytestmark = pytest.mark.gpu
ALL = P.dtype_bit(P.F64) | P.dtype_bit(P.F32) | P.dtype_bit(P.BF16)


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    O.build()
    torch.cuda.init()


def setup(A, **kw):
    perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, dtypes=ALL, **kw)
    P.pars3_upload(h)
    return h, perm


def solve(h, perm, alpha, b, inner=P.F64, **kw):
    bp = torch.from_numpy(np.ascontiguousarray(b[perm])).cuda()
    xp = torch.zeros_like(bp)
    res = P.pars3_mrs(h, alpha, bp, xp, inner=inner, **kw)
    torch.cuda.synchronize()
    x = np.empty_like(b)
    x[perm] = xp.cpu().numpy()
    return x, res


@pytest.mark.parametrize("alpha", [1.0, 0.2])
def test_iterates_match_oracle(alpha):
    A = W.random_skew(400, 0.02, 3, "normal")
    h, perm = setup(A, T=64, W=32)
    b = W.vector("uniform", A.n, 3)
    F = O.Full(A)
    for k in (1, 2, 3, 7, 20):
        x, res = solve(h, perm, alpha, b, rtol=1e-30, max_iter=k, raise_on_noconv=False)
        assert res["iters"] == k
        xo, info = O.mrs(lambda v: F.apply(0.0, v), A.n, alpha, b, rtol=0.0, maxit=k)
        assert np.linalg.norm(x - xo) <= 1e-11 * np.linalg.norm(xo), k


@pytest.mark.parametrize("inner", [P.F64, P.F32, P.BF16], ids=["f64", "f32-ir", "bf16-ir"])
@pytest.mark.parametrize("alpha", [1.0, 0.1])
def test_small_solve_reaches_target(inner, alpha):
    A = W.random_skew(300, 0.03, 7, "normal")
    h, perm = setup(A, T=64, W=32)
    b = W.vector("uniform", A.n, 7)
    x, res = solve(h, perm, alpha, b, inner=inner, rtol=1e-10, inner_rtol=1e-3)
    F = O.Full(A)
    rel = np.linalg.norm(b - F.apply(alpha, x)) / np.linalg.norm(b)
    assert rel <= 1e-10 * 1.05, rel
    assert abs(res["true_relres"] - rel) <= 1e-12 + 0.05 * rel
    exact = np.linalg.solve(alpha * np.eye(A.n) + O.dense(A), b)
    cond = np.linalg.cond(alpha * np.eye(A.n) + O.dense(A))
    assert np.linalg.norm(x - exact) <= 5 * cond * 1e-10 * np.linalg.norm(exact)
    if inner != P.F64:
        assert res["outer"] >= 1


def test_long_rows_and_halo_in_the_loop():
    """The Lanczos step uses the same fold as the product: long rows and halo
    rows must be finished (and their norms counted) inside the loop."""
    A = W.rmat(12, 30000, seed=31, value_kind="normal")
    h, perm = setup(A, T=256, W=128, long_row=40)
    info = P.pars3_info_get(h)
    assert info["long_rows"] > 0 and info["halo_targets"] > 0
    b = W.vector("uniform", A.n, 8)
    F = O.Full(A)
    for inner in (P.F64, P.F32):
        x, res = solve(h, perm, 1.0, b, inner=inner, rtol=1e-10, inner_rtol=1e-4)
        rel = np.linalg.norm(b - F.apply(1.0, x)) / np.linalg.norm(b)
        assert rel <= 1e-10 * 1.05, (inner, rel)


def test_heavy_long_rows_in_the_loop():
    """Rows of at least 64 pieces are folded by a warp in the MRS fold too (a
    hub joined to 3,600 grid vertices, pieces of 8 entries: 450 pieces)."""
    u, v = W.grid_edges((60, 60))
    n = 3601
    hub = n - 1
    u = np.concatenate([np.asarray(u, np.int64), np.full(3600, hub, np.int64)])
    v = np.concatenate([np.asarray(v, np.int64), np.arange(3600, dtype=np.int64)])
    A = W.from_keys(n, np.unique(np.maximum(u, v) * n + np.minimum(u, v)), "normal", 5)
    h, perm = setup(A, T=512, W=32, long_row=32, piece=8)
    assert P.pars3_info_get(h)["long_pieces"] >= 450
    b = W.vector("uniform", A.n, 9)
    F = O.Full(A)
    for inner in (P.F64, P.F32):
        x, res = solve(h, perm, 1.0, b, inner=inner, rtol=1e-10, inner_rtol=1e-4)
        rel = np.linalg.norm(b - F.apply(1.0, x)) / np.linalg.norm(b)
        assert rel <= 1e-10 * 1.05, (inner, rel)


def test_config3_alpha1_fp64_and_fp32():
    A, _, _ = W.config1()
    h, perm = setup(A, T=2048, W=32)
    b = W.config3_rhs(A.n)
    F = O.Full(A)
    for inner in (P.F64, P.F32):
        x, res = solve(h, perm, 1.0, b, inner=inner, rtol=1e-10, inner_rtol=1e-4)
        rel = np.linalg.norm(b - F.apply(1.0, x)) / np.linalg.norm(b)
        assert rel <= 1e-10 * 1.05, (inner, rel, res)


def test_errors_and_trivial_cases():
    A = W.random_skew(100, 0.05, 1)
    h, perm = setup(A, T=64, W=32)
    b = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    x = torch.ones_like(b)
    res = P.pars3_mrs(h, 1.0, b, x)
    assert res["iters"] == 0 and torch.count_nonzero(x).item() == 0
    with pytest.raises(P.Pars3Error) as e:
        P.pars3_mrs(h, 0.0, b, x)
    assert e.value.code == P.EINVAL
    h64 = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, dtypes=P.dtype_bit(P.F64))
    P.pars3_upload(h64)
    with pytest.raises(P.Pars3Error) as e:
        P.pars3_mrs(h64, 1.0, b, x, inner=P.F32)
    assert e.value.code == P.EUNSUPPORTED
