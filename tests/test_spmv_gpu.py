"""GPU parity of the skew SpMV (C ABI) against the FP64 oracle.

Tolerance (per entry, over the full row of S): |y - y_ref| <= tau * b_i with
b_i = |alpha||x_i| + sum_j |s_ij||x_j|, tau = 1e-12 for fp64 and 2e-6 for
fp32 values and vectors (y_ref on the original fp64 values).  bf16 values
are compared with the oracle applied to the bf16-rounded values (fp32
accumulation, tau = 2e-6).  The device works in the RCM numbering: x' =
x[perm], y' = y[perm].
"""
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
    """Round fp64 -> fp32 -> bf16 (round to nearest, ties to even) -> fp64."""
    f = np.asarray(v, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def make(A, perm=None, T=0, Wc=0, dtypes=7, long_row=0):
    if perm is None:
        perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, T=T, W=Wc, dtypes=dtypes, long_row=long_row)
    P.pars3_upload(h)
    return h, perm


def run(h, dtype, alpha, xp_np):
    vt = torch.float64 if dtype == P.F64 else torch.float32
    xp = torch.from_numpy(np.ascontiguousarray(xp_np)).to("cuda", vt)
    y = torch.full_like(xp, float("nan"))
    P.pars3_spmv(h, dtype, alpha, xp, y)
    torch.cuda.synchronize()
    P.pars3_check(h)
    return y.double().cpu().numpy()


def check(A, h, perm, dtype, alpha, x):
    if dtype == P.BF16:
        Ar = W.SkewMatrix(A.n, A.rowptr, A.col, bf16_round(A.val))
        xr = x.astype(np.float32).astype(np.float64)
        F = O.Full(Ar)
        ref = F.apply(alpha, xr)
        bound = F.abs_bound(alpha, xr)
    else:
        F = O.Full(A)
        ref = F.apply(alpha, x)
        bound = F.abs_bound(alpha, x)
    y = run(h, dtype, alpha, x[perm])
    err = np.abs(y - ref[perm])
    lim = TAU[dtype] * bound[perm] + (1e-300 if dtype == P.F64 else 1e-30)
    bad = np.nonzero(~(err <= lim))[0]
    assert bad.size == 0, f"{bad.size} rows off, worst {err[bad].max() if bad.size else 0:.3e} at {bad[:5]}"
    return y


CASES = [
    ("rand1", lambda: W.random_skew(1, 0.5, 1), {}),
    ("rand2", lambda: W.random_skew(2, 1.0, 2), {}),
    ("rand37", lambda: W.random_skew(37, 0.2, 3), {"T": 32, "Wc": 32}),
    ("rand600", lambda: W.random_skew(600, 0.01, 4), {"T": 64, "Wc": 32}),
    ("band3000", lambda: W.banded_skew(3000, 40, 0.3, 5), {"T": 256, "Wc": 64}),
    ("band_ragged", lambda: W.banded_skew(5003, 100, 0.2, 6), {"T": 1024, "Wc": 128}),
    ("grid2d", lambda: W.grid((90, 70), "uniform", 7), {}),
    ("grid3d", lambda: W.grid((22, 21, 20), "normal", 8), {"T": 1024, "Wc": 512}),
    ("grid3d_small_window", lambda: W.grid((22, 21, 20), "normal", 8), {"T": 256, "Wc": 64}),
    ("grid+rand", lambda: W.grid_plus_random((20, 20, 20), 0.01, "normal", 9), {"T": 512, "Wc": 256}),
    ("rmat_long", lambda: W.rmat(13, 60000, seed=10), {"T": 256, "Wc": 256, "long_row": 64}),
    ("overfull", lambda: W.banded_skew(4096, 1024, 0.05, 11), {"T": 1024, "Wc": 1024}),
    ("config0", lambda: W.config0()[0], {}),
    ("fem_half", lambda: W.fem_grid2d(24, 30, 3, "normal", 12), {"T": 256, "Wc": 128}),
    ("fem_full", lambda: W.fem_grid2d(24, 30, 3, "normal", 12), {"T": 512, "Wc": 32}),
]


@pytest.mark.parametrize("name,gen,kw", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("dtype", [P.F64, P.F32, P.BF16], ids=["f64", "f32", "bf16"])
def test_spmv_parity(name, gen, kw, dtype):
    A = gen()
    h, perm = make(A, **kw)
    x = W.vector("uniform", A.n, 77)
    for alpha in (0.0, 0.5, -1.25):
        check(A, h, perm, dtype, alpha, x)


def test_bitwise_determinism():
    A = W.rmat(13, 60000, seed=10)
    h, perm = make(A, T=256, Wc=256, long_row=64)
    x = W.vector("normal", A.n, 5)[perm]
    for dtype in (P.F64, P.F32):
        ys = [run(h, dtype, 0.3, x) for _ in range(3)]
        assert all(np.array_equal(ys[0].view(np.uint64), y.view(np.uint64)) for y in ys[1:])


def test_unit_vector_probing_exact():
    """y' = S' e_j reproduces column j of the reordered S bit-exactly."""
    A = W.grid_plus_random((9, 8, 7), 0.02, "normal", 12)
    h, perm = make(A, T=64, Wc=32)
    Sp = O.dense(A)[np.ix_(perm, perm)]
    for j in list(range(0, A.n, 37)) + [A.n - 1]:
        e = np.zeros(A.n)
        e[j] = 1.0
        y = run(h, P.F64, 0.0, e)
        assert np.array_equal(y, Sp[:, j])


def test_empty_pattern_is_shift():
    A = W.random_skew(1000, 0.0, 1)
    assert A.nnz == 0
    h, perm = make(A)
    x = W.vector("uniform", A.n, 3)
    y = run(h, P.F64, 1.5, x[perm])
    assert np.array_equal(y, 1.5 * x[perm])


def test_empty_matrix():
    A = W.random_skew(0, 0.0, 1)
    h = P.pars3_split(0, A.rowptr, A.col, A.val)
    P.pars3_upload(h)
    x = torch.zeros(0, dtype=torch.float64, device="cuda")
    y = torch.zeros(0, dtype=torch.float64, device="cuda")
    P.pars3_spmv(h, P.F64, 1.0, x, y)
    torch.cuda.synchronize()


def test_permute_roundtrip_and_host_entry():
    A, _, x = W.config0()
    h, perm = make(A)
    xt = torch.from_numpy(x).cuda()
    xp = torch.empty_like(xt)
    P.pars3_permute(h, P.F64, xt, xp)
    assert np.array_equal(xp.cpu().numpy(), x[perm])
    back = torch.empty_like(xt)
    P.pars3_unpermute(h, P.F64, xp, back)
    assert np.array_equal(back.cpu().numpy(), x)
    y = np.empty_like(x)
    P.pars3_spmv_host(h, P.F64, 0.7, x, y)
    F = O.Full(A)
    assert np.all(np.abs(y - F.apply(0.7, x)) <= 1e-12 * F.abs_bound(0.7, x) + 1e-300)


def test_rejects_misaligned_vectors():
    A, _, x = W.config0()
    h, perm = make(A)
    buf = torch.zeros(A.n + 1, dtype=torch.float64, device="cuda")
    y = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(P.Pars3Error) as e:
        P.pars3_spmv(h, P.F64, 1.0, buf[1:], y)
    assert e.value.code == P.EINVAL


def test_fp64_fma_rate_probe():
    """The fp64 FMA rate helper returns a plausible rate for a GB300-class
    part (between 0.05 and 10 T FMA/s) and the same order twice."""
    r1 = P.pars3_fp64_fma_rate()
    r2 = P.pars3_fp64_fma_rate()
    assert 5e10 < r1 < 1e13 and 5e10 < r2 < 1e13
    assert 0.5 < r1 / r2 < 2.0


def test_product_with_local_rcm_order():
    """A grid with shortcuts ordered by PARS3_RCM_LOCAL: the product in that
    numbering matches the oracle (fp64 and fp32)."""
    A = W.grid_plus_random((40, 30, 8), 0.01, "normal", 41)
    perm = P.pars3_reorder(A.n, A.rowptr, A.col, P.RCM_GUARD | P.RCM_LOCAL)[0]
    F = O.Full(A)
    x = W.vector("uniform", A.n, 42)
    for dtype, tau in ((P.F64, 1e-12), (P.F32, 2e-6)):
        h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, T=1024, W=64, dtypes=P.dtype_bit(dtype))
        P.pars3_upload(h)
        vt = torch.float64 if dtype == P.F64 else torch.float32
        xp = torch.from_numpy(x[perm]).to("cuda", vt)
        y = torch.full_like(xp, float("nan"))
        P.pars3_spmv(h, dtype, 0.5, xp, y)
        torch.cuda.synchronize()
        ref = F.apply(0.5, x)[perm]
        assert np.all(np.abs(y.double().cpu().numpy() - ref) <= tau * F.abs_bound(0.5, x)[perm] + 1e-30)
        h.close()
