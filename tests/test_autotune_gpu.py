"""pars3_autotune on the GPU: the chosen cut points are valid powers of two,
the split at those cut points is bit-exact against the oracle and its
product matches the oracle; the search leaves no device memory behind."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from paper_2407_17651_gb300 import _build
from paper_2407_17651_gb300 import pars3 as P

pytestmark = pytest.mark.gpu
KEYS = ("rowptr", "col", "val", "cls", "tile_ptr", "tile_list", "outer_csr", "outer_csc", "counts")


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    O.build()
    torch.cuda.init()


def pow2(v):
    return v > 0 and (v & (v - 1)) == 0


def assert_valid_layout_params(r):
    assert r["long_row"] in (0, 32, 64, 128) and r["piece"] in (0, 128, 192, 255), r
    assert r["long_slices"] in (0, 16, 32) and r["lane_bytes"] in (0, 4, 8, 16, 32), r
    assert r["variant"] in (0, P.VARIANT_LOOKAHEAD), r


@pytest.mark.parametrize("dtype,k", [(P.F64, 1), (P.F32, 1), (P.F32, 8), (P.F64, 4)],
                         ids=["f64k1", "f32k1", "f32k8", "f64k4"])
def test_power_law_choice_valid_bit_exact_and_correct(dtype, k):
    """On an R-MAT graph the search also covers the long-row settings and the
    kernel variant or lane width; the split at the returned parameters is
    bit-exact against the oracle and its product (and multi-vector product)
    matches the oracle."""
    A = W.rmat(14, 120000, seed=33)
    perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
    r = P.pars3_autotune(A.n, A.rowptr, A.col, A.val, perm, dtype=dtype, k=k)
    assert_valid_layout_params(r)
    kw = P.split_kwargs(r)
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, **kw)
    ex = P.pars3_split_export(h)
    so = O.split(A, perm, r["T"], r["W"])
    for key in KEYS:
        assert np.array_equal(ex[key], so[key]), key
    assert P.pars3_layout_check(h) == 0
    P.pars3_upload(h)
    F = O.Full(A)
    vt = torch.float64 if dtype == P.F64 else torch.float32
    tau = 1e-12 if dtype == P.F64 else 2e-6
    X = W.vector("uniform", (A.n, k), 7)
    Xd = torch.from_numpy(np.ascontiguousarray(X[perm] if k > 1 else X[perm, 0])).to("cuda", vt)
    Yd = torch.full_like(Xd, float("nan"))
    if k == 1:
        P.pars3_spmv(h, dtype, 0.5, Xd, Yd)
    else:
        P.pars3_spmm(h, dtype, 0.5, Xd, Yd)
    torch.cuda.synchronize()
    Y = Yd.double().cpu().numpy().reshape(A.n, k)
    for c in range(k):
        ref = F.apply(0.5, X[:, c])[perm]
        bound = F.abs_bound(0.5, X[:, c])[perm]
        assert np.all(np.abs(Y[:, c] - ref) <= tau * bound + 1e-30), c


@pytest.mark.parametrize("dtype,k", [(P.F64, 1), (P.F32, 4), (P.BF16, 16)], ids=["f64k1", "f32k4", "bf16k16"])
def test_choice_valid_bit_exact_and_correct(dtype, k):
    A = W.grid_plus_random((24, 24, 24), 0.01, "normal", 5)
    perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
    r = P.pars3_autotune(A.n, A.rowptr, A.col, A.val, perm, dtype=dtype, k=k)
    T, Wc = r["T"], r["W"]
    assert pow2(T) and pow2(Wc) and 32 <= Wc <= T <= 8192, r
    assert r["us"] > 0 and r["dtypes"] & P.dtype_bit(dtype)
    assert_valid_layout_params(r)
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, **P.split_kwargs(r))
    ex = P.pars3_split_export(h)
    so = O.split(A, perm, T, Wc)
    for key in KEYS:
        assert np.array_equal(ex[key], so[key]), key
    P.pars3_upload(h)
    x = W.vector("uniform", A.n, 6)
    F = O.Full(A)
    xp = torch.from_numpy(x[perm]).cuda()
    y = torch.empty_like(xp)
    P.pars3_spmv(h, P.F64, 0.25, xp, y)
    torch.cuda.synchronize()
    ref = F.apply(0.25, x)[perm]
    assert np.all(np.abs(y.cpu().numpy() - ref) <= 1e-12 * F.abs_bound(0.25, x)[perm] + 1e-300)


def test_band_limited_search_and_no_device_memory_left():
    A = W.banded_skew(30000, 48, 0.4, 8)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    r = P.pars3_autotune(A.n, A.rowptr, A.col, A.val, None, dtype=P.F64, k=1)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert abs(free0 - free1) <= 64 << 20
    # the band is 48 wide: no candidate W above 64 is tried
    assert r["W"] <= 64 and pow2(r["T"])


def test_trivial_and_invalid():
    E = np.zeros(1, np.int32)
    r = P.pars3_autotune(0, E, np.zeros(0, np.int32), np.zeros(0), None)
    assert (r["T"], r["W"]) == (1024, 32)
    A = W.random_skew(200, 0.05, 2)
    for k in (0, 33):
        with pytest.raises(P.Pars3Error) as e:
            P.pars3_autotune(A.n, A.rowptr, A.col, A.val, None, k=k)
        assert e.value.code == P.EINVAL
    bad = A.col.copy()
    if bad.size:
        bad[0] = A.n + 5
        with pytest.raises(P.Pars3Error):
            P.pars3_autotune(A.n, A.rowptr, bad, A.val, None)
