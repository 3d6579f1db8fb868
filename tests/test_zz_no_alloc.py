"""pars3_spmv_noalloc: the product for callers that cannot have the library
allocate device memory for scratch (all device memory already handed to
another allocator or pool, or a fixed memory budget); its scratch is a fixed
library-wide device array.  Checked through the C ABI against the fp64
oracle on the original values, and against pars3_spmv, on two calls in a row
(the second with another x, so that stale scratch contents from the first
call would show), with the fp64/fp32 tolerance of the parity tests.  This
file is collected last on purpose."""
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


def _handle(A, **kw):
    perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, dtypes=P.dtype_bit(P.F64) | P.dtype_bit(P.F32), **kw)
    P.pars3_upload(h)
    return h, perm


def grid_with_hub(a: int, every: int, seed: int):
    """a x a 5-point grid plus a hub vertex joined to every `every`-th grid
    vertex: a banded part with cross-tile middle entries (halo sums) and one
    long row (piece sums), the two kinds of scratch."""
    u, v = W.grid_edges((a, a))
    n = a * a + 1
    hub = n - 1
    spokes = np.arange(0, a * a, every, dtype=np.int64)
    u = np.concatenate([np.asarray(u, np.int64), np.full(spokes.size, hub, np.int64)])
    v = np.concatenate([np.asarray(v, np.int64), spokes])
    keys = np.unique(np.maximum(u, v) * n + np.minimum(u, v))
    return W.from_keys(n, keys, "normal", seed, name=f"grid{a}_hub")


@pytest.mark.parametrize("name,gen,kw", [
    ("grid_hub_long_rows_and_halo", lambda: grid_with_hub(100, 7, 10), {"T": 256, "W": 128, "long_row": 64}),
    ("band_halo", lambda: W.banded_skew(20000, 100, 0.3, 3), {"T": 256, "W": 128}),
])
def test_noalloc_matches_oracle_on_two_calls(name, gen, kw):
    A = gen()
    h, perm = _handle(A, **kw)
    info = P.pars3_info_get(h)
    assert info["halo_targets"] > 0
    if name.startswith("grid_hub"):
        assert info["long_rows"] > 0 and info["long_pieces"] > 1
    F = O.Full(A)
    for dtype in (P.F64, P.F32):
        vt = torch.float64 if dtype == P.F64 else torch.float32
        for call, seed in enumerate((11, 12)):
            x = W.vector("uniform", A.n, seed)
            xp = torch.from_numpy(x[perm]).to("cuda", vt)
            y_lib = torch.full_like(xp, float("nan"))
            y_new = torch.full_like(xp, float("nan"))
            P.pars3_spmv_noalloc(h, dtype, 0.75, xp, y_new)
            P.pars3_spmv(h, dtype, 0.75, xp, y_lib)
            torch.cuda.synchronize()
            P.pars3_check(h)
            a = y_new.double().cpu().numpy()
            ref = F.apply(0.75, x)[perm]          # fp64 oracle on the original values
            bound = F.abs_bound(0.75, x)[perm]
            assert np.all(np.abs(a - ref) <= TAU[dtype] * bound + 1e-30), (name, dtype, call)
            b = y_lib.double().cpu().numpy()
            assert np.all(np.abs(a - b) <= TAU[dtype] * bound + 1e-30), (name, dtype, call)


def test_noalloc_rejects_scratch_beyond_its_array():
    """Over 524,288 halo targets need more than the 4 MiB array in fp64."""
    A = W.banded_skew(1_200_000, 32, 0.25, 5)
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, None, T=32, W=32)
    P.pars3_upload(h)
    assert P.pars3_info_get(h)["halo_targets"] > (4 << 20) // 8
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    y = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(P.Pars3Error) as e:
        P.pars3_spmv_noalloc(h, P.F64, 1.0, x, y)
    assert e.value.code == P.EUNSUPPORTED
