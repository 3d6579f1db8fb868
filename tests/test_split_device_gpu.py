"""The canonical split on the GPU (pars3_split_device) against the host split
and the oracle (Sec. 3.1.2, Eq. 2, Figs. 7-8): every exported array --
reordered CSR with the re-triangularization sign flip, classes, per-tile
middle lists in (col, row) order, outer lists in CSR and CSC order, counts,
cut points -- must be identical, element for element; the device layout,
built on the GPU, must equal the host-built one (same digest over every
layout array, same products bit for bit)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_2407_17651_gb300 import _build
from paper_2407_17651_gb300 import pars3 as P

pytestmark = pytest.mark.gpu

KEYS = ("perm", "rowptr", "col", "val", "cls", "tile_ptr", "tile_list", "outer_csr", "outer_csc", "counts")


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    _build.build()
    O.build()
    torch.cuda.init()


def _dev(A, perm=None):
    import torch
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()
    return (t(A.rowptr, np.int32), t(A.col, np.int32), t(A.val, np.float64),
            None if perm is None else t(perm, np.int32))


def _compare(A, perm, oracle=True, **kw):
    rp, ci, v, pm = _dev(A, perm)
    hd = P.pars3_split_device(A.n, rp, ci, v, pm, **kw)
    hh = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, **kw)
    ed, eh = P.pars3_split_export(hd), P.pars3_split_export(hh)
    for k in KEYS + ("T", "W", "ntiles", "nnz"):
        assert np.array_equal(np.asarray(ed[k]), np.asarray(eh[k])), (A.name, k, kw)
    assert P.pars3_info_get(hd) == P.pars3_info_get(hh), A.name
    assert P.pars3_layout_digest(hd) == P.pars3_layout_digest(hh), (A.name, kw)   # the layout built on the GPU
    assert P.pars3_layout_check(hd) == 0
    if oracle:
        so = O.split(A, perm if perm is not None else np.arange(A.n, dtype=np.int32), ed["T"], ed["W"],
                     **({"mirror": 1} if kw.get("symmetric") else {}))
        for k in ("rowptr", "col", "val", "cls", "tile_ptr", "tile_list", "outer_csr", "outer_csc", "counts"):
            assert np.array_equal(ed[k], so[k]), (A.name, k)
    return hd, hh


def _matrices():
    return [
        W.grid((37, 23), "normal", 1),
        W.grid((9, 8, 7), "normal", 2),
        W.grid_plus_random((30, 30), 0.05, "normal", 3),
        W.rmat(12, 30000, seed=4),
        W.banded_skew(3000, 40, 0.3, 5),
        W.random_skew(2000, 0.002, 6),
    ]


@pytest.mark.parametrize("cut", [(0, 0), (64, 32), (256, 64), (1024, 32)], ids=lambda c: f"T{c[0]}W{c[1]}")
def test_matches_host_and_oracle(cut):
    for A in _matrices():
        perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
        _compare(A, perm, T=cut[0], W=cut[1])


def test_identity_random_perm_and_symmetric():
    rng = np.random.default_rng(9)
    for A in _matrices()[:4]:
        _compare(A, None, T=128, W=32)
        _compare(A, rng.permutation(A.n).astype(np.int32), T=256, W=64)
        _compare(A, P.pars3_reorder(A.n, A.rowptr, A.col)[0], T=256, W=32, symmetric=True)


def test_layout_parameters_and_precisions():
    A = W.rmat(13, 60000, seed=10)   # long rows: pieces, folds
    perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
    both = P.dtype_bit(P.F64) | P.dtype_bit(P.F32) | P.dtype_bit(P.BF16)
    _compare(A, perm, oracle=False, T=512, W=32, dtypes=both, long_row=32, piece=37, long_slices=4)
    _compare(A, perm, oracle=False, T=1024, W=64, dtypes=both, lane_bytes=16, variant=P.VARIANT_LOOKAHEAD)


def test_products_identical():
    import torch
    A = W.grid_plus_random((64, 48), 0.02, "normal", 11)
    perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
    hd, hh = _compare(A, perm, T=256, W=64)
    x = torch.from_numpy(W.vector("uniform", A.n, 5)[perm]).cuda()
    ys = []
    for h in (hd, hh):
        P.pars3_upload(h)
        y = torch.empty_like(x)
        P.pars3_spmv(h, P.F64, 0.5, x, y)
        ys.append(y.cpu().numpy())
    assert np.array_equal(ys[0], ys[1])


def test_with_device_rcm_permutation():
    A = W.grid_plus_random((40, 40), 0.01, "normal", 12)
    rp, ci, v, _ = _dev(A)
    pd = P.pars3_reorder_device(A.n, rp, ci)[0]
    hd = P.pars3_split_device(A.n, rp, ci, v, pd, T=256, W=32)
    hh = P.pars3_split(A.n, A.rowptr, A.col, A.val, P.pars3_reorder(A.n, A.rowptr, A.col)[0], T=256, W=32)
    ed, eh = P.pars3_split_export(hd), P.pars3_split_export(hh)
    for k in KEYS:
        assert np.array_equal(ed[k], eh[k]), k


def test_edge_cases_and_errors():
    import torch
    mk = lambda a, dt=torch.int32: torch.tensor(a, dtype=dt, device="cuda")
    # empty matrix, one vertex, no entries
    for n in (0, 1, 5):
        A = W.SkewMatrix(n, np.zeros(n + 1, np.int32), np.zeros(0, np.int32), np.zeros(0))
        _compare(A, None, oracle=False)
    rp, v = mk([0, 0, 1, 3]), mk([1.0, 2.0, 3.0], torch.float64)
    for bad_col in ([0, 1, 1], [0, 1, 0], [0, 0, 2], [1, 0, 1]):   # duplicate, unsorted, diagonal, upper
        with pytest.raises(P.Pars3Error) as ei:
            P.pars3_split_device(3, rp, mk(bad_col), v)
        assert ei.value.code == P.ENOTSKEW, bad_col
    ci = mk([0, 0, 1])   # rows {0}, {0, 1}
    v[1] = float("nan")
    with pytest.raises(P.Pars3Error) as ei:
        P.pars3_split_device(3, rp, ci, v)
    assert ei.value.code == P.ENONFINITE
    v[1] = 2.0
    for bad_perm in ([0, 0, 2], [0, 1, 3], [-1, 1, 2]):
        with pytest.raises(P.Pars3Error) as ei:
            P.pars3_split_device(3, rp, ci, v, mk(bad_perm))
        assert ei.value.code == P.EINVAL, bad_perm
    for kw in (dict(T=64, W=0), dict(T=48, W=32), dict(T=32, W=64), dict(dtypes=8), dict(piece=3)):
        with pytest.raises(P.Pars3Error) as ei:
            P.pars3_split_device(3, rp, ci, v, **kw)
        assert ei.value.code == P.EINVAL, kw
    h = P.pars3_split_device(3, rp, ci, v, mk([2, 0, 1]))   # still usable
    assert P.pars3_layout_check(h) == 0


@pytest.mark.slow
@pytest.mark.parametrize("name,cut", [("cfg1", (2048, 32)), ("cfg2", (2048, 32)), ("cfg2", (1024, 32))])
def test_full_size_bit_exact(name, cut):
    A = W.config1()[0] if name == "cfg1" else W.config2()[0]
    perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
    _compare(A, perm, T=cut[0], W=cut[1])


@pytest.mark.slow
def test_all_batched_matrices_bit_exact():
    for m, shp in enumerate(W.config4_shapes()):
        A = W.config4_matrix(m, shp)
        perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
        _compare(A, perm, T=512, W=32)
