"""Host-side checks of libpars3 (no GPU): the C ABI loads and exports every
entry point declared in include/pars3.h; RCM and the canonical split match
the oracle bit-exactly; the device layout reconstructs the split; invalid
input is rejected with the documented status codes."""
import os
import re

import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import ROOT
from paper_2407_17651_gb300 import _build
from paper_2407_17651_gb300 import pars3 as P


@pytest.fixture(scope="session", autouse=True)
def built():
    _build.build()
    O.build()


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "pars3.h")).read()
    declared = set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pars3_\w+)\s*\(", hdr, flags=re.M))
    assert "pars3_spmv" in declared and "pars3_reorder" in declared
    L = P.lib()
    for name in sorted(declared):
        assert hasattr(L, name), f"{name} declared in pars3.h but not exported"
    assert set(P.exported_symbols()) <= declared
    assert P.pars3_version()[2] == 103


def _mats():
    yield W.random_skew(1, 0.5, 1)
    yield W.random_skew(2, 1.0, 2)
    yield W.random_skew(37, 0.2, 3)
    yield W.random_skew(600, 0.01, 4)
    yield W.banded_skew(3000, 40, 0.3, 5)
    yield W.grid((30, 20), "uniform", 6)
    yield W.grid((12, 11, 10), "normal", 7)
    yield W.grid_plus_random((16, 16, 16), 0.01, "normal", 8)
    yield W.rmat(12, 20000, seed=9)


@pytest.mark.parametrize("idx", range(9))
def test_rcm_bit_exact(idx):
    A = list(_mats())[idx]
    for guard in (1, 0):
        perm, b0, b1 = P.pars3_reorder(A.n, A.rowptr, A.col, guard)
        po, ob0, ob1 = O.rcm(A, guard=bool(guard))
        assert np.array_equal(perm, po)
        assert (b0, b1) == (ob0, ob1)


@pytest.mark.parametrize("idx", range(9))
def test_local_rcm_bit_exact(idx):
    """PARS3_RCM_LOCAL (with and without the guard and pseudo-peripheral
    starts) against the oracle's local-edge RCM."""
    A = list(_mats())[idx]
    for flags in (P.RCM_LOCAL, P.RCM_LOCAL | P.RCM_GUARD, P.RCM_LOCAL | P.RCM_PERIPHERAL,
                  P.RCM_LOCAL | P.RCM_GUARD | P.RCM_PERIPHERAL):
        perm, b0, b1 = P.pars3_reorder(A.n, A.rowptr, A.col, flags)
        po, ob0, ob1 = O.rcm(A, guard=bool(flags & P.RCM_GUARD), peripheral=bool(flags & P.RCM_PERIPHERAL),
                             local=True)
        assert np.array_equal(perm, po), flags
        assert (b0, b1) == (ob0, ob1)


def test_unknown_reorder_flag_rejected():
    A = W.grid((10, 10), "uniform", 1)
    with pytest.raises(P.Pars3Error) as e:
        P.pars3_reorder(A.n, A.rowptr, A.col, 8)
    assert e.value.code == P.EINVAL


def test_rcm_bit_exact_config0_and_hand_example():
    A, _, _ = W.config0()
    perm, b0, b1 = P.pars3_reorder(A.n, A.rowptr, A.col)
    po, ob0, ob1 = O.rcm(A)
    assert np.array_equal(perm, po) and b1 == ob1 == 101
    import json
    from conftest import GOLDEN
    g = json.load(open(os.path.join(GOLDEN, "rcm_hand_9.json")))
    n = g["n"]
    keys = np.array(sorted(max(a, b) * n + min(a, b) for a, b in g["edges"]), dtype=np.int64)
    H = W.from_keys(n, keys, "uniform", 0)
    perm, b0, b1 = P.pars3_reorder(n, H.rowptr, H.col)
    assert perm.tolist() == g["expected_perm_new_to_old"] and (b0, b1) == (5, 3)


KEYS = ("rowptr", "col", "val", "cls", "tile_ptr", "tile_list", "outer_csr", "outer_csc", "counts")


@pytest.mark.parametrize("idx", range(9))
@pytest.mark.parametrize("TW", [(32, 32), (64, 32), (1024, 256)])
def test_split_bit_exact(idx, TW):
    A = list(_mats())[idx]
    T, Wc = TW
    perm = O.rcm(A)[0] if idx % 2 else np.random.default_rng(idx).permutation(A.n).astype(np.int32)
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, T=T, W=Wc, dtypes=7)
    ex = P.pars3_split_export(h)
    so = O.split(A, perm, T, Wc)
    for k in KEYS:
        assert np.array_equal(ex[k], so[k]), k
    assert P.pars3_layout_check(h) == 0


def test_split_bit_exact_hand_fixture():
    import json
    from conftest import GOLDEN
    g = json.load(open(os.path.join(GOLDEN, "split_hand_6.json")))
    n = g["n"]
    trip = sorted(tuple(t) for t in g["stored"])
    keys = np.array([r * n + c for r, c, _ in trip], dtype=np.int64)
    A = W.from_keys(n, keys, "uniform", 0)
    A.val = np.array([v for _, _, v in trip])
    for c in g["cases"]:
        # the library needs W >= 32: scale the example by tiling it into a
        # larger index space would change it, so compare through the oracle
        so = O.split(A, np.array(c["perm"]), g["T"], g["W"])
        for k in KEYS:
            assert so[k].tolist() == c[k]


def test_default_cut_rule_matches_oracle():
    A, _, _ = W.config0()
    perm, _, bw = P.pars3_reorder(A.n, A.rowptr, A.col)
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm)
    info = P.pars3_info_get(h)
    assert (info["T"], info["W"]) == O.auto_cut(bw, 32, 1024, 1024)
    h32 = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, dtypes=P.dtype_bit(P.F32))
    assert (P.pars3_info_get(h32)["T"], P.pars3_info_get(h32)["W"]) == O.auto_cut(bw, 32, 2048, 1024)


def test_layout_routes_long_rows_and_full_tiles():
    A = W.rmat(13, 60000, seed=21)
    perm, _, _ = P.pars3_reorder(A.n, A.rowptr, A.col)
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, T=256, W=256, long_row=64)
    info = P.pars3_info_get(h)
    assert info["long_rows"] > 0 and info["long_pieces"] >= 1
    assert info["half_entries"] + (info["full_entries"] + info["long_entries"]) // 2 == A.nnz
    assert P.pars3_layout_check(h) == 0


@pytest.mark.parametrize("T,long_row,piece", [(32, 1, 0), (256, 2, 8), (4096, 2, 0), (1024, 128, 255), (512, 3, 9)])
def test_long_row_pieces_cover_every_long_entry(T, long_row, piece):
    """Pieces of the long rows: every long row with at least one entry, all
    of its pieces but the last of the full length, each piece once in the
    long slices, the long rows' entries reconstructing the split
    (pars3_layout_check)."""
    A = W.grid((120, 110), "normal", 17)
    perm, _, _ = P.pars3_reorder(A.n, A.rowptr, A.col)
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, T=T, W=32, long_row=long_row, piece=piece)
    info = P.pars3_info_get(h)
    assert info["half_entries"] + (info["full_entries"] + info["long_entries"]) // 2 == A.nnz
    if long_row < 4:
        assert info["long_rows"] > A.n // 2 and info["long_pieces"] >= info["long_rows"]
    assert P.pars3_layout_check(h) == 0


def test_piece_length_and_long_slices_range():
    A = W.grid((30, 20), "uniform", 6)
    for bad in (-1, 1, 7, 256):
        with pytest.raises(P.Pars3Error) as e:
            P.pars3_split(A.n, A.rowptr, A.col, A.val, None, T=32, W=32, piece=bad)
        assert e.value.code == P.EINVAL
    for bad in (-1, 1025):
        with pytest.raises(P.Pars3Error) as e:
            P.pars3_split(A.n, A.rowptr, A.col, A.val, None, T=32, W=32, long_slices=bad)
        assert e.value.code == P.EINVAL
    for good in (1, 16, 1024):
        h = P.pars3_split(A.n, A.rowptr, A.col, A.val, None, T=32, W=32, long_row=2, long_slices=good)
        assert P.pars3_layout_check(h) == 0


def test_overfull_tile_leaves_the_half_path():
    """A tile whose middle entries do not fit in shared memory is stored in
    full (both triangles) instead; the layout still reconstructs the split."""
    A = W.banded_skew(4096, 1024, 0.05, 11)
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, T=1024, W=1024)
    info = P.pars3_info_get(h)
    assert info["half_entries"] < A.nnz
    assert info["full_entries"] + info["long_entries"] > 0
    assert info["half_entries"] + (info["full_entries"] + info["long_entries"]) // 2 == A.nnz
    assert P.pars3_layout_check(h) == 0


def test_invalid_inputs():
    A = W.random_skew(20, 0.3, 1)
    bad = W.random_skew(20, 0.3, 1)
    bad.col = bad.col.copy()
    bad.col[0] = 19                                      # above the diagonal
    with pytest.raises(P.Pars3Error) as e:
        P.pars3_reorder(bad.n, bad.rowptr, bad.col)
    assert e.value.code == P.ENOTSKEW
    with pytest.raises(P.Pars3Error) as e:
        P.pars3_split(bad.n, bad.rowptr, bad.col, bad.val)
    assert e.value.code == P.ENOTSKEW
    nan = A.val.copy()
    nan[3] = np.nan
    with pytest.raises(P.Pars3Error) as e:
        P.pars3_split(A.n, A.rowptr, A.col, nan)
    assert e.value.code == P.ENONFINITE
    for T, Wc in ((64, 128), (48, 32), (32, 16), (65536, 32)):
        with pytest.raises(P.Pars3Error) as e:
            P.pars3_split(A.n, A.rowptr, A.col, A.val, T=T, W=Wc)
        assert e.value.code == P.EINVAL
    with pytest.raises(P.Pars3Error) as e:
        P.pars3_split(A.n, A.rowptr, A.col, A.val, perm=np.zeros(20, dtype=np.int32))
    assert e.value.code == P.EINVAL
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val)
    assert P.lib().pars3_spmv(h, 0, 1.0, None, None, None) == P.ESTATE
    assert P.lib().pars3_spmv(h, 2, 1.0, None, None, None) == P.EUNSUPPORTED
    assert P.pars3_strerror(P.ENOTSKEW).startswith("input is not")


@pytest.mark.parametrize("idx", range(9))
@pytest.mark.parametrize("TW", [(32, 32), (1024, 256)])
def test_symmetric_split_bit_exact(idx, TW):
    """PARS3_SPLIT_SYMMETRIC: an entry whose orientation flips keeps its
    sign; the split is the oracle's with mirror sign +1, bit for bit."""
    A = list(_mats())[idx]
    T, Wc = TW
    perm = O.rcm(A)[0] if idx % 2 else np.random.default_rng(idx).permutation(A.n).astype(np.int32)
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, T=T, W=Wc, dtypes=7, symmetric=True)
    ex = P.pars3_split_export(h)
    so = O.split(A, perm, T, Wc, mirror=+1.0)
    for k in KEYS:
        assert np.array_equal(ex[k], so[k]), k
    assert P.pars3_layout_check(h) == 0
    assert P.pars3_info_get(h)["symmetric"] == 1


def test_split_rejects_unknown_flags():
    A = list(_mats())[0]
    prm = P.pars3_split_params(T=64, W=32, dtypes=1, flags=2)
    out = P.C.c_void_p()
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.col, dtype=np.int32)
    v = np.ascontiguousarray(A.val, dtype=np.float64)
    rc = P.lib().pars3_split(A.n, P._p(rp), P._p(ci), P._p(v), None, P.C.byref(prm), P.C.byref(out))
    assert rc == P.EINVAL


@pytest.mark.parametrize("idx", range(9))
def test_rcm_peripheral_bit_exact(idx):
    """PARS3_RCM_PERIPHERAL: the library's pseudo-peripheral starts and the
    resulting permutation equal the oracle's bit for bit (with and without
    the guard)."""
    A = list(_mats())[idx]
    for guard in (True, False):
        flags = P.RCM_PERIPHERAL | (P.RCM_GUARD if guard else 0)
        perm, b0, b1 = P.pars3_reorder(A.n, A.rowptr, A.col, flags=flags)
        po, o0, o1 = O.rcm(A, guard=guard, peripheral=True)
        assert np.array_equal(perm, po) and (b0, b1) == (o0, o1)


def test_rcm_peripheral_hand_example_and_bad_flags():
    import json
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "rcm_spider_peripheral.json")))
    low = sorted({(max(a, b), min(a, b)) for a, b in g["edges"]})
    rp = np.zeros(g["n"] + 1, dtype=np.int32)
    for i, _ in low:
        rp[i + 1] += 1
    rp = np.cumsum(rp).astype(np.int32)
    col = np.array([j for _, j in low], dtype=np.int32)
    perm, b0, b1 = P.pars3_reorder(g["n"], rp, col, flags=P.RCM_GUARD | P.RCM_PERIPHERAL)
    assert perm.tolist() == g["perm_peripheral"] and (b0, b1) == (g["bw_before"], g["bw_after"])
    with pytest.raises(P.Pars3Error) as e:
        P.pars3_reorder(g["n"], rp, col, flags=8)
    assert e.value.code == P.EINVAL


def test_binding_rejects_mismatched_vectors():
    """The binding checks precision, length and layout of vectors before any
    library call (a wrong element size would otherwise be read silently)."""
    import torch
    A = list(_mats())[0]
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val)
    x64 = torch.zeros(A.n, dtype=torch.float64)
    x32 = torch.zeros(A.n, dtype=torch.float32)
    with pytest.raises(ValueError):
        P._vec(x32, P.F64, A.n, "x")
    with pytest.raises(ValueError):
        P._vec(x64, P.F32, A.n, "x")
    with pytest.raises(ValueError):
        P._vec(torch.zeros(A.n + 1, dtype=torch.float64), P.F64, A.n, "x")
    with pytest.raises(ValueError):   # not a CUDA tensor
        P._vec(x64, P.F64, A.n, "x")
    with pytest.raises(ValueError):
        P.pars3_spmv_host(h, P.F64, 1.0, np.zeros(A.n, dtype=np.float32), np.zeros(A.n))
