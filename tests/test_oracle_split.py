"""Pins of the oracle's canonical 3-way split (Sec. 3.1.2, Figs. 7-8): a
hand-worked example, exact reconstruction of P S P^T by numpy indexing, an
independent split-based product compared with the unreordered operator, and
the default cut-point rule."""
import json
import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import GOLDEN


def _from_triplets(n, trip):
    trip = sorted(trip)
    keys = np.array([r * n + c for r, c, _ in trip], dtype=np.int64)
    A = W.from_keys(n, keys, "uniform", 0)
    A.val = np.array([v for _, _, v in trip], dtype=np.float64)
    return A


@pytest.mark.parametrize("case", [0, 1])
def test_hand_worked_split(case):
    g = json.load(open(os.path.join(GOLDEN, "split_hand_6.json")))
    A = _from_triplets(g["n"], [tuple(t) for t in g["stored"]])
    c = g["cases"][case]
    sp = O.split(A, np.array(c["perm"]), g["T"], g["W"])
    for key in ("rowptr", "col", "val", "cls", "tile_ptr", "tile_list", "outer_csr", "outer_csc", "counts"):
        assert sp[key].tolist() == c[key], key


def _split_product(sp, alpha, xp):
    """y' = (alpha I + P S P^T) x' assembled class by class with numpy
    scatter-adds (a different arithmetic route from the oracle's row sums)."""
    n = sp["n"]
    rows = np.repeat(np.arange(n), np.diff(sp["rowptr"]))
    cols = sp["col"]
    v = sp["val"]
    y = alpha * xp.copy()
    for cls in (O.MID_LOCAL, O.MID_HALO, O.OUTER):
        m = sp["cls"] == cls
        np.add.at(y, rows[m], v[m] * xp[cols[m]])
        np.add.at(y, cols[m], -v[m] * xp[rows[m]])
    return y


@pytest.mark.parametrize("n,density,seed,T,W_", [(40, 0.15, 1, 8, 3), (97, 0.05, 2, 16, 16), (300, 0.02, 3, 64, 32)])
def test_reconstruction_and_product(n, density, seed, T, W_):
    A = W.random_skew(n, density, seed)
    perm = np.random.default_rng(seed).permutation(n).astype(np.int32)
    sp = O.split(A, perm, T, W_)
    # exact reconstruction of P S P^T
    Sp = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(sp["rowptr"]))
    assert np.all(sp["col"] < rows)
    Sp[rows, sp["col"]] = sp["val"]
    Sp[sp["col"], rows] = -sp["val"]
    S = O.dense(A)
    assert np.array_equal(Sp, S[np.ix_(perm, perm)])
    # classes partition the entries; distances respect the cut
    d = rows - sp["col"]
    assert sp["counts"].sum() == A.nnz
    assert np.all(d[sp["cls"] == O.OUTER] > W_)
    assert np.all(d[sp["cls"] != O.OUTER] <= W_)
    tile_of_row = rows // T
    tile_of_col = sp["col"] // T
    assert np.all(tile_of_col[sp["cls"] == O.MID_LOCAL] == tile_of_row[sp["cls"] == O.MID_LOCAL])
    assert np.all(tile_of_col[sp["cls"] == O.MID_HALO] == tile_of_row[sp["cls"] == O.MID_HALO] - 1)
    # per-tile lists: exactly the tile's middle entries, (column, row) sorted
    for t in range(len(sp["tile_ptr"]) - 1):
        lst = sp["tile_list"][sp["tile_ptr"][t]:sp["tile_ptr"][t + 1]]
        want = np.nonzero((tile_of_row == t) & (sp["cls"] != O.OUTER))[0]
        assert sorted(lst.tolist()) == want.tolist()
        keys = list(zip(sp["col"][lst], rows[lst]))
        assert keys == sorted(keys)
    oc = sp["outer_csr"]
    assert oc.tolist() == np.nonzero(sp["cls"] == O.OUTER)[0].tolist()
    keys = list(zip(sp["col"][sp["outer_csc"]], rows[sp["outer_csc"]]))
    assert keys == sorted(keys) and sorted(sp["outer_csc"].tolist()) == oc.tolist()
    # the operator through the split equals the unreordered one, permuted
    x = W.vector("uniform", n, seed)
    y = O.spmv_full(A, 0.4, x)
    yp = _split_product(sp, 0.4, x[perm])
    bound = O.Full(A).abs_bound(0.4, x)[perm]
    assert np.all(np.abs(yp - y[perm]) <= 1e-14 * bound + 1e-300)


def test_config0_split_counts():
    A, _, _ = W.config0()
    perm, _, bw = O.rcm(A)
    T, Wc = O.auto_cut(bw, 32, 4096, 1024)
    assert (T, Wc) == (1024, 128)
    sp = O.split(A, perm, T, Wc)
    assert sp["counts"][2] == 0 and sp["counts"].sum() == A.nnz


@pytest.mark.parametrize("bw,exp", [(0, (1024, 32)), (101, (1024, 128)), (128, (1024, 128)),
                                    (129, (1024, 256)), (5000, (8192, 8192)), (10**7, (8192, 8192))])
def test_auto_cut_rule(bw, exp):
    assert O.auto_cut(bw, 32, 8192, 1024) == exp


def test_split_rejects_bad_cut():
    A = W.random_skew(20, 0.2, 1)
    perm = np.arange(20, dtype=np.int32)
    with pytest.raises(ValueError):
        O.split(A, perm, 4, 5)   # W > T
    with pytest.raises(ValueError):
        O.split(A, perm, 4, 0)
