"""RCM on the GPU (pars3_reorder_device) against the oracle's RCM (Sec. 1,
Sec. 3.1.2): the permutation and both bandwidths must be identical, element
for element, for the guard on and off and for pseudo-peripheral starts.
Covers many components, isolated vertices, paths, stars, grids, R-MAT and,
at full size, the matrices the benchmark runs."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_2407_17651_gb300 import _build
from paper_2407_17651_gb300 import pars3 as P

pytestmark = pytest.mark.gpu

FLAGS = [0, P.RCM_GUARD, P.RCM_GUARD | P.RCM_PERIPHERAL, P.RCM_PERIPHERAL]
LOCAL_FLAGS = [P.RCM_LOCAL, P.RCM_GUARD | P.RCM_LOCAL, P.RCM_GUARD | P.RCM_PERIPHERAL | P.RCM_LOCAL]


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    _build.build()
    O.build()
    torch.cuda.init()


def _dev(A):
    import torch
    return (torch.from_numpy(np.ascontiguousarray(A.rowptr, dtype=np.int32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(A.col, dtype=np.int32)).cuda())


def _check(A, flags):
    rp, ci = _dev(A)
    perm, b0, b1 = P.pars3_reorder_device(A.n, rp, ci, flags)
    po, ob0, ob1 = _oracle(A, flags)
    got = perm.cpu().numpy()
    assert np.array_equal(got, po), (A.name, flags)
    assert (b0, b1) == (ob0, ob1), (A.name, flags)
    return got


def _oracle(A, flags):
    return O.rcm(A, guard=bool(flags & P.RCM_GUARD), peripheral=bool(flags & P.RCM_PERIPHERAL),
                 local=bool(flags & P.RCM_LOCAL))


def _from_pairs(n, pairs, name=""):
    pairs = sorted({(max(i, j), min(i, j)) for i, j in pairs if i != j})
    rp = np.zeros(n + 1, dtype=np.int64)
    for i, _ in pairs:
        rp[i + 1] += 1
    rp = np.cumsum(rp).astype(np.int32)
    ci = np.array([j for _, j in pairs], dtype=np.int32)
    return W.SkewMatrix(n, rp, ci, np.ones(len(ci)), name=name)


def _random_graph(n, m, seed):
    rng = np.random.default_rng(seed)
    pairs = set()
    m = min(m, n * (n - 1) // 2)
    while len(pairs) < m:
        i, j = (int(v) for v in rng.integers(0, n, 2))
        if i != j:
            pairs.add((i, j))
    return _from_pairs(n, pairs, f"random n={n} m={m} seed={seed}")


@pytest.mark.parametrize("flags", FLAGS)
def test_small_random_graphs(flags):
    # sparse enough that most have several components and isolated vertices
    for seed in range(30):
        rng = np.random.default_rng(seed)
        n = int(rng.integers(1, 200))
        _check(_random_graph(n, int(rng.integers(0, 2 * n)), seed), flags)


@pytest.mark.parametrize("flags", FLAGS)
def test_special_patterns(flags):
    cases = [
        _from_pairs(1, [], "one vertex"),
        _from_pairs(7, [], "no edges"),
        _from_pairs(50, [(i, i + 1) for i in range(49)], "path"),
        _from_pairs(40, [(0, i) for i in range(1, 40)], "star at 0"),
        _from_pairs(40, [(39, i) for i in range(39)], "star at 39"),
        _from_pairs(30, [(i, j) for i in range(30) for j in range(i)], "complete"),
        _from_pairs(60, [(i, i + 1) for i in range(0, 58, 3)] + [(5, 40)], "many small components"),
        _from_pairs(5000, [(i, (i * 7919 + 1) % 5000) for i in range(5000)], "one long cycle-ish"),
    ]
    for A in cases:
        _check(A, flags)


@pytest.mark.parametrize("flags", FLAGS)
def test_structured_matrices(flags):
    cases = [
        W.grid((37, 23), "normal", 1),
        W.grid((9, 8, 7), "normal", 2),
        W.grid_plus_random((30, 30), 0.05, "normal", 3),
        W.rmat(12, 30000, seed=4),
        W.banded_skew(3000, 40, 0.3, 5),
        W.random_skew(2000, 0.002, 6),
    ]
    for A in cases:
        _check(A, flags)


def test_agrees_with_host_ordering():
    A = W.grid_plus_random((64, 64), 0.01, "normal", 7)
    for flags in FLAGS:
        ph, hb0, hb1 = P.pars3_reorder(A.n, A.rowptr, A.col, flags)
        rp, ci = _dev(A)
        pd, db0, db1 = P.pars3_reorder_device(A.n, rp, ci, flags)
        assert np.array_equal(pd.cpu().numpy(), ph) and (hb0, hb1) == (db0, db1)


def test_empty_and_errors():
    import torch
    z = torch.zeros(1, dtype=torch.int32, device="cuda")
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    perm, b0, b1 = P.pars3_reorder_device(0, z, e)
    assert perm.numel() == 0 and (b0, b1) == (0, 0)
    # entries on or above the diagonal, unsorted or duplicate columns, bad row pointers
    bad = [
        ([0, 1, 1], [0]),          # (0, 0) on the diagonal
        ([0, 0, 1], [1]),          # (1, 1)
        ([0, 0, 1, 3], [0, 1, 0]),  # row 2 unsorted
        ([0, 0, 1, 3], [0, 1, 1]),  # row 2 duplicate
        ([0, 0, 2, 2], [0, 0]),     # row 1 duplicate
        ([1, 1, 1], [0]),           # rowptr[0] != 0
        ([0, 2, 1, 2], [0, 0]),     # decreasing rowptr
    ]
    for rp, ci in bad:
        n = len(rp) - 1
        with pytest.raises(P.Pars3Error) as ei:
            P.pars3_reorder_device(n, torch.tensor(rp, dtype=torch.int32, device="cuda"),
                                   torch.tensor(ci, dtype=torch.int32, device="cuda"))
        assert ei.value.code == P.ENOTSKEW, (rp, ci)
    rp = torch.tensor([0, 0, 1], dtype=torch.int32, device="cuda")
    ci = torch.tensor([0], dtype=torch.int32, device="cuda")
    with pytest.raises(P.Pars3Error) as ei:
        P.pars3_reorder_device(2, rp, ci, 64)
    assert ei.value.code == P.EINVAL
    # the library still works after the rejected calls
    perm, _, _ = P.pars3_reorder_device(2, rp, ci, 0)
    assert sorted(perm.cpu().tolist()) == [0, 1]


def test_run_to_run_identical():
    A = W.rmat(14, 120000, seed=8)
    rp, ci = _dev(A)
    first = P.pars3_reorder_device(A.n, rp, ci, P.RCM_GUARD | P.RCM_PERIPHERAL)[0].cpu().numpy()
    for _ in range(3):
        again = P.pars3_reorder_device(A.n, rp, ci, P.RCM_GUARD | P.RCM_PERIPHERAL)[0].cpu().numpy()
        assert np.array_equal(first, again)


@pytest.mark.slow
@pytest.mark.parametrize("name", ["cfg1", "cfg2"])
def test_full_size_bit_exact(name):
    A = W.config1()[0] if name == "cfg1" else W.config2()[0]
    for flags in (P.RCM_GUARD, P.RCM_GUARD | P.RCM_PERIPHERAL):
        _check(A, flags)


@pytest.mark.slow
def test_all_batched_matrices_bit_exact():
    for m, shp in enumerate(W.config4_shapes()):
        _check(W.config4_matrix(m, shp), P.RCM_GUARD)


def _batch_cases():
    cases = [_from_pairs(0, [], "empty"), _from_pairs(1, [], "one vertex"), _from_pairs(9, [], "no edges")]
    cases += [_random_graph(int(n), int(2 * n), s) for s, n in enumerate((5, 17, 60, 150, 301))]
    cases += [W.grid((21, 13), "normal", 11), W.grid((6, 5, 4), "normal", 12),
              W.grid_plus_random((25, 25), 0.05, "normal", 13), W.rmat(10, 6000, seed=14),
              _from_pairs(0, [], "empty again"), _from_pairs(40, [(0, i) for i in range(1, 40)], "star")]
    return cases


@pytest.mark.parametrize("flags", FLAGS + LOCAL_FLAGS)
def test_batched_matches_oracle_per_matrix(flags):
    cases = _batch_cases()
    pats = [(A.n,) + _dev(A) for A in cases]
    out = P.pars3_reorder_device_batched(pats, flags)
    assert len(out) == len(cases)
    for A, (perm, b0, b1) in zip(cases, out):
        po, ob0, ob1 = _oracle(A, flags)
        assert np.array_equal(perm.cpu().numpy(), po), (A.name, flags)
        assert (b0, b1) == (ob0, ob1), (A.name, flags)


def test_batched_rejects_a_bad_matrix():
    import torch
    cases = _batch_cases()[:6]
    pats = [(A.n,) + _dev(A) for A in cases]
    bad = (3, torch.tensor([0, 0, 1, 3], dtype=torch.int32, device="cuda"),
           torch.tensor([0, 1, 1], dtype=torch.int32, device="cuda"))   # duplicate column in row 2
    with pytest.raises(P.Pars3Error) as ei:
        P.pars3_reorder_device_batched(pats[:3] + [bad] + pats[3:])
    assert ei.value.code == P.ENOTSKEW
    # a row pointer reaching past its own matrix's entries, into the next
    # matrix's (rows 1 and 2 claim entries [0, 3) and [3, 2) of two stored)
    bad2 = (3, torch.tensor([0, 0, 3, 2], dtype=torch.int32, device="cuda"),
            torch.tensor([0, 1], dtype=torch.int32, device="cuda"))
    with pytest.raises(P.Pars3Error) as ei:
        P.pars3_reorder_device_batched([bad2] + pats)
    assert ei.value.code == P.ENOTSKEW
    out = P.pars3_reorder_device_batched(pats)   # still usable
    assert len(out) == len(pats)
    assert P.pars3_reorder_device_batched([]) == []


@pytest.mark.slow
def test_batched_all_64_matrices_in_one_call():
    mats = [W.config4_matrix(m, shp) for m, shp in enumerate(W.config4_shapes())]
    for flags in (P.RCM_GUARD, P.RCM_GUARD | P.RCM_PERIPHERAL):
        out = P.pars3_reorder_device_batched([(A.n,) + _dev(A) for A in mats], flags)
        for A, (perm, b0, b1) in zip(mats, out):
            po, ob0, ob1 = O.rcm(A, guard=True, peripheral=bool(flags & P.RCM_PERIPHERAL))
            assert np.array_equal(perm.cpu().numpy(), po) and (b0, b1) == (ob0, ob1), A.name


@pytest.mark.parametrize("flags", LOCAL_FLAGS)
def test_local_edge_rcm(flags):
    """PARS3_RCM_LOCAL on the GPU: the RCM of the edges on a triangle or a
    4-cycle (degree products above 4096 kept untested), bandwidths and guard
    over every edge, against orc_rcm with the local flag."""
    rng = np.random.default_rng(21)
    cases = [_random_graph(int(n), int(3 * n), s) for s, n in enumerate(rng.integers(5, 300, 12))]
    cases += [W.grid_plus_random((40, 30), 0.02, "normal", 22), W.grid_plus_random((12, 10, 9), 0.01, "normal", 23),
              W.grid((33, 17), "normal", 24), W.rmat(11, 12000, seed=25),
              _from_pairs(100, [(0, i) for i in range(1, 100)] + [(i, i + 1) for i in range(1, 99)], "wheel"),
              _from_pairs(7, [], "no edges")]
    for A in cases:
        _check(A, flags)


@pytest.mark.slow
def test_local_edge_rcm_full_size():
    _check(W.config1()[0], P.RCM_GUARD | P.RCM_LOCAL)
