"""Seeded synthetic skew-symmetric workloads.

This module only *generates inputs*: sparsity patterns, random symmetric
relabelings, random values and random vectors.  It contains none of the
method's arithmetic (no reordering, no splitting, no products), so both the
CPU oracle and the CUDA path can draw their inputs from it.

Every matrix is returned as the strict lower triangle L of a skew-symmetric
S = L - L^T in CSR form (row pointers int32[n+1], sorted unique column
indices int32[nnz], float64 values), i.e. the half storage of Sec. 3 of the
paper (the SSS layout without a diagonal: S has a zero diagonal).

The workloads stand in for the SuiteSparse matrices of Table 1, which are not
available here; their shapes follow the five benchmark configurations of the
build (2D/3D grid graphs, grids with random long-range edges, R-MAT power-law
graphs, batches of uneven grids).  Random numbers come from numpy's PCG64
seeded through SeedSequence([seed, stream]) so that the pattern, the
relabeling, the values and the vectors use independent streams.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 240717651  # base seed; configuration c uses SEED_BASE + c

# independent random streams per seed
_S_PATTERN, _S_PERM, _S_VALUES, _S_VECTOR, _S_SHAPE = 0, 1, 2, 3, 4


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([int(seed), int(stream)]))


@dataclass
class SkewMatrix:
    """Strict-lower CSR of a skew-symmetric matrix plus a description."""
    n: int
    rowptr: np.ndarray   # int32[n+1]
    col: np.ndarray      # int32[nnz]
    val: np.ndarray      # float64[nnz]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])


# --------------------------------------------------------------------------
# pattern helpers (pure index bookkeeping)
# --------------------------------------------------------------------------

def _sorted_unique(k: np.ndarray) -> np.ndarray:
    """Sorted unique values (sort based; independent of numpy's unique path)."""
    k = np.sort(k, kind="stable")
    if k.shape[0] == 0:
        return k
    keep = np.empty(k.shape[0], dtype=bool)
    keep[0] = True
    np.not_equal(k[1:], k[:-1], out=keep[1:])
    return k[keep]


def _first_occurrence(k: np.ndarray):
    """(sorted unique values, index of each value's first occurrence)."""
    order = np.argsort(k, kind="stable")
    ks = k[order]
    if ks.shape[0] == 0:
        return ks, order
    keep = np.empty(ks.shape[0], dtype=bool)
    keep[0] = True
    np.not_equal(ks[1:], ks[:-1], out=keep[1:])
    return ks[keep], order[keep]


def _in_sorted(k: np.ndarray, sorted_ref: np.ndarray) -> np.ndarray:
    """Membership test of k in a sorted unique array."""
    if sorted_ref.shape[0] == 0:
        return np.zeros(k.shape[0], dtype=bool)
    pos = np.searchsorted(sorted_ref, k)
    pos = np.minimum(pos, sorted_ref.shape[0] - 1)
    return sorted_ref[pos] == k


def _pairs_to_lower_keys(n: int, u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Map undirected pairs to unique sorted keys row*n+col with row > col."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    r = np.maximum(u, v)
    c = np.minimum(u, v)
    return _sorted_unique(r * n + c)


def _keys_to_csr(n: int, keys: np.ndarray):
    rows = keys // n
    cols = (keys - rows * n).astype(np.int32)
    counts = np.bincount(rows, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("too many nonzeros for int32 indices")
    return rowptr.astype(np.int32), cols


def _relabel(n: int, keys: np.ndarray, seed: int) -> np.ndarray:
    """Apply a random symmetric permutation v -> p[v] to a set of edges."""
    p = _rng(seed, _S_PERM).permutation(n).astype(np.int64)
    rows = keys // n
    cols = keys - rows * n
    return _pairs_to_lower_keys(n, p[rows], p[cols])


def _values(kind: str, m: int, seed: int) -> np.ndarray:
    g = _rng(seed, _S_VALUES)
    if kind == "uniform":
        return g.uniform(-1.0, 1.0, size=m)
    if kind == "normal":
        return g.standard_normal(size=m)
    raise ValueError(kind)


def vector(kind: str, shape, seed: int, stream: int = _S_VECTOR) -> np.ndarray:
    """Random float64 vector / row-major block of vectors."""
    g = _rng(seed, stream)
    if kind == "uniform":
        return g.uniform(-1.0, 1.0, size=shape)
    if kind == "normal":
        return g.standard_normal(size=shape)
    raise ValueError(kind)


def grid_edges(dims) -> tuple[np.ndarray, np.ndarray]:
    """Edges of the 2D 5-point or 3D 7-point grid graph (natural labels)."""
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    idx = np.arange(n, dtype=np.int64).reshape(dims[::-1])  # C order: last dim fastest
    us, vs = [], []
    for axis in range(len(dims)):
        sl_a = [slice(None)] * len(dims)
        sl_b = [slice(None)] * len(dims)
        sl_a[axis] = slice(0, -1)
        sl_b[axis] = slice(1, None)
        us.append(idx[tuple(sl_a)].ravel())
        vs.append(idx[tuple(sl_b)].ravel())
    return np.concatenate(us), np.concatenate(vs)


def from_keys(n: int, keys: np.ndarray, value_kind: str, seed: int, name: str = "",
              meta: dict | None = None) -> SkewMatrix:
    """Build the strict-lower CSR; values drawn in (row, col) order."""
    rowptr, col = _keys_to_csr(n, keys)
    val = _values(value_kind, col.shape[0], seed)
    return SkewMatrix(n, rowptr, col, val, name, dict(meta or {}))


# --------------------------------------------------------------------------
# workload families
# --------------------------------------------------------------------------

def grid(dims, value_kind: str, seed: int, permute: bool = True, name: str = "") -> SkewMatrix:
    """2D/3D grid graph, optionally under a random symmetric permutation."""
    n = int(np.prod(dims))
    u, v = grid_edges(dims)
    keys = _pairs_to_lower_keys(n, u, v)
    if permute:
        keys = _relabel(n, keys, seed)
    return from_keys(n, keys, value_kind, seed, name or f"grid{'x'.join(map(str, dims))}",
                     {"dims": list(map(int, dims)), "permuted": permute})


def fem_grid2d(a: int, b: int, dofs: int, value_kind: str, seed: int, permute: bool = True,
               name: str = "") -> SkewMatrix:
    """A finite-element-like pattern: an a x b grid of nodes with `dofs`
    unknowns each, every unknown coupled to all unknowns of its node and of
    the 8 surrounding nodes (9-point stencil).  About 9 * dofs - 1 entries
    per full row and an RCM bandwidth near (min(a, b) + 1) * dofs: the shape
    of the paper's benchmark matrices (35-56 entries per row, bandwidth a few
    thousandths to a few hundredths of n, Table 1)."""
    nn = a * b
    n = nn * dofs
    node = np.arange(nn, dtype=np.int64).reshape(a, b)
    pu, pv = [node.ravel()], [node.ravel()]   # self pairs (different unknowns of one node)
    for di, dj in ((0, 1), (1, -1), (1, 0), (1, 1)):
        i0, i1 = max(0, -di), a - max(0, di)
        j0, j1 = max(0, -dj), b - max(0, dj)
        pu.append(node[i0:i1, j0:j1].ravel())
        pv.append(node[i0 + di:i1 + di, j0 + dj:j1 + dj].ravel())
    pu = np.concatenate(pu)
    pv = np.concatenate(pv)
    k = np.arange(dofs, dtype=np.int64)
    u = (pu[:, None, None] * dofs + k[None, :, None]).repeat(dofs, axis=2).ravel()
    v = (pv[:, None, None] * dofs + k[None, None, :]).repeat(dofs, axis=1).ravel()
    keys = _pairs_to_lower_keys(n, u, v)
    if permute:
        keys = _relabel(n, keys, seed)
    return from_keys(n, keys, value_kind, seed, name or f"fem{a}x{b}x{dofs}",
                     {"nodes": [int(a), int(b)], "dofs": int(dofs), "permuted": permute})


def grid_plus_random(dims, frac_extra: float, value_kind: str, seed: int, name: str = "") -> SkewMatrix:
    """Grid graph plus round(frac_extra * #grid edges) distinct random pairs
    that are neither grid edges nor self loops, then a random relabeling."""
    n = int(np.prod(dims))
    u, v = grid_edges(dims)
    gkeys = _pairs_to_lower_keys(n, u, v)
    m_extra = int(round(frac_extra * gkeys.shape[0]))
    g = _rng(seed, _S_PATTERN)
    extra = np.empty(0, dtype=np.int64)
    while extra.shape[0] < m_extra:
        need = m_extra - extra.shape[0]
        a = g.integers(0, n, size=2 * need + 1024, dtype=np.int64)
        b = g.integers(0, n, size=2 * need + 1024, dtype=np.int64)
        keep = a != b
        a, b = a[keep], b[keep]
        k = np.maximum(a, b) * n + np.minimum(a, b)
        k = k[~_in_sorted(k, gkeys)]
        k = k[~_in_sorted(k, np.sort(extra))]
        # first occurrences in draw order
        _, first = _first_occurrence(k)
        k = k[np.sort(first)]
        extra = np.concatenate([extra, k[:need]])
    keys = _sorted_unique(np.concatenate([gkeys, extra]))
    keys = _relabel(n, keys, seed)
    return from_keys(n, keys, value_kind, seed, name or "grid+random",
                     {"dims": list(map(int, dims)), "extra_edges": int(m_extra)})


def rmat(scale: int, nnz_target: int, abcd=(0.57, 0.19, 0.19, 0.05), value_kind="uniform",
         seed: int = 0, name: str = "") -> SkewMatrix:
    """Symmetric R-MAT pattern: edges drawn bit by bit with quadrant
    probabilities (a, b, c, d), self loops dropped, symmetrized and
    deduplicated; batches are drawn until at least nnz_target unique
    strict-lower pairs exist, then exactly nnz_target of them are kept,
    chosen uniformly at random; finally the graph is randomly relabeled."""
    n = 1 << scale
    a, b, c, _ = abcd
    g = _rng(seed, _S_PATTERN)
    keys = np.empty(0, dtype=np.int64)
    batch = int(nnz_target * 1.12) + 1024
    while keys.shape[0] < nnz_target:
        r = np.zeros(batch, dtype=np.uint32)
        cc = np.zeros(batch, dtype=np.uint32)
        for _lvl in range(scale):
            x = g.random(batch, dtype=np.float32)
            r <<= 1
            cc <<= 1
            r += x >= np.float32(a + b)                                   # quadrants c, d
            cc += ((x >= np.float32(a)) & (x < np.float32(a + b))) | (x >= np.float32(a + b + c))  # b, d
        keep = r != cc
        r64 = r[keep].astype(np.int64)
        c64 = cc[keep].astype(np.int64)
        k = np.maximum(r64, c64) * n + np.minimum(r64, c64)
        keys = _sorted_unique(np.concatenate([keys, k]))
        batch = max(1024, int((nnz_target - keys.shape[0]) * 1.5) + 1024)
    if keys.shape[0] > nnz_target:
        pick = g.permutation(keys.shape[0])[:nnz_target]
        keys = keys[np.sort(pick)]
    keys = _relabel(n, keys, seed)
    return from_keys(n, keys, value_kind, seed, name or f"rmat{scale}",
                     {"scale": scale, "abcd": list(abcd)})


def random_skew(n: int, density: float, seed: int, value_kind: str = "uniform") -> SkewMatrix:
    """Small random skew-symmetric matrix with an i.i.d. Bernoulli pattern
    (for tests on tiny inputs)."""
    g = _rng(seed, _S_PATTERN)
    if n < 2:
        return from_keys(n, np.empty(0, dtype=np.int64), value_kind, seed, f"rand{n}")
    i, j = np.tril_indices(n, -1)
    keep = g.random(i.shape[0]) < density
    keys = np.sort(i[keep].astype(np.int64) * n + j[keep])
    return from_keys(n, keys, value_kind, seed, f"rand{n}_{density}")


def banded_skew(n: int, bw: int, density: float, seed: int, value_kind: str = "uniform") -> SkewMatrix:
    """Random skew matrix whose stored entries satisfy 1 <= i-j <= bw."""
    g = _rng(seed, _S_PATTERN)
    rows, cols = [], []
    for d in range(1, min(bw, n - 1) + 1):
        i = np.arange(d, n, dtype=np.int64)
        keep = g.random(i.shape[0]) < density
        rows.append(i[keep])
        cols.append(i[keep] - d)
    if rows:
        keys = np.sort(np.concatenate(rows) * n + np.concatenate(cols))
    else:
        keys = np.empty(0, dtype=np.int64)
    return from_keys(n, keys, value_kind, seed, f"band{n}_{bw}")


# --------------------------------------------------------------------------
# the five benchmark configurations
# --------------------------------------------------------------------------

def config0():
    """2D 5-point grid 200x100 (n=20,000, 39,700 stored), random relabeling,
    values U(-1,1), alpha=0, x ~ U(-1,1)."""
    s = SEED_BASE + 0
    A = grid((200, 100), "uniform", s, name="grid2d_200x100")
    x = vector("uniform", A.n, s)
    return A, 0.0, x


def config1():
    """3D 7-point grid 128^3 (n=2,097,152) plus 1% of its edge count as random
    long-range pairs, random relabeling, values N(0,1), alpha=0.5,
    x ~ U(-1,1); the SpMV is repeated 200 times after one reorder+split."""
    s = SEED_BASE + 1
    A = grid_plus_random((128, 128, 128), 0.01, "normal", s, name="grid3d_128^3+1%")
    x = vector("uniform", A.n, s)
    return A, 0.5, x


def config2(value_kind="uniform"):
    """R-MAT scale 22 (n=4,194,304), (a,b,c,d)=(0.57,0.19,0.19,0.05),
    exactly 20,000,000 stored pairs, values U(-1,1), alpha=0, x ~ N(0,1)."""
    s = SEED_BASE + 2
    A = rmat(22, 20_000_000, value_kind=value_kind, seed=s, name="rmat22")
    x = vector("normal", A.n, s)
    return A, 0.0, x


def config3_rhs(n: int):
    """Right-hand side b ~ U(-1,1) for the MRS solves (matrix = config 1's)."""
    return vector("uniform", n, SEED_BASE + 3)


CONFIG3_ALPHAS = (1.0, 0.1, 0.01)
CONFIG4_KS = (1, 4, 16, 32)


def config4_shapes(count: int = 64):
    """Grid shapes of the batched workload: n log-uniform in [1e4, 5e5],
    2D or 3D by a fair coin."""
    shapes = []
    for m in range(count):
        g = _rng(SEED_BASE + 4 + m, _S_SHAPE)
        n = int(round(math.exp(g.uniform(math.log(1e4), math.log(5e5)))))
        if g.random() < 0.5:
            a = int(round(math.sqrt(n)))
            b = int(round(n / a))
            shapes.append((a, b))
        else:
            a = int(round(n ** (1.0 / 3.0)))
            c = int(round(n / (a * a)))
            shapes.append((a, a, c))
    return shapes


def config4_matrix(m: int, shape=None) -> SkewMatrix:
    s = SEED_BASE + 4 + m
    shape = shape or config4_shapes(m + 1)[m]
    return grid(shape, "normal", s, name=f"batch{m}_{'x'.join(map(str, shape))}")


def config4_rhs(n: int, k: int, m: int) -> np.ndarray:
    return vector("uniform", (n, k), SEED_BASE + 4 + m, stream=_S_VECTOR + 16 + k)
