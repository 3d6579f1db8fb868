"""FP64 CPU oracle for the PARS3 hot path -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library and the library never calls it.

The heavy lifting is plain C (``oracle.c``, compiled on first use with gcc,
FP contraction off so that x86 and Arm give the same bits); this module wraps
it with ctypes and adds the numpy parts:

* ``dense``/``dense_apply``: the n x n brute force of y = (alpha I + S) x
  (Sec. 1, Eq. 1), for tiny n;
* ``mrs``: the minimal-residual iteration for shifted skew-symmetric systems
  (Sec. 1 names MRS: one product and one inner product per iteration),
  written from the Lanczos/Givens derivation restated in its docstring.

Parity status: every function here is pinned by tests/test_oracle_*.py
against values that do not come from the oracle itself (worked example of
Eqs. 2-6, closed forms, invariants, brute force, library routines).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MID_LOCAL, MID_HALO, OUTER = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (plain gcc, -O2, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            i32, i64, f64 = C.c_int32, C.c_int64, C.c_double
            lib.orc_validate.argtypes = [i32, P, P]
            lib.orc_full_csr.argtypes = [i32, P, P, P, f64, P, P, P]
            lib.orc_spmv_full.argtypes = [i32, f64, P, P, P, P, P]
            lib.orc_spmv_full.restype = None
            lib.orc_spmm_full.argtypes = [i32, i32, f64, P, P, P, P, P]
            lib.orc_spmm_full.restype = None
            lib.orc_spmv_sss.argtypes = [i32, f64, f64, P, P, P, P, P]
            lib.orc_spmv_sss.restype = None
            lib.orc_bandwidth.argtypes = [i32, P, P, P]
            lib.orc_bandwidth.restype = i64
            lib.orc_rcm.argtypes = [i32, P, P, i32, P, P, P]
            lib.orc_split.argtypes = [i32, P, P, P, f64, P, i32, i32, P, P, P, P, P, P, P, P, P]
            lib.orc_auto_cut.argtypes = [i64, i32, i32, i32, P, P]
            lib.orc_auto_cut.restype = None
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _csr(A):
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.col, dtype=np.int32)
    v = np.ascontiguousarray(A.val, dtype=np.float64)
    return rp, ci, v


# ---------------------------------------------------------------------------
# O1 operator
# ---------------------------------------------------------------------------

def validate(A) -> int:
    rp, ci, _ = _csr(A)
    return int(_L().orc_validate(A.n, _p(rp), _p(ci)))


class Full:
    """Full-storage CSR of S = L + mirror L^T (mirror -1: skew-symmetric, the
    paper's case; +1: symmetric)."""

    def __init__(self, A, mirror: float = -1.0):
        rp, ci, v = _csr(A)
        self.n = A.n
        self.rowptr = np.zeros(A.n + 1, dtype=np.int64)
        self.col = np.zeros(2 * ci.shape[0], dtype=np.int32)
        self.val = np.zeros(2 * ci.shape[0], dtype=np.float64)
        rc = _L().orc_full_csr(A.n, _p(rp), _p(ci), _p(v), float(mirror), _p(self.rowptr), _p(self.col),
                               _p(self.val))
        if rc != 0:
            raise MemoryError("orc_full_csr")

    def apply(self, alpha: float, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(self.n, dtype=np.float64)
        _L().orc_spmv_full(self.n, float(alpha), _p(self.rowptr), _p(self.col), _p(self.val), _p(x), _p(y))
        return y

    def apply_block(self, alpha: float, X: np.ndarray) -> np.ndarray:
        X = np.ascontiguousarray(X, dtype=np.float64)
        k = X.shape[1]
        Y = np.empty_like(X)
        _L().orc_spmm_full(self.n, k, float(alpha), _p(self.rowptr), _p(self.col), _p(self.val), _p(X), _p(Y))
        return Y

    def abs_bound(self, alpha: float, x: np.ndarray) -> np.ndarray:
        """Per-row error scale |alpha||x_i| + sum_j |s_ij||x_j| (tolerance denominator)."""
        ax = np.abs(np.asarray(x, dtype=np.float64))
        out = np.empty(self.n, dtype=np.float64)
        absval = np.abs(self.val)
        _L().orc_spmv_full(self.n, abs(float(alpha)), _p(self.rowptr), _p(self.col), _p(absval),
                           _p(np.ascontiguousarray(ax)), _p(out))
        return out

    def abs_bound_block(self, alpha: float, X: np.ndarray) -> np.ndarray:
        absval = np.abs(self.val)
        aX = np.ascontiguousarray(np.abs(X), dtype=np.float64)
        Y = np.empty_like(aX)
        _L().orc_spmm_full(self.n, aX.shape[1], abs(float(alpha)), _p(self.rowptr), _p(self.col),
                           _p(absval), _p(aX), _p(Y))
        return Y


def spmv_full(A, alpha: float, x: np.ndarray, mirror: float = -1.0) -> np.ndarray:
    """y = (alpha I + S) x through the full-storage CSR of the unreordered S."""
    return Full(A, mirror).apply(alpha, x)


def spmv_sss(A, alpha: float, x: np.ndarray, mirror: float = -1.0) -> np.ndarray:
    """The serial SSS skew SpMV of Sec. 3.1.1 (pair update of Eqs. 2-6)."""
    rp, ci, v = _csr(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(A.n, dtype=np.float64)
    _L().orc_spmv_sss(A.n, float(alpha), float(mirror), _p(rp), _p(ci), _p(v), _p(x), _p(y))
    return y


def dense(A, mirror: float = -1.0) -> np.ndarray:
    """Dense S = L + mirror L^T (brute force for tiny n)."""
    S = np.zeros((A.n, A.n), dtype=np.float64)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    S[rows, A.col] = A.val
    S[A.col, rows] = mirror * A.val
    return S


def dense_apply(A, alpha: float, x: np.ndarray) -> np.ndarray:
    return alpha * np.asarray(x) + dense(A) @ np.asarray(x)


# ---------------------------------------------------------------------------
# O2 reordering
# ---------------------------------------------------------------------------

def bandwidth(A, perm=None) -> int:
    rp, ci, _ = _csr(A)
    p = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
    return int(_L().orc_bandwidth(A.n, _p(rp), _p(ci), None if p is None else _p(p)))


def rcm(A, guard: bool = True, peripheral: bool = False, local: bool = False):
    """(perm new->old, bandwidth before, bandwidth after); peripheral: start
    each component at a George-Liu pseudo-peripheral vertex; local: RCM of the
    pattern's local edges only, those on a triangle or a 4-cycle
    (orc_rcm_local)."""
    rp, ci, _ = _csr(A)
    perm = np.empty(A.n, dtype=np.int32)
    b0 = np.zeros(1, dtype=np.int64)
    b1 = np.zeros(1, dtype=np.int64)
    flags = (1 if guard else 0) | (2 if peripheral else 0) | (4 if local else 0)
    rc = _L().orc_rcm(A.n, _p(rp), _p(ci), flags, _p(perm), _p(b0), _p(b1))
    if rc != 0:
        raise RuntimeError(f"orc_rcm failed ({rc})")
    return perm, int(b0[0]), int(b1[0])


# ---------------------------------------------------------------------------
# O3 split
# ---------------------------------------------------------------------------

def split(A, perm, T: int, W: int, mirror: float = -1.0) -> dict:
    """Canonical 3-way split (see orc_split in oracle.c)."""
    rp, ci, v = _csr(A)
    n, nnz = A.n, ci.shape[0]
    ntiles = (n + T - 1) // T
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    out = dict(
        rowptr=np.zeros(n + 1, dtype=np.int32), col=np.zeros(nnz, dtype=np.int32),
        val=np.zeros(nnz, dtype=np.float64), cls=np.zeros(nnz, dtype=np.uint8),
        tile_ptr=np.zeros(ntiles + 1, dtype=np.int32), tile_list=np.zeros(nnz, dtype=np.int32),
        outer_csr=np.zeros(nnz, dtype=np.int32), outer_csc=np.zeros(nnz, dtype=np.int32),
        counts=np.zeros(3, dtype=np.int64))
    rc = _L().orc_split(n, _p(rp), _p(ci), _p(v), float(mirror), _p(perm), int(T), int(W),
                        _p(out["rowptr"]), _p(out["col"]), _p(out["val"]), _p(out["cls"]),
                        _p(out["tile_ptr"]), _p(out["tile_list"]), _p(out["outer_csr"]),
                        _p(out["outer_csc"]), _p(out["counts"]))
    if rc != 0:
        raise ValueError(f"orc_split failed ({rc})")
    nmid = int(out["counts"][0] + out["counts"][1])
    nout = int(out["counts"][2])
    out["tile_list"] = out["tile_list"][:nmid]
    out["outer_csr"] = out["outer_csr"][:nout]
    out["outer_csc"] = out["outer_csc"][:nout]
    out["perm"] = perm
    out["T"], out["W"], out["n"] = int(T), int(W), int(n)
    return out


def auto_cut(bw: int, w_min: int, w_cap: int, t_min: int):
    T = np.zeros(1, dtype=np.int32)
    W = np.zeros(1, dtype=np.int32)
    _L().orc_auto_cut(int(bw), int(w_min), int(w_cap), int(t_min), _p(T), _p(W))
    return int(T[0]), int(W[0])


# ---------------------------------------------------------------------------
# O4 MRS
# ---------------------------------------------------------------------------

def mrs(apply_S, n: int, alpha: float, b: np.ndarray, x0=None, rtol: float = 1e-10,
        maxit: int = 100000, history: bool = False, true_residual=None):
    """Minimal residual method for (alpha I + S) x = b with S skew (Sec. 1).

    x_k minimizes ||b - A x|| over x0 + K_k(A, r0), and K_k(A, r0) = K_k(S, r0).
    Skew Lanczos: v_1 = r0/beta_0; w = S v_j + beta_{j-1} v_{j-1}
    (v_j^T S v_j = 0, so there is no diagonal coefficient), beta_j = ||w||,
    v_{j+1} = w/beta_j.  Then A V_k = V_{k+1} H_k where column j of H_k holds
    -beta_{j-1} (row j-1), alpha (row j), beta_j (row j+1).  Givens rotations
    G_j zero beta_j: gamma_1 = alpha, rho_j = hypot(gamma_j, beta_j),
    c_j = gamma_j/rho_j, s_j = beta_j/rho_j, gamma_{j+1} = alpha/c_j; the
    first superdiagonal of R vanishes and R[j-2, j] = -s_{j-2} beta_{j-1}.
    Search directions p_j = (v_j - R[j-2, j] p_{j-2}) / rho_j; with t_1 = beta_0,
    tau_j = c_j t_j, t_{j+1} = -s_j t_j, x_j = x_{j-1} + tau_j p_j and
    ||b - A x_j|| = |t_{j+1}| in exact arithmetic.

    Stops when the recursive estimate |t_{j+1}| <= rtol ||b|| and, if
    ``true_residual`` (callable x -> ||b - A x||) is given, the true residual
    confirms it; or when beta_j == 0 (the Krylov space is invariant: exact).
    Returns (x, info) with info = {iters, est, hist}.
    """
    if alpha == 0.0:
        raise ValueError("MRS needs alpha != 0 (gamma recursion divides by c_j)")
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - (alpha * x + apply_S(x))
    nb = float(np.linalg.norm(b))
    beta_prev = float(np.linalg.norm(r))          # beta_0
    hist = [beta_prev] if history else None
    if beta_prev == 0.0:
        return x, dict(iters=0, est=0.0, hist=hist)
    v_prev = np.zeros(n)
    v = r / beta_prev
    t = beta_prev                                  # t_1
    gamma = alpha                                  # gamma_1
    s_hist = [0.0, 0.0]                            # s_{j-2}, s_{j-1} (s_{-1} = s_0 = 0)
    p_hist = [np.zeros(n), np.zeros(n)]            # p_{j-2}, p_{j-1}
    j = 0
    for j in range(1, maxit + 1):
        w = apply_S(v) + beta_prev * v_prev
        beta = float(np.linalg.norm(w))
        rho = float(np.hypot(gamma, beta))
        c, s = gamma / rho, beta / rho
        r_2j = -s_hist[0] * beta_prev              # R[j-2, j]
        p = (v - r_2j * p_hist[0]) / rho
        tau = c * t
        t = -s * t
        x = x + tau * p
        if history:
            hist.append(abs(t))
        if beta == 0.0:
            break
        if abs(t) <= rtol * nb:
            if true_residual is None or true_residual(x) <= rtol * nb:
                break
        v_prev, v = v, w / beta
        beta_prev = beta
        gamma = alpha / c
        s_hist = [s_hist[1], s]
        p_hist = [p_hist[1], p]
    return x, dict(iters=j, est=abs(t), hist=hist)
