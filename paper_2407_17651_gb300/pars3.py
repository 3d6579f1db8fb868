"""Python binding of libpars3 (include/pars3.h): argument marshalling only.

Every entry point keeps its C name.  Host arrays are numpy arrays; device
vectors are torch CUDA tensors (torch provides device memory and streams,
the library's kernels do all the work).  A status other than PARS3_OK raises
Pars3Error; there is no fallback path: if libpars3.so is missing, loading
fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

F64, F32, BF16 = 0, 1, 2
RCM_GUARD = 1
RCM_PERIPHERAL = 2
RCM_LOCAL = 4
SPLIT_SYMMETRIC = 1
VARIANT_LOOKAHEAD = 1

OK, EINVAL, ENOTSKEW, ENOMEM, ECUDA, ENOCONV, ETIMEOUT, EUNSUPPORTED, ESTATE, ENONFINITE = \
    0, -1, -2, -3, -4, -5, -6, -7, -8, -9


def dtype_bit(d: int) -> int:
    return 1 << d


class Pars3Error(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {pars3_strerror(code)} ({code})")


class pars3_split_params(C.Structure):
    _fields_ = [("T", C.c_int32), ("W", C.c_int32), ("dtypes", C.c_int32), ("long_row", C.c_int32),
                ("flags", C.c_int32), ("piece", C.c_int32), ("long_slices", C.c_int32),
                ("lane_bytes", C.c_int32), ("variant", C.c_int32), ("reserved", C.c_int32 * 3)]


class pars3_canonical(C.Structure):
    _fields_ = [("n", C.c_int32), ("T", C.c_int32), ("W", C.c_int32), ("ntiles", C.c_int32),
                ("nnz", C.c_int64), ("counts", C.c_int64 * 3),
                ("perm", C.POINTER(C.c_int32)), ("rowptr", C.POINTER(C.c_int32)),
                ("col", C.POINTER(C.c_int32)), ("val", C.POINTER(C.c_double)),
                ("cls", C.POINTER(C.c_uint8)), ("tile_ptr", C.POINTER(C.c_int32)),
                ("tile_list", C.POINTER(C.c_int32)), ("outer_csr", C.POINTER(C.c_int32)),
                ("outer_csc", C.POINTER(C.c_int32))]


class pars3_info(C.Structure):
    _fields_ = [("n", C.c_int32), ("T", C.c_int32), ("W", C.c_int32), ("ntiles", C.c_int32),
                ("dtypes", C.c_int32), ("nnz", C.c_int64), ("half_entries", C.c_int64),
                ("full_entries", C.c_int64), ("long_entries", C.c_int64), ("long_rows", C.c_int32),
                ("long_pieces", C.c_int32), ("halo_targets", C.c_int64), ("max_tile_half", C.c_int32),
                ("smem_bytes", C.c_int32 * 3), ("device_bytes", C.c_int64),
                ("bytes_per_spmv", C.c_int64 * 3), ("bandwidth", C.c_int64), ("symmetric", C.c_int32),
                ("reserved", C.c_int32)]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if hasattr(v, "__len__") else v
        return d


class pars3_mrs_opts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("max_iter", C.c_int32), ("inner", C.c_int32),
                ("inner_rtol", C.c_double), ("max_outer", C.c_int32), ("check_every", C.c_int32),
                ("reserved", C.c_int32 * 4)]


class pars3_mrs_result(C.Structure):
    _fields_ = [("iters", C.c_int32), ("outer", C.c_int32), ("true_relres", C.c_double),
                ("est_relres", C.c_double), ("status", C.c_int32), ("reserved", C.c_int32 * 3)]

    def as_dict(self):
        return dict(iters=self.iters, outer=self.outer, true_relres=self.true_relres,
                    est_relres=self.est_relres, status=self.status)


_lib = None


def lib() -> C.CDLL:
    """Load libpars3.so from the package's build folder (raises if absent)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libpars3.so is not built ({path}); run paper_2407_17651_gb300._build.build()")
    L = C.CDLL(path)
    P, i32, i64, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "pars3_strerror": ([C.c_int], C.c_char_p),
        "pars3_version": ([P, P, P], C.c_int),
        "pars3_reorder": ([i32, P, P, i32, P, P, P], C.c_int),
        "pars3_reorder_device": ([i32, P, P, i32, P, P, P, P], C.c_int),
        "pars3_reorder_device_batched": ([i32, P, P, P, i32, P, P, P, P], C.c_int),
        "pars3_split": ([i32, P, P, P, P, P, P], C.c_int),
        "pars3_split_device": ([i32, P, P, P, P, P, P, P], C.c_int),
        "pars3_layout_digest": ([P, P], C.c_int),
        "pars3_split_export": ([P, P], C.c_int),
        "pars3_info_get": ([P, P], C.c_int),
        "pars3_layout_check": ([P], C.c_int),
        "pars3_upload": ([P, P], C.c_int),
        "pars3_spmv": ([P, i32, f64, P, P, P], C.c_int),
        "pars3_spmv_noalloc": ([P, i32, f64, P, P, P], C.c_int),
        "pars3_spmm": ([P, i32, f64, i32, P, P, P], C.c_int),
        "pars3_spmm_batched": ([P, i32, i32, P, i32, P, P, i32, P], C.c_int),
        "pars3_mrs": ([P, f64, P, P, P, P, P], C.c_int),
        "pars3_permute": ([P, i32, i32, P, P, P], C.c_int),
        "pars3_unpermute": ([P, i32, i32, P, P, P], C.c_int),
        "pars3_spmv_host": ([P, i32, f64, P, P, P], C.c_int),
        "pars3_check": ([P, P], C.c_int),
        "pars3_autotune": ([i32, P, P, P, P, P, i32, i32, P, P], C.c_int),
        "pars3_fp64_fma_rate": ([P, P], C.c_int),
        "pars3_free": ([P], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def exported_symbols():
    """Names of the entry points the binding expects (all declared in include/pars3.h)."""
    return ["pars3_strerror", "pars3_version", "pars3_reorder", "pars3_split", "pars3_split_export",
            "pars3_info_get", "pars3_layout_check", "pars3_upload", "pars3_spmv", "pars3_spmm",
            "pars3_spmm_batched", "pars3_mrs", "pars3_permute", "pars3_unpermute", "pars3_spmv_host",
            "pars3_check", "pars3_autotune", "pars3_free", "pars3_spmv_noalloc", "pars3_fp64_fma_rate",
            "pars3_reorder_device", "pars3_reorder_device_batched", "pars3_split_device",
            "pars3_layout_digest"]


def _chk(rc: int, where: str):
    if rc != OK:
        raise Pars3Error(rc, where)


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _dptr(t):
    """Device pointer of a torch tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device vectors must be CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("device vectors must be contiguous")
    return C.c_void_p(t.data_ptr())


def _vec(t, dtype: int, n: int, what: str):
    """Device pointer of a vector / row-major block for precision `dtype`:
    fp64 tensors for F64, fp32 tensors for F32 and BF16 (bf16 stores only
    the matrix values), n rows."""
    import torch
    want = torch.float64 if int(dtype) == F64 else torch.float32
    if t.dtype != want:
        raise ValueError(f"{what}: expected {want} for precision {dtype}, got {t.dtype}")
    if t.dim() not in (1, 2) or t.shape[0] != n:
        raise ValueError(f"{what}: expected {n} rows, got shape {tuple(t.shape)}")
    return _dptr(t)


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


# ---------------------------------------------------------------- host calls

def pars3_strerror(code: int) -> str:
    return lib().pars3_strerror(int(code)).decode()


def pars3_version():
    a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
    _chk(lib().pars3_version(C.byref(a), C.byref(b), C.byref(c)), "pars3_version")
    return a.value, b.value, c.value


def pars3_reorder(n: int, rowptr, col, flags: int = RCM_GUARD):
    """(perm new->old int32[n], bandwidth before, bandwidth after)."""
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(col, dtype=np.int32)
    perm = np.empty(n, dtype=np.int32)
    b0, b1 = C.c_int64(), C.c_int64()
    _chk(lib().pars3_reorder(int(n), _p(rp), _p(ci), int(flags), _p(perm), C.byref(b0), C.byref(b1)),
         "pars3_reorder")
    return perm, b0.value, b1.value



def pars3_reorder_device(n: int, rowptr, col, flags: int = RCM_GUARD, stream=None):
    """The same ordering as pars3_reorder, computed on the GPU: rowptr / col
    are int32 CUDA tensors of the strict lower pattern.  Returns (perm new->old
    as an int32 CUDA tensor, bandwidth before, bandwidth after)."""
    import torch
    for t, what in ((rowptr, "rowptr"), (col, "col")):
        if t.dtype != torch.int32:
            raise ValueError(f"{what} must be int32")
    if rowptr.numel() != int(n) + 1:
        raise ValueError("rowptr must hold n + 1 entries")
    perm = torch.empty(max(int(n), 0), dtype=torch.int32, device=rowptr.device)
    b0, b1 = C.c_int64(), C.c_int64()
    colp = _dptr(col) if col.numel() else None
    _chk(lib().pars3_reorder_device(int(n), _dptr(rowptr), colp, int(flags), _dptr(perm) if n else None,
                                    C.byref(b0), C.byref(b1), _stream(stream)), "pars3_reorder_device")
    return perm, b0.value, b1.value


def pars3_reorder_device_batched(patterns, flags: int = RCM_GUARD, stream=None):
    """pars3_reorder_device for a list of (n, rowptr, col) with int32 CUDA
    tensors, all searched in one call.  Returns a list of (perm CUDA tensor,
    bandwidth before, bandwidth after)."""
    import torch
    count = len(patterns)
    ns = np.array([int(n) for n, _, _ in patterns], dtype=np.int32)
    perms, keep = [], []
    for (n, rp, ci) in patterns:
        if rp.dtype != torch.int32 or ci.dtype != torch.int32:
            raise ValueError("rowptr and col must be int32")
        if rp.numel() != int(n) + 1:
            raise ValueError("rowptr must hold n + 1 entries")
        perms.append(torch.empty(max(int(n), 0), dtype=torch.int32, device=rp.device))
        keep += [rp, ci]
    ptrs = lambda ts: (C.c_void_p * max(count, 1))(*[t.data_ptr() if t.numel() else None for t in ts])
    rps = ptrs([p[1] for p in patterns])
    cis = ptrs([p[2] for p in patterns])
    pps = ptrs(perms)
    b0 = np.zeros(max(count, 1), dtype=np.int64)
    b1 = np.zeros(max(count, 1), dtype=np.int64)
    _chk(lib().pars3_reorder_device_batched(count, _p(ns) if count else None, rps, cis, int(flags), pps,
                                            _p(b0), _p(b1), _stream(stream)), "pars3_reorder_device_batched")
    return [(perms[m], int(b0[m]), int(b1[m])) for m in range(count)]

class Handle:
    """Owns a pars3_handle*; released by pars3_free on close/garbage collection."""

    def __init__(self, ptr: C.c_void_p, n: int):
        self.ptr = ptr
        self.n = n

    def close(self):
        if self.ptr:
            lib().pars3_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        if not self.ptr:
            raise ValueError("handle is closed")
        return self.ptr


def pars3_split(n: int, rowptr, col, val, perm=None, T: int = 0, W: int = 0, dtypes: int = 0,
                long_row: int = 0, symmetric: bool = False, piece: int = 0, long_slices: int = 0,
                lane_bytes: int = 0, variant: int = 0) -> Handle:
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(col, dtype=np.int32)
    v = np.ascontiguousarray(val, dtype=np.float64)
    pm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
    prm = pars3_split_params(T=T, W=W, dtypes=dtypes, long_row=long_row,
                             flags=SPLIT_SYMMETRIC if symmetric else 0, piece=piece, long_slices=long_slices,
                             lane_bytes=lane_bytes, variant=variant)
    out = C.c_void_p()
    _chk(lib().pars3_split(int(n), _p(rp), _p(ci), _p(v), None if pm is None else _p(pm), C.byref(prm),
                           C.byref(out)), "pars3_split")
    return Handle(out, n)


def pars3_split_device(n: int, rowptr, col, val, perm=None, T: int = 0, W: int = 0, dtypes: int = 0,
                       long_row: int = 0, symmetric: bool = False, piece: int = 0, long_slices: int = 0,
                       lane_bytes: int = 0, variant: int = 0, stream=None) -> Handle:
    """pars3_split with the canonical split computed on the GPU: rowptr / col /
    perm are int32 CUDA tensors, val a float64 CUDA tensor."""
    import torch
    for t, what, dt in ((rowptr, "rowptr", torch.int32), (col, "col", torch.int32), (val, "val", torch.float64)):
        if t.dtype != dt:
            raise ValueError(f"{what} must be {dt}")
    if perm is not None and perm.dtype != torch.int32:
        raise ValueError("perm must be int32")
    if rowptr.numel() != int(n) + 1:
        raise ValueError("rowptr must hold n + 1 entries")
    prm = pars3_split_params(T=T, W=W, dtypes=dtypes, long_row=long_row,
                             flags=SPLIT_SYMMETRIC if symmetric else 0, piece=piece, long_slices=long_slices,
                             lane_bytes=lane_bytes, variant=variant)
    out = C.c_void_p()
    nz = lambda t: _dptr(t) if t is not None and t.numel() else None
    _chk(lib().pars3_split_device(int(n), _dptr(rowptr), nz(col), nz(val), nz(perm), C.byref(prm), C.byref(out),
                                  _stream(stream)), "pars3_split_device")
    return Handle(out, n)


def pars3_split_export(h: Handle) -> dict:
    c = pars3_canonical()
    _chk(lib().pars3_split_export(h, C.byref(c)), "pars3_split_export")
    nnz, n, nt = c.nnz, c.n, c.ntiles
    nmid = int(c.counts[0] + c.counts[1])
    nout = int(c.counts[2])

    def arr(ptr, m, dt):
        if m == 0:
            return np.zeros(0, dtype=dt)
        return np.ctypeslib.as_array(ptr, shape=(m,)).astype(dt, copy=True)

    return dict(n=n, T=c.T, W=c.W, ntiles=nt, nnz=nnz, counts=np.array(list(c.counts), dtype=np.int64),
                perm=arr(c.perm, n, np.int32), rowptr=arr(c.rowptr, n + 1, np.int32),
                col=arr(c.col, nnz, np.int32), val=arr(c.val, nnz, np.float64),
                cls=arr(c.cls, nnz, np.uint8), tile_ptr=arr(c.tile_ptr, nt + 1, np.int32),
                tile_list=arr(c.tile_list, nmid, np.int32), outer_csr=arr(c.outer_csr, nout, np.int32),
                outer_csc=arr(c.outer_csc, nout, np.int32))


def pars3_layout_digest(h: Handle) -> int:
    d = C.c_uint64()
    _chk(lib().pars3_layout_digest(h, C.byref(d)), "pars3_layout_digest")
    return d.value


def pars3_info_get(h: Handle) -> dict:
    i = pars3_info()
    _chk(lib().pars3_info_get(h, C.byref(i)), "pars3_info_get")
    return i.as_dict()


def pars3_layout_check(h: Handle) -> int:
    return int(lib().pars3_layout_check(h))


# -------------------------------------------------------------- device calls

def pars3_upload(h: Handle, stream=None):
    _chk(lib().pars3_upload(h, _stream(stream)), "pars3_upload")


def pars3_spmv(h: Handle, dtype: int, alpha: float, x, y, stream=None):
    _chk(lib().pars3_spmv(h, int(dtype), float(alpha), _vec(x, dtype, h.n, "x"), _vec(y, dtype, h.n, "y"),
                          _stream(stream)), "pars3_spmv")


def pars3_spmv_noalloc(h: Handle, dtype: int, alpha: float, x, y, stream=None):
    """pars3_spmv with its scratch in the library's fixed device array (the call allocates nothing)."""
    _chk(lib().pars3_spmv_noalloc(h, int(dtype), float(alpha), _vec(x, dtype, h.n, "x"), _vec(y, dtype, h.n, "y"),
                                  _stream(stream)),
         "pars3_spmv_noalloc")


def pars3_spmm(h: Handle, dtype: int, alpha: float, X, Y, stream=None):
    k = 1 if X.dim() == 1 else int(X.shape[1])
    if Y.shape != X.shape:
        raise ValueError(f"Y: expected shape {tuple(X.shape)}, got {tuple(Y.shape)}")
    _chk(lib().pars3_spmm(h, int(dtype), float(alpha), k, _vec(X, dtype, h.n, "X"), _vec(Y, dtype, h.n, "Y"),
                          _stream(stream)), "pars3_spmm")


def pars3_spmm_batched(hs, dtype: int, alphas, Xs, Ys, capture: bool = False, stream=None):
    m = len(hs)
    k = 1 if Xs[0].dim() == 1 else int(Xs[0].shape[1])
    harr = (C.c_void_p * m)(*[h.ptr for h in hs])
    a = np.ascontiguousarray(alphas, dtype=np.float64)
    if not (len(Xs) == len(Ys) == len(alphas) == m):
        raise ValueError("hs, alphas, Xs and Ys must have the same length")
    for h, X, Y in zip(hs, Xs, Ys):
        kk = 1 if X.dim() == 1 else int(X.shape[1])
        if kk != k or Y.shape != X.shape:
            raise ValueError("every X and Y of a batch must have the batch's k columns")
        _vec(X, dtype, h.n, "X")
        _vec(Y, dtype, h.n, "Y")
    xa = (C.c_void_p * m)(*[X.data_ptr() for X in Xs])
    ya = (C.c_void_p * m)(*[Y.data_ptr() for Y in Ys])
    _chk(lib().pars3_spmm_batched(harr, m, int(dtype), _p(a), k, xa, ya, 1 if capture else 0, _stream(stream)),
         "pars3_spmm_batched")


def pars3_permute(h: Handle, dtype: int, src, dst, stream=None):
    k = 1 if src.dim() == 1 else int(src.shape[1])
    _chk(lib().pars3_permute(h, int(dtype), k, _vec(src, dtype, h.n, "src"), _vec(dst, dtype, h.n, "dst"),
                             _stream(stream)), "pars3_permute")


def pars3_unpermute(h: Handle, dtype: int, src, dst, stream=None):
    k = 1 if src.dim() == 1 else int(src.shape[1])
    _chk(lib().pars3_unpermute(h, int(dtype), k, _vec(src, dtype, h.n, "src"), _vec(dst, dtype, h.n, "dst"),
                               _stream(stream)), "pars3_unpermute")


def pars3_spmv_host(h: Handle, dtype: int, alpha: float, x_host: np.ndarray, y_host: np.ndarray, stream=None):
    """x_host/y_host: numpy (or pinned torch CPU tensors' numpy views), original numbering."""
    want = np.float64 if int(dtype) == F64 else np.float32
    for a, what in ((x_host, "x_host"), (y_host, "y_host")):
        if a.dtype != want or a.size != h.n or not a.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{what}: expected {h.n} contiguous {np.dtype(want).name} values")
    _chk(lib().pars3_spmv_host(h, int(dtype), float(alpha), C.c_void_p(x_host.ctypes.data),
                               C.c_void_p(y_host.ctypes.data), _stream(stream)), "pars3_spmv_host")


def pars3_check(h: Handle, stream=None):
    _chk(lib().pars3_check(h, _stream(stream)), "pars3_check")


def pars3_mrs(h: Handle, alpha: float, b, x, rtol: float = 1e-10, max_iter: int = 200000,
              inner: int = F64, inner_rtol: float = 1e-5, max_outer: int = 50, check_every: int = 8,
              stream=None, raise_on_noconv: bool = True) -> dict:
    o = pars3_mrs_opts(rtol=rtol, max_iter=max_iter, inner=inner, inner_rtol=inner_rtol,
                       max_outer=max_outer, check_every=check_every)
    r = pars3_mrs_result()
    rc = lib().pars3_mrs(h, float(alpha), _vec(b, F64, h.n, "b"), _vec(x, F64, h.n, "x"), C.byref(o), C.byref(r),
                         _stream(stream))
    if rc != OK and not (rc == ENOCONV and not raise_on_noconv):
        raise Pars3Error(rc, "pars3_mrs")
    return r.as_dict()


SPLIT_KEYS = ("T", "W", "dtypes", "long_row", "piece", "long_slices", "lane_bytes", "variant")


def pars3_autotune(n: int, rowptr, col, val, perm=None, dtype: int = F64, k: int = 1, dtypes: int = 0,
                   T: int = 0, W: int = 0, long_row: int = 0, symmetric: bool = False):
    """Split parameters chosen by timing pars3_spmm with k right-hand sides on
    the current device; returns a dict of SPLIT_KEYS plus the time "us".
    Pass it on with split_kwargs(result) to pars3_split."""
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(col, dtype=np.int32)
    v = np.ascontiguousarray(val, dtype=np.float64)
    pm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
    base = pars3_split_params(T=T, W=W, dtypes=dtypes, long_row=long_row,
                              flags=SPLIT_SYMMETRIC if symmetric else 0)
    best = pars3_split_params()
    us = C.c_double()
    _chk(lib().pars3_autotune(int(n), _p(rp), _p(ci), _p(v), None if pm is None else _p(pm), C.byref(base),
                              int(dtype), int(k), C.byref(best), C.byref(us)), "pars3_autotune")
    out = {key: getattr(best, key) for key in SPLIT_KEYS}
    out["us"] = us.value
    return out


def split_kwargs(tuned: dict) -> dict:
    """The pars3_split keyword arguments of an autotune result."""
    return {key: tuned[key] for key in SPLIT_KEYS}


def pars3_fp64_fma_rate(stream=None) -> float:
    """fp64 FMAs per second of the current device (measurement helper)."""
    r = C.c_double()
    _chk(lib().pars3_fp64_fma_rate(C.byref(r), _stream(stream)), "pars3_fp64_fma_rate")
    return r.value


def pars3_free(h: Handle):
    h.close()
