#!/usr/bin/env python
"""Benchmark of the GB300 skew SpMV (and the MRS solver) -- one JSON line.

Workload (default): the largest configuration, an R-MAT graph of scale 22
(n = 4,194,304, 20,000,000 stored lower entries, power-law degrees), values
U(-1,1), alpha = 0, x ~ N(0,1); one reorder + autotuned split, then a step
= 200 repeated y = (alpha I + S) x through pars3_spmv, inputs resident in
HBM.  Metric: effective skew-SpMV GB/s = algorithmic bytes (half storage:
nnz*(value+4) + (n+1)*4 + 2*n*vector bytes) per product / time.  The other
workloads (the 128^3 + 1% grid, the band-friendly and finite-element-like
matrices, the batched set) and the MRS comparison on the 128^3 + 1% matrix
are reported in the same line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica (the method
has no exchange step on one matrix per GPU); value = products of all ranks /
max time.  --impl reference times the FP64 CPU oracle (the plain full-storage
row-sum SpMV) on rank 0 on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "skew-SpMV GB/s (% HBM peak); mixed-prec MRS time-to-1e-10 vs FP64 MRS"
REPEATS = 200
L2_FLUSH_BYTES = 512 << 20
FALLBACK_HBM_GBS = 6800.0


def alg_bytes(n: int, nnz: int, sv: int, sx: int, k: int = 1) -> int:
    """Half-storage algorithmic bytes of one product: every stored lower entry
    once (value + 4-byte column), the row pointers, x read once, y written once."""
    return nnz * (sv + 4) + (n + 1) * 4 + 2 * n * sx * k


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", FALLBACK_HBM_GBS)), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """nvidia-smi sampling (100 ms); only samples stamped inside the timed
    region [mark_begin, mark_end] are summarised."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self.t_begin = self.t_end = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t0 = time.time()   # wait for the sampler's first line (up to 5 s)
        while time.time() - t0 < 5.0 and os.path.getsize(self.path) == 0:
            time.sleep(0.05)

    def mark_begin(self):
        self.t_begin = time.time()

    def mark_end(self):
        self.t_end = time.time()

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        import datetime
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [c.strip() for c in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                smv, mxv = float(f[2]), float(f[3])
            except ValueError:
                continue
            if self.t_begin is not None and not (self.t_begin - 0.05 <= ts <= (self.t_end or ts) + 0.05):
                continue
            sm.append(smv)
            mx.append(mxv)
            for nm, v in zip(names, f[6:10]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v: float) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(name: str):
    import workloads as W
    if name == "cfg1":
        A, alpha, x = W.config1()
        desc = "grid3d 128^3 + 1% random long-range edges, N(0,1) values, alpha=0.5, 200 repeated SpMVs"
    elif name == "cfg2":
        A, alpha, x = W.config2()
        desc = "R-MAT scale 22 (a,b,c,d=.57,.19,.19,.05), 20M stored, U(-1,1) values, alpha=0"
    elif name == "cfg0":
        A, alpha, x = W.config0()
        desc = "grid2d 200x100, U(-1,1) values, alpha=0"
    elif name == "grid2d":
        A = W.grid((2048, 1024), "normal", W.SEED_BASE + 5, name="grid2d_2048x1024")
        alpha, x = 0.5, W.vector("uniform", A.n, W.SEED_BASE + 5)
        desc = "grid2d 2048x1024 (band-friendly: RCM bandwidth ~1024), N(0,1), alpha=0.5"
    else:
        raise SystemExit(f"unknown workload {name}")
    return A, alpha, x, desc


def time_products(P, torch, h, dt, alpha, xp, y, flush, reps=50, groups=5):
    """Median microseconds per product over `groups` groups of `reps`
    products, L2 flushed before every group."""
    st = torch.cuda.current_stream()
    for _ in range(3):
        P.pars3_spmv(h, dt, alpha, xp, y, st)
    ts = []
    for _ in range(groups):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            P.pars3_spmv(h, dt, alpha, xp, y, st)
        e1.record(st)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) * 1e3 / reps)
    return statistics.median(ts)


def extra_section(args, peak):
    """The other workloads, each reported beside the headline: a
    band-friendly 2D grid (2048 x 1024, RCM bandwidth about 1024: the
    half-storage middle band holds the matrix), the headline matrix as a
    symmetric operator, the R-MAT matrix in FP64 and
    FP32 (cut points from pars3_autotune), and the batched workload (64
    uneven grids, k in {1, 4, 16, 32}, FP32 and FP64, one persistent launch
    replayed from a CUDA graph, cut points from pars3_autotune per matrix)."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2407_17651_gb300 import pars3 as P
    out = {}
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    both = P.dtype_bit(P.F64) | P.dtype_bit(P.F32)

    def single(name, A, alpha, x, desc, symmetric=False, precisions=("f64", "f32"), reorder_flags=P.RCM_GUARD):
        """Split parameters autotuned separately for each precision."""
        t0 = time.perf_counter()
        perm, bw0, bw1 = P.pars3_reorder(A.n, A.rowptr, A.col, reorder_flags)
        t_rcm = time.perf_counter() - t0
        row = {"workload": desc, "n": A.n, "nnz_stored": A.nnz, "alpha": alpha, "rcm_bandwidth": bw1,
               "rcm_s": t_rcm}
        for dt, nm, vt, sv, sx in ((P.F64, "f64", torch.float64, 8, 8), (P.F32, "f32", torch.float32, 4, 4)):
            if nm not in precisions:
                continue
            t0 = time.perf_counter()
            tune = P.pars3_autotune(A.n, A.rowptr, A.col, A.val, perm, dtype=dt, k=1, dtypes=P.dtype_bit(dt),
                                    symmetric=symmetric)
            t_tune = time.perf_counter() - t0
            h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, symmetric=symmetric, **P.split_kwargs(tune))
            P.pars3_upload(h)
            info = P.pars3_info_get(h)
            xp = torch.from_numpy(x[perm]).to("cuda", vt)
            y = torch.empty_like(xp)
            us = time_products(P, torch, h, dt, alpha, xp, y, flush)
            P.pars3_check(h)
            ub = alg_bytes(A.n, A.nnz, sv, sx)
            lb = info["bytes_per_spmv"][dt]
            row[nm] = {"us": us, "GBps": ub / us / 1e3, "frac_of_peak": ub / us / 1e3 / peak,
                       "layout_GBps": lb / us / 1e3, "GFLOPs": (4 * A.nnz + (2 * A.n if alpha else 0)) / us / 1e3,
                       "T": info["T"], "W": info["W"], "half_entries": info["half_entries"],
                       "full_entries": info["full_entries"], "long_entries": info["long_entries"],
                       "split_params": P.split_kwargs(tune), "autotune_s": t_tune}
            h.close()
        out[name] = row

    t0 = time.perf_counter()
    A, alpha, x = W.config0()
    single("cfg0", A, alpha, x, "grid2d 200x100 (n = 20,000), U(-1,1), alpha=0 (small: latency-bound, report us)")
    out["cfg0"]["section_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    A = W.grid((2048, 1024), "normal", W.SEED_BASE + 5, name="grid2d_2048x1024")
    single("grid2d", A, 0.5, W.vector("uniform", A.n, W.SEED_BASE + 5),
           "grid2d 2048x1024 (band-friendly: RCM bandwidth ~1024), N(0,1), alpha=0.5")
    out["grid2d"]["section_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    A = W.fem_grid2d(256, 512, 4, "normal", W.SEED_BASE + 6)
    single("fem_like", A, 0.5, W.vector("uniform", A.n, W.SEED_BASE + 6),
           "finite-element-like pattern shaped like the paper's Table 1 matrices: 256 x 512 nodes, 4 unknowns "
           "each, 9-point coupling (n = 524,288, 34.9 entries per full row, RCM bandwidth 2047), alpha=0.5")
    out["fem_like"]["section_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    A, alpha, x = W.config1()
    single("cfg1", A, alpha, x, "grid3d 128^3 + 1% random long-range edges, N(0,1), alpha=0.5")
    out["cfg1"]["section_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    single("cfg1_local_rcm", A, alpha, x, "the 128^3 + 1% matrix ordered by the RCM of its local edges "
           "(PARS3_RCM_LOCAL: the random long-range edges do not steer the ordering), alpha=0.5",
           reorder_flags=P.RCM_GUARD | P.RCM_LOCAL)
    out["cfg1_local_rcm"]["section_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    single("cfg1_symmetric", A, alpha, x, "the 128^3 + 1% matrix as the symmetric S = L + L^T "
           "(PARS3_SPLIT_SYMMETRIC), alpha=0.5", symmetric=True)
    out["cfg1_symmetric"]["section_s"] = time.perf_counter() - t0
    if args.workload != "cfg2" or args.dtype != "f32":
        t0 = time.perf_counter()
        A, alpha, x = W.config2()
        single("cfg2", A, alpha, x, "R-MAT scale 22, 20M stored, U(-1,1), alpha=0, split parameters autotuned",
               precisions=("f32",) if args.workload == "cfg2" else ("f64", "f32"))
        out["cfg2"]["section_s"] = time.perf_counter() - t0
    del A, x

    # batched uneven workload
    t0 = time.perf_counter()
    shapes = W.config4_shapes()
    mats = [W.config4_matrix(m, shp) for m, shp in enumerate(shapes)]
    prep = {"generate": time.perf_counter() - t0}
    # RCM of all 64 matrices in one GPU call (pars3_reorder_device_batched),
    # timed after a first call; the host ordering is timed beside it
    pats = [(A.n, torch.from_numpy(A.rowptr).cuda(), torch.from_numpy(A.col).cuda()) for A in mats]
    P.pars3_reorder_device_batched(pats)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    outs = P.pars3_reorder_device_batched(pats)
    torch.cuda.synchronize()
    prep["rcm_device_batched"] = time.perf_counter() - t1
    perms = [p.cpu().numpy() for p, _, _ in outs]
    t1 = time.perf_counter()
    host_perms = [P.pars3_reorder(A.n, A.rowptr, A.col)[0] for A in mats]
    prep["rcm_host"] = time.perf_counter() - t1
    prep["rcm_device_same_as_host"] = all(np.array_equal(a, b) for a, b in zip(perms, host_perms))
    del host_perms
    # split parameters from the autotuner; the handles the products run on come
    # from the GPU split (pars3_split_device), the host split is timed beside it
    hs, ns, nnzs, cuts = [], [], [], []
    prep["autotune"] = prep["split_device"] = prep["split_host"] = prep["upload"] = 0.0
    same = True
    for A, perm, (_, rp_d, ci_d), (perm_d, _, _) in zip(mats, perms, pats, outs):
        t1 = time.perf_counter()
        tune = P.pars3_autotune(A.n, A.rowptr, A.col, A.val, perm, dtype=P.F32, k=4, dtypes=both)
        kw = P.split_kwargs(tune)
        val_d = torch.from_numpy(A.val).cuda()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        h = P.pars3_split_device(A.n, rp_d, ci_d, val_d, perm_d, **kw)
        t3 = time.perf_counter()
        hh = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, **kw)
        t4 = time.perf_counter()
        ed, eh = P.pars3_split_export(h), P.pars3_split_export(hh)
        same = same and all(np.array_equal(np.asarray(ed[k]), np.asarray(eh[k])) for k in ed)
        hh.close()
        del val_d
        t5 = time.perf_counter()
        P.pars3_upload(h)
        prep["autotune"] += t2 - t1
        prep["split_device"] += t3 - t2
        prep["split_host"] += t4 - t3
        prep["upload"] += time.perf_counter() - t5
        hs.append(h); ns.append(A.n); nnzs.append(A.nnz); cuts.append((tune["T"], tune["W"], tune["lane_bytes"]))
    prep["split_device_same_as_host"] = same
    del mats, pats, outs
    t_prep = time.perf_counter() - t0
    rows = {}
    st = torch.cuda.current_stream()
    for dt, nm, vt, sv, sx in ((P.F32, "f32", torch.float32, 4, 4), (P.F64, "f64", torch.float64, 8, 8)):
        for k in W.CONFIG4_KS:
            Xs, Ys = [], []
            for m, h in enumerate(hs):
                X = W.config4_rhs(ns[m], k, m)[perms[m]]
                X = X[:, 0] if k == 1 else X
                Xs.append(torch.from_numpy(np.ascontiguousarray(X)).to("cuda", vt))
                Ys.append(torch.empty_like(Xs[-1]))
            alphas = [1.0] * len(hs)
            for _ in range(3):
                P.pars3_spmm_batched(hs, dt, alphas, Xs, Ys, capture=True, stream=st)
            ts = []
            for _ in range(5):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                for _ in range(10):
                    P.pars3_spmm_batched(hs, dt, alphas, Xs, Ys, capture=True, stream=st)
                e1.record(st)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1) * 1e3 / 10)
            us = statistics.median(ts)
            ub = sum(alg_bytes(n, z, sv, sx, k) for n, z in zip(ns, nnzs))
            rows[f"{nm}_k{k}"] = {"us": us, "GBps": ub / us / 1e3, "frac_of_peak": ub / us / 1e3 / peak,
                                  "GFLOPs": sum(4 * z * k + 2 * n * k for n, z in zip(ns, nnzs)) / us / 1e3}
            del Xs, Ys
    for h in hs:
        h.close()
    out["cfg4"] = {"workload": "64 uneven grids (n log-uniform in [1e4, 5e5], 2D/3D), N(0,1), alpha=1, "
                               "one persistent launch + fold per call, replayed from a CUDA graph",
                   "sum_n": sum(ns), "sum_nnz_stored": sum(nnzs), "prep_s": t_prep, "prep_breakdown_s": prep,
                   "cut_points_T_W_lane_bytes": sorted(set(cuts)), "results": rows,
                   "section_s": time.perf_counter() - t0}
    return out


def run_reference(args, ws, rank):
    """Oracle arm: FP64 full-storage row-sum SpMV (plain C, one thread)."""
    if rank != 0:
        return
    import numpy as np
    import oracle as O
    A, alpha, x, desc = workload(args.workload)
    F = O.Full(A)
    unit_bytes = alg_bytes(A.n, A.nnz, 8, 8)
    F.apply(alpha, x)
    per_step = max(1, args.ref_spmvs)
    for _ in range(args.warmup):
        F.apply(alpha, x)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for _ in range(per_step):
            F.apply(alpha, x)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    gbs = unit_bytes * per_step * args.steps / tot / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {desc}", "n": A.n, "nnz_stored": A.nnz,
                       "sample": f"{per_step} SpMVs per step (of the {REPEATS}-product step)"},
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": f"{per_step * args.steps} full-storage SpMVs of the whole matrix"},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(A, alpha, x, budget_s: float):
    """The oracle on one host core: its full-storage row-sum SpMV (the
    value) and the paper's serial SSS pair-update SpMV (Sec. 3.1.1, the
    denominator of the paper's speedups), each on a bounded sample."""
    import oracle as O
    F = O.Full(A)
    F.apply(alpha, x)

    def timed(fn, budget):
        t0 = time.perf_counter()
        cnt = 0
        while True:
            fn()
            cnt += 1
            el = time.perf_counter() - t0
            if el >= budget or cnt >= REPEATS:
                return cnt, el

    cnt, el = timed(lambda: F.apply(alpha, x), budget_s)
    ub = alg_bytes(A.n, A.nnz, 8, 8)
    c2, e2 = timed(lambda: O.spmv_sss(A, alpha, x), max(budget_s / 4, 0.05))
    return {"value": ub * cnt / el / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"{cnt} full-storage fp64 SpMVs of the whole matrix ({el:.1f} s, single thread)",
            "serial_sss": {"value": ub * c2 / e2 / 1e9, "unit": "GB/s", "us_per_product": 1e6 * e2 / c2,
                           "sample": f"{c2} serial SSS pair-update SpMVs (Sec. 3.1.1), single thread"},
            "all_cores": all_cores_baseline(F, alpha, x, ub, max(budget_s / 2, 0.05))}


def all_cores_baseline(F, alpha, x, unit_bytes: int, budget_s: float):
    """The same single-threaded oracle product run as independent replicas,
    one host thread per core the process may use, all sharing the matrix
    (the C call releases the interpreter lock, so the replicas run in
    parallel): aggregate products per second x algorithmic bytes."""
    import threading
    cores = len(os.sched_getaffinity(0))
    counts = [0] * cores
    go = threading.Barrier(cores + 1)

    def replica(i):
        go.wait()
        t0 = time.perf_counter()
        while True:
            F.apply(alpha, x)
            counts[i] += 1
            if time.perf_counter() - t0 >= budget_s or counts[i] >= REPEATS:
                return

    threads = [threading.Thread(target=replica, args=(i,)) for i in range(cores)]
    for t in threads:
        t.start()
    go.wait()
    t0 = time.perf_counter()
    for t in threads:
        t.join()
    el = time.perf_counter() - t0
    tot = sum(counts)
    return {"value": unit_bytes * tot / el / 1e9, "unit": "GB/s", "cores": cores,
            "sample": f"{tot} full-storage fp64 SpMVs of the whole matrix by {cores} single-threaded "
                      f"replicas ({el:.1f} s)"}


MRS_CUT = (2048, 32)   # the cut the autotuner picks for the 128^3 + 1% matrix in fp64


def mrs_section(alphas, budget_iters: int):
    """Configuration 3: (alpha I + S) x = b on the configuration-1 matrix,
    time to a true relative residual of 1e-10: plain fp64 MRS against an
    fp32 / bf16-value inner MRS inside fp64 refinement (wall time of one
    pars3_mrs call, graph capture done by an untimed warm-up solve)."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2407_17651_gb300 import pars3 as P
    A, _, _ = W.config1()
    perm = P.pars3_reorder(A.n, A.rowptr, A.col)[0]
    T, Wc = MRS_CUT
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, T=T, W=Wc,
                      dtypes=P.dtype_bit(P.F64) | P.dtype_bit(P.F32) | P.dtype_bit(P.BF16))
    P.pars3_upload(h)
    b = torch.from_numpy(W.config3_rhs(A.n)[perm]).cuda()
    x = torch.zeros_like(b)
    inner_rtol = {P.F64: 0.0, P.F32: 1e-4, P.BF16: 1e-2}
    names = {P.F64: "fp64", P.F32: "fp32-ir", P.BF16: "bf16-ir"}
    for inner in (P.F64, P.F32, P.BF16):   # capture the loops
        x.zero_()
        P.pars3_mrs(h, 1.0, b, x, rtol=1e-10, inner=inner, inner_rtol=inner_rtol[inner], max_iter=5,
                    raise_on_noconv=False)
    out = {}
    for alpha in alphas:
        row = {}
        for inner in (P.F64, P.F32, P.BF16):
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = P.pars3_mrs(h, alpha, b, x, rtol=1e-10, inner=inner, inner_rtol=inner_rtol[inner],
                            max_iter=budget_iters, max_outer=40, raise_on_noconv=False)
            el = time.perf_counter() - t0
            row[names[inner]] = {"time_s": el, "iters": r["iters"], "outer": r["outer"],
                                 "true_relres": r["true_relres"], "converged": r["status"] == 0,
                                 "inner_rtol": inner_rtol[inner] or None}
        t64 = row["fp64"]["time_s"]
        for k in ("fp32-ir", "bf16-ir"):
            row[k]["speedup_vs_fp64"] = (t64 / row[k]["time_s"]) if row[k]["converged"] and row["fp64"]["converged"] else None
        out[str(alpha)] = row
    h.close()
    return out


def mrs_summary(mrs):
    """Seconds to a true relative residual of 1e-10 per alpha and precision,
    and the mixed-precision speedups, compactly (kept at the end of the line)."""
    if not mrs:
        return None
    out = {}
    for a, row in mrs.items():
        out[a] = {"fp64_s": round(row["fp64"]["time_s"], 5), "fp32_ir_s": round(row["fp32-ir"]["time_s"], 5),
                  "bf16_ir_s": round(row["bf16-ir"]["time_s"], 5),
                  "speedup_fp32_ir": row["fp32-ir"].get("speedup_vs_fp64"),
                  "speedup_bf16_ir": row["bf16-ir"].get("speedup_vs_fp64"),
                  "max_true_relres": max(row[k]["true_relres"] for k in ("fp64", "fp32-ir", "bf16-ir")),
                  "all_converged": all(row[k]["converged"] for k in ("fp64", "fp32-ir", "bf16-ir"))}
    return out


def traffic_from_profile(key: str, kernel_hash: str, split_kw: dict, layout_bytes: int):
    """DRAM bytes per launch from the committed ncu summary of `key`, if it
    was taken on the current kernel source with the same split parameters, or
    with parameters (the autotuner's choice may differ from run to run) whose
    layout streams the same bytes within 2 %."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    ent = d.get(key)
    if not ent or ent.get("source_hash") != kernel_hash:
        return None
    if ent.get("split_params") not in (None, split_kw):
        lb = ent.get("layout_bytes_per_launch")
        if not lb or abs(layout_bytes - lb) > 0.02 * lb:
            return None
    return float(ent["dram_bytes_per_launch"])


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("spmv_kernels.cuh", "spmv.cu", "devcommon.cuh", "smem_layout.h", "host_split.cpp", "internal.h",
              "autotune.cu"):
        h.update(open(os.path.join(ROOT, "paper_2407_17651_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cfg2")
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32", "bf16"])
    ap.add_argument("--k", type=int, default=1, help="right-hand sides (k > 1 times pars3_spmm on an n x k block)")
    ap.add_argument("--T", type=int, default=-1, help="tile rows (default: pars3_autotune)")
    ap.add_argument("--W", type=int, default=-1, help="middle bandwidth (with --T)")
    ap.add_argument("--split", default="", help="split parameters as JSON (the keys of an autotune result); "
                                                "skips the autotuner, e.g. to profile a known choice")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--ref-spmvs", type=int, default=10)
    ap.add_argument("--mrs", default="1,0.1,0.01", help="alphas of the MRS comparison ('' to skip)")
    ap.add_argument("--mrs-iters", type=int, default=60000)
    ap.add_argument("--extra", type=int, default=1, help="1: also report the band-friendly grid, R-MAT and batched workloads")
    args = ap.parse_args()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    import numpy as np
    import torch
    from paper_2407_17651_gb300 import _build
    from paper_2407_17651_gb300 import pars3 as P

    if rank == 0 or ws == 1:
        _build.build()
    barrier(ws)
    torch.cuda.set_device(local)
    dt = {"f64": P.F64, "f32": P.F32, "bf16": P.BF16}[args.dtype]
    vt = torch.float64 if dt == P.F64 else torch.float32
    sv = {P.F64: 8, P.F32: 4, P.BF16: 2}[dt]
    sx = 8 if dt == P.F64 else 4

    A, alpha, x, desc = workload(args.workload)
    t0 = time.perf_counter()
    perm, bw0, bw1 = P.pars3_reorder(A.n, A.rowptr, A.col)
    t_rcm = time.perf_counter() - t0
    # the same ordering on the GPU (pars3_reorder_device), timed after a first call
    rp_d, ci_d = torch.from_numpy(A.rowptr).cuda(), torch.from_numpy(A.col).cuda()
    P.pars3_reorder_device(A.n, rp_d, ci_d)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    perm_d = P.pars3_reorder_device(A.n, rp_d, ci_d)[0]
    torch.cuda.synchronize()
    t_rcm_dev = time.perf_counter() - t0
    rcm_dev_same = bool(np.array_equal(perm_d.cpu().numpy(), perm))
    del rp_d, ci_d, perm_d
    t_tune = None
    if args.split:
        split_kw = dict(json.loads(args.split))
        split_kw.setdefault("dtypes", P.dtype_bit(dt))
    elif args.T >= 0:
        split_kw = dict(T=args.T, W=args.W, dtypes=P.dtype_bit(dt))
    else:   # split parameters from the autotuner (untimed preprocessing)
        t0 = time.perf_counter()
        tune = P.pars3_autotune(A.n, A.rowptr, A.col, A.val, perm, dtype=dt, k=max(1, args.k),
                                dtypes=P.dtype_bit(dt))
        t_tune = time.perf_counter() - t0
        split_kw = P.split_kwargs(tune)
    t0 = time.perf_counter()
    h = P.pars3_split(A.n, A.rowptr, A.col, A.val, perm, **split_kw)
    t_split = time.perf_counter() - t0
    # the same split with its canonical part on the GPU (pars3_split_device)
    dev_in = [torch.from_numpy(a).cuda() for a in (A.rowptr, A.col, A.val, perm)]
    P.pars3_split_device(A.n, *dev_in, **split_kw).close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hd = P.pars3_split_device(A.n, *dev_in, **split_kw)
    t_split_dev = time.perf_counter() - t0
    ed, eh = P.pars3_split_export(hd), P.pars3_split_export(h)
    split_dev_same = all(np.array_equal(np.asarray(ed[k]), np.asarray(eh[k])) for k in ed)
    hd.close()
    del dev_in, ed, eh
    t0 = time.perf_counter()
    P.pars3_upload(h)
    t_up = time.perf_counter() - t0
    info = P.pars3_info_get(h)

    k = max(1, args.k)
    if k == 1:
        xp = torch.from_numpy(x[perm]).to("cuda", vt)
    else:   # the workload's x in column 0, further columns from the same generator
        import workloads as W
        Xk = W.vector("uniform", (A.n, k), W.SEED_BASE + 1, stream=91)
        Xk[:, 0] = x
        xp = torch.from_numpy(np.ascontiguousarray(Xk[perm])).to("cuda", vt)
    y = torch.empty_like(xp)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def product():
        if k == 1:
            P.pars3_spmv(h, dt, alpha, xp, y, stream)
        else:
            P.pars3_spmm(h, dt, alpha, xp, y, stream)

    def step(evs=None):
        """200 products.  evs: None, a (start, end) pair around the step, or
        REPEATS + 1 events with one between every two products."""
        per_product = evs is not None and len(evs) > 2
        if evs is not None:
            evs[0].record(stream)
        for r in range(REPEATS):
            if per_product and r > 0:
                evs[r].record(stream)
            product()
        if evs is not None:
            evs[-1].record(stream)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    P.pars3_check(h)

    # two events per step: an event between every two products would add its own gap to the step
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    clocks = Clocks(local)
    clocks.start()
    barrier(ws)
    torch.cuda.synchronize()
    clocks.mark_begin()
    for s in range(args.steps):
        flush.zero_()
        step(evs[s])
    torch.cuda.synchronize()
    clocks.mark_end()
    barrier(ws)
    clk = clocks.stop()
    P.pars3_check(h)
    step_ms = [evs[s][0].elapsed_time(evs[s][1]) for s in range(args.steps)]
    tot_s_local = sum(step_ms) / 1e3
    tot_s = max_over_ranks(ws, tot_s_local)
    # one more (untimed) step with an event between every two products, for
    # the spread of single products
    dev = [torch.cuda.Event(enable_timing=True) for _ in range(REPEATS + 1)]
    flush.zero_()
    step(dev)
    torch.cuda.synchronize()
    spmv_ms = [dev[r].elapsed_time(dev[r + 1]) for r in range(REPEATS)]
    ub = alg_bytes(A.n, A.nnz, sv, sx, k)
    value = ub * REPEATS * args.steps * ws / tot_s / 1e9
    peak, peak_kind = measured_peaks()
    avg_spmv_s = tot_s_local / (REPEATS * args.steps)   # average product (launch) duration, timed region
    achieved = ub / avg_spmv_s / 1e9
    khash = kernel_source_hash()
    traffic = (traffic_from_profile(f"tile_kernel_{args.dtype}_{args.workload}", khash, split_kw,
                                    info["bytes_per_spmv"][dt]) if k == 1 else None)
    # the fp64 products do one FMA per stored entry and direction: measure the
    # device's fp64 FMA rate in the same run (a kernel of independent chains)
    fp64 = None
    if dt == P.F64:
        rate = P.pars3_fp64_fma_rate()
        fmas = (2 * A.nnz + (A.n if alpha else 0)) * k
        fp64 = {"fma_per_launch": fmas, "achieved_fma_per_s": fmas / avg_spmv_s, "peak_fma_per_s": rate,
                "frac": fmas / avg_spmv_s / rate if rate > 0 else None,
                "floor_us": 1e6 * fmas / rate if rate > 0 else None,
                "how": "2 FMA per stored entry (row sum and mirrored sum) plus alpha x; peak from "
                       "pars3_fp64_fma_rate (independent FMA chains on every SM, CUDA events)"}

    # end to end through the host-buffer entry point (original numbering)
    e2e = None
    if args.e2e_steps > 0 and k == 1:
        xh = torch.from_numpy(x.astype(np.float64 if dt == P.F64 else np.float32)).pin_memory().numpy()
        yh = torch.empty(A.n, dtype=vt).pin_memory().numpy()
        P.pars3_spmv_host(h, dt, alpha, xh, yh)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            for _ in range(REPEATS):
                P.pars3_spmv_host(h, dt, alpha, xh, yh)
        el = time.perf_counter() - t0
        el = max_over_ranks(ws, el)
        e2e = {"value": ub * REPEATS * args.e2e_steps * ws / el / 1e9, "unit": "GB/s",
               "h2d_bytes_per_step": REPEATS * A.n * sx, "d2h_bytes_per_step": REPEATS * A.n * sx,
               "api": "pars3_spmv_host (H2D, permute, SpMV, unpermute, D2H, sync per product)"}

    cpu = cpu_baseline(A, alpha, x, args.cpu_budget) if (rank == 0 and ws == 1) else None
    mrs = None
    if args.mrs and k == 1 and rank == 0:
        mrs = mrs_section([float(a) for a in args.mrs.split(",")], args.mrs_iters)
    launches_per_spmv = 1 + (1 if info["halo_targets"] + info["long_rows"] > 0 else 0)
    extra = extra_section(args, peak) if (args.extra and rank == 0) else None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "pct_hbm_peak": value / ws / peak,
            "config": {"workload": f"{args.workload}: {desc}" + (f", k = {k} right-hand sides" if k > 1 else ""),
                       "n": A.n, "nnz_stored": A.nnz, "alpha": alpha, "k": k,
                       "repeats_per_step": REPEATS, "T": info["T"], "W": info["W"],
                       "rcm_bandwidth": bw1, "original_bandwidth": bw0,
                       "half_entries": info["half_entries"], "full_entries": info["full_entries"],
                       "long_rows": info["long_rows"], "halo_targets": info["halo_targets"],
                       "l2": "L2 (126 MB) flushed by a 512 MB write before every step; the matrix "
                             f"({info['bytes_per_spmv'][dt] / 1e6:.0f} MB per product as laid out) exceeds L2; "
                             "x and y stay device-resident across the 200 products as in a Krylov loop",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                         "kernel": ("pars3_spmv: tile kernel" if k == 1 else "pars3_spmm: spmm kernel")
                                   + (" + fold kernel" if launches_per_spmv > 1 else " (one launch per product)")
                                   + "; average duration = CUDA-event time of the timed steps / products",
                         "algorithmic_bytes_per_launch": ub,
                         "layout_bytes_per_launch": info["bytes_per_spmv"][dt],
                         # the DRAM bytes the profile counted, over the same average duration: how
                         # close the kernel's actual traffic runs to the copy ceiling
                         "traffic_GBps": traffic / avg_spmv_s / 1e9 if traffic else None,
                         "traffic_frac": traffic / avg_spmv_s / 1e9 / peak if traffic else None,
                         "hbm_floor_us": 1e6 * ub / (peak * 1e9),
                         "fp64_pipe": fp64},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches_per_spmv * REPEATS * args.steps,
            "mrs": mrs,
            "clocks": clk,
            "preprocess_s": {"rcm": t_rcm, "rcm_device": t_rcm_dev, "rcm_device_same_as_host": rcm_dev_same,
                             "autotune": t_tune, "split": t_split, "split_device": t_split_dev,
                             "split_device_same_as_host": split_dev_same, "upload": t_up},
            "other_workloads": extra,
            "spmv_us": {"mean": 1e6 * avg_spmv_s,
                        "single_products": {"median": 1e3 * statistics.median(spmv_ms), "min": 1e3 * min(spmv_ms),
                                            "max": 1e3 * max(spmv_ms),
                                            "how": "one extra untimed step with an event between every two "
                                                   "products"}},
            "kernel_source_hash": khash,
            "split_params": split_kw,
            "mrs_summary": mrs_summary(mrs),
        }
        print(json.dumps(line), flush=True)
    h.close()


if __name__ == "__main__":
    main()
