// autotune.cu -- pars3_autotune: choose the split parameters by timing
// pars3_spmm on the current device.  First the cut points (T, W) of the
// 3-way split (Sec. 3.1.2: the tile a thread block owns and the middle
// bandwidth), then the layout choices that are this implementation's own.
//
// The search is coordinate-wise, so that a matrix is split at most about
// fifteen times:
//   1. W = 32, T in {512, 1024, 2048, 4096}            -> T1
//   2. T = T1, W in {64, ..., min(T1, w_max)}          -> W2
//   3. W = W2, T in {T1 / 2, 2 T1} not yet timed       -> (T, W)
//   4. matrices with rows of more than 32 full-storage entries: the long-row
//      threshold, piece length and long slices per block, from a short list
//      of measured good settings (power-law rows want shorter tile rows and
//      longer pieces);
//   5. k = 1 with fp32 / bf16 values: the look-ahead tile kernel variant;
//      k > 1: the other lane widths of the multi-vector product.
// w_max is the reordered bandwidth rounded up to a power of two, capped like
// the default rule (1024 with F64 packed, else 2048): a middle band wider
// than the matrix's band holds no more entries.  A candidate replaces the
// incumbent only when it is at least 2 % faster, so near-ties keep the
// earlier (simpler) choice.  Candidates the layout cannot hold (shared
// memory) are skipped.  The matrix is reordered and sorted once, on the GPU
// (the cut-independent stages of pars3_split_device); each candidate re-runs
// only the cut-dependent stages, also on the GPU, is uploaded, timed (3
// warm-up products, then the median of 3 groups of 8 products measured with
// CUDA events) and freed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

using namespace pars3;

namespace {

struct Timer {
    int32_t n = 0, dtype = 0, k = 1;
    DevBase *base = nullptr;   // reordered matrix on the device; candidates re-cut it
    void *X = nullptr, *Y = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;

    // microseconds per product, or +inf when the candidate cannot be laid out
    int time(const pars3_split_params &p, double *us) {
        *us = INFINITY;
        pars3_handle *h = nullptr;
        int rc = devbase_cut(base, p, &h, st);
        if (rc == PARS3_EUNSUPPORTED) return PARS3_OK;
        if (rc != PARS3_OK) return rc;
        rc = pars3_upload(h, st);
        if (rc == PARS3_ENOMEM) {
            pars3_free(h);
            return PARS3_OK;
        }
        std::vector<float> groups;
        for (int it = 0; rc == PARS3_OK && it < 3; ++it) rc = pars3_spmm(h, dtype, 1.0, k, X, Y, st);
        for (int g = 0; rc == PARS3_OK && g < 3; ++g) {
            cudaEventRecord(e0, st);
            for (int it = 0; rc == PARS3_OK && it < 8; ++it) rc = pars3_spmm(h, dtype, 1.0, k, X, Y, st);
            cudaEventRecord(e1, st);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) rc = cuda_status(e);
            float ms = 0.f;
            if (rc == PARS3_OK) {
                e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) rc = cuda_status(e);
            }
            groups.push_back(ms);
        }
        if (rc == PARS3_OK) rc = pars3_check(h, st);
        pars3_free(h);
        if (rc == PARS3_EUNSUPPORTED) return PARS3_OK;
        if (rc != PARS3_OK) return rc;
        std::sort(groups.begin(), groups.end());
        *us = 1e3 * groups[1] / 8.0;
        return PARS3_OK;
    }
};

// longest row of the full-storage (both triangles) pattern: the largest
// vertex degree, which no reordering changes
int64_t max_full_row(int32_t n, const int32_t *rowptr, const int32_t *col) {
    std::vector<int32_t> deg(static_cast<size_t>(n), 0);
    for (int32_t i = 0; i < n; ++i) {
        deg[i] += rowptr[i + 1] - rowptr[i];
        for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) ++deg[col[e]];
    }
    int64_t m = 0;
    for (int32_t d : deg) m = std::max<int64_t>(m, d);
    return m;
}

// the inputs on the device, for building the reordered matrix there
int device_base(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val, const int32_t *perm,
                int symmetric, cudaStream_t st, DevBase **out) {
    const int64_t nnz = rowptr[n];
    int32_t *d_rp = nullptr, *d_ci = nullptr, *d_perm = nullptr;
    double *d_val = nullptr;
    cudaError_t e = cudaMalloc(&d_rp, sizeof(int32_t) * (n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&d_ci, sizeof(int32_t) * std::max<int64_t>(1, nnz));
    if (e == cudaSuccess) e = cudaMalloc(&d_val, sizeof(double) * std::max<int64_t>(1, nnz));
    if (e == cudaSuccess && perm) e = cudaMalloc(&d_perm, sizeof(int32_t) * std::max(1, n));
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_rp, rowptr, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(d_ci, col, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(d_val, val, sizeof(double) * nnz, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && perm) e = cudaMemcpyAsync(d_perm, perm, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st);
    int rc = cuda_status(e);
    if (rc == PARS3_OK) rc = devbase_create(n, d_rp, d_ci, d_val, d_perm, symmetric, out, st);
    cudaStreamSynchronize(st);
    cudaFree(d_rp);
    cudaFree(d_ci);
    cudaFree(d_val);
    if (d_perm) cudaFree(d_perm);
    return rc;
}

int32_t pow2_ceil(int64_t v) {
    int32_t p = 32;
    while (p < v && p < (1 << 15)) p <<= 1;
    return p;
}

}  // namespace

extern "C" int pars3_autotune(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                              const int32_t *perm, const pars3_split_params *base, int32_t dtype, int32_t k,
                              pars3_split_params *best, double *best_us) {
    if (!best || n < 0 || !rowptr || k < 1 || k > 32 || dtype < 0 || dtype >= kNumDtypes) return PARS3_EINVAL;
    int rc = validate_lower(n, rowptr, col);
    if (rc != PARS3_OK) return rc;
    Timer tm;
    tm.n = n;
    tm.dtype = dtype;
    tm.k = k;
    pars3_split_params b0{};
    if (base) b0 = *base;
    if (b0.dtypes == 0) b0.dtypes = PARS3_DTYPE_BIT(PARS3_F64);
    if (check_layout_params(b0) != PARS3_OK) return PARS3_EINVAL;
    // the long-row stage only searches when the caller left those settings at their defaults
    const bool base_layout_default = b0.long_row == 0 && b0.piece == 0 && b0.long_slices == 0;
    b0.dtypes |= PARS3_DTYPE_BIT(dtype);
    *best = b0;
    if (best_us) *best_us = 0.0;
    if (n == 0) {
        best->T = 1024;
        best->W = 32;
        return PARS3_OK;
    }

    if (rowptr[n] > 0 && !val) return PARS3_EINVAL;
    if ((b0.flags & ~PARS3_SPLIT_SYMMETRIC) || (b0.dtypes & ~7)) return PARS3_EINVAL;
    const int32_t wcap = (b0.dtypes & PARS3_DTYPE_BIT(PARS3_F64)) ? 1024 : 2048;
    cudaError_t e = cudaStreamCreateWithFlags(&tm.st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_status(e);
    rc = device_base(n, rowptr, col, val, perm, (b0.flags & PARS3_SPLIT_SYMMETRIC) ? 1 : 0, tm.st, &tm.base);
    if (rc != PARS3_OK) {
        cudaStreamDestroy(tm.st);
        return rc;
    }
    const int32_t wmax = std::min(pow2_ceil(devbase_bandwidth(tm.base)), wcap);

    const size_t vsz = dtype == PARS3_F64 ? 8 : 4;
    const size_t bytes = std::max<size_t>(16, static_cast<size_t>(n) * k * vsz);
    e = cudaMalloc(&tm.X, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&tm.Y, bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(tm.X, 0, bytes, tm.st);
    if (e == cudaSuccess) e = cudaEventCreate(&tm.e0);
    if (e == cudaSuccess) e = cudaEventCreate(&tm.e1);
    rc = cuda_status(e);

    std::vector<pars3_split_params> tried;
    pars3_split_params bp = b0;
    bp.T = 0;
    double bus = INFINITY;
    auto same = [](const pars3_split_params &x, const pars3_split_params &y) {
        return x.T == y.T && x.W == y.W && x.long_row == y.long_row && x.piece == y.piece &&
               x.long_slices == y.long_slices && x.lane_bytes == y.lane_bytes && x.variant == y.variant;
    };
    auto consider = [&](const pars3_split_params &c) {
        if (rc != PARS3_OK || c.W > c.T || c.T > 32768) return;
        for (auto &t : tried)
            if (same(t, c)) return;
        tried.push_back(c);
        double us;
        rc = tm.time(c, &us);
        if (rc == PARS3_OK && us < 0.98 * bus) {
            bus = us;
            bp = c;
        }
    };
    auto cut = [&](int32_t T, int32_t W) {
        pars3_split_params c = bp.T > 0 ? bp : b0;
        c.T = T;
        c.W = W;
        consider(c);
    };
    for (int32_t T : {512, 1024, 2048, 4096}) cut(T, 32);
    const int32_t T1 = bp.T;
    if (T1 > 0)
        for (int32_t W = 64; W <= std::min(T1, wmax); W <<= 1) cut(T1, W);
    if (T1 > 0) {
        const int32_t W2 = bp.W;
        cut(std::max(T1 / 2, W2), W2);
        cut(T1 * 2, W2);
    }
    // 4. long rows: (threshold, piece, slices per block) against the incumbent's
    // defaults (128, 192, 32)
    if (bp.T > 0 && base_layout_default && max_full_row(n, rowptr, col) > 32) {
        const int32_t T4 = bp.T;
        struct L3 { int32_t long_row, piece, slices; };
        for (const L3 &l : {L3{32, 255, 16}, L3{128, 255, 16}, L3{32, 192, 32}, L3{64, 128, 32}}) {
            pars3_split_params c = bp;
            c.long_row = l.long_row;
            c.piece = l.piece;
            c.long_slices = l.slices;
            consider(c);
        }
        // shorter tiles with the chosen long-row settings
        pars3_split_params c = bp;
        c.T = std::max(T4 / 2, bp.W);
        consider(c);
    }
    // 5. kernel variant (k = 1) or lane width (k > 1)
    if (bp.T > 0 && k == 1 && dtype != PARS3_F64 && b0.variant == 0) {
        pars3_split_params c = bp;
        c.variant = PARS3_VARIANT_LOOKAHEAD;
        consider(c);
    }
    if (bp.T > 0 && k > 1 && b0.lane_bytes == 0) {
        const int32_t elem = dtype == PARS3_F64 ? 8 : 4;
        for (int32_t lb : {32, 16, elem}) {
            pars3_split_params c = bp;
            c.lane_bytes = lb;
            consider(c);
        }
    }

    if (tm.e0) cudaEventDestroy(tm.e0);
    if (tm.e1) cudaEventDestroy(tm.e1);
    if (tm.X) cudaFree(tm.X);
    if (tm.Y) cudaFree(tm.Y);
    if (tm.st) cudaStreamDestroy(tm.st);
    devbase_free(tm.base);
    if (rc != PARS3_OK) return rc;
    if (bp.T == 0) return PARS3_EUNSUPPORTED;
    *best = bp;
    if (best_us) *best_us = bus;
    return PARS3_OK;
}
