// device_split.cu -- pars3_split_device: the canonical split of pars3_split
// (Sec. 3.1.2, Eq. 2 and Figs. 7-8) computed on the GPU from device arrays:
//   1. the pattern, values and permutation are checked;
//   2. every stored entry (i, j) moves to (pinv i, pinv j) and is
//      re-triangularized: an entry that lands above the diagonal is stored
//      mirrored, negated for a skew-symmetric S (Eq. 2);
//   3. the entries are sorted by (row, col) -- stable radix sorts by column,
//      then by row -- giving the reordered strict-lower CSR;
//   4. each entry is classified middle-local / middle-halo / outer for the
//      cut (T, W); the middle entries of every tile are listed in (col, row)
//      order and the outer entries in CSR and in CSC order (stable sorts of
//      position lists).
// The arrays are the same, element for element, as the host split's; they
// are copied into the handle, and the device layout is then built from them
// on the host exactly as pars3_split builds it.
#include "device_prims.cuh"

#include <cmath>
#include <memory>
#include <new>

namespace pars3 {
namespace {

constexpr int kErrValue = 2;   // a NaN or Inf value
constexpr int kErrPerm = 4;    // perm is not a permutation of 0 .. n-1

// seen[v] counts how often v occurs in perm; out-of-range entries are flagged
__global__ void perm_count_kernel(int n, const int32_t *__restrict__ perm, int32_t *seen, int *err) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int v = perm[k];
        if (v < 0 || v >= n) atomicOr(err, kErrPerm);
        else atomicAdd(&seen[v], 1);
    }
}

// every vertex must occur exactly once; pinv[perm[k]] = k
__global__ void perm_inverse_kernel(int n, const int32_t *__restrict__ perm, const int32_t *__restrict__ seen,
                                    int32_t *__restrict__ pinv, int *err) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        if (seen[k] != 1) atomicOr(err, kErrPerm);
        const int v = perm[k];
        if (v >= 0 && v < n) pinv[v] = k;
    }
}

__global__ void finite_kernel(int nnz, const double *__restrict__ val, int *err) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += gridDim.x * blockDim.x)
        if (!isfinite(val[k])) atomicOr(err, kErrValue);
}

// Entry e = (i, j) moves to (r, c) = (max, min) of (pinv i, pinv j); when the
// orientation flips (pinv i < pinv j) its value is negated unless S is
// symmetric.  ckey/rkey receive c and r, v the (possibly negated) value.
__global__ void retriangularize_kernel(int nnz, const int32_t *__restrict__ rowof, const int32_t *__restrict__ ci,
                                       const double *__restrict__ val, const int32_t *__restrict__ pinv,
                                       int symmetric, uint32_t *__restrict__ ckey, uint32_t *__restrict__ rkey,
                                       int32_t *__restrict__ idx, double *__restrict__ v) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += gridDim.x * blockDim.x) {
        const int a = pinv[rowof[e]], b = pinv[ci[e]];
        const bool keep = a > b;
        rkey[e] = static_cast<uint32_t>(keep ? a : b);
        ckey[e] = static_cast<uint32_t>(keep ? b : a);
        v[e] = (keep || symmetric) ? val[e] : -val[e];
        idx[e] = e;
    }
}

// out[q] = key[idx[q]] (32-bit keys)
__global__ void gather_key_kernel(int count, const int32_t *__restrict__ idx, const uint32_t *__restrict__ key,
                                  uint32_t *__restrict__ out) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x) out[q] = key[idx[q]];
}

// The sorted entries: col[q] = c of entry idx[q], val[q] its value; row
// counts for the row pointers; the reordered bandwidth max(r - c).
__global__ void emit_kernel(int nnz, const int32_t *__restrict__ idx, const uint32_t *__restrict__ rsorted,
                            const uint32_t *__restrict__ ckey, const double *__restrict__ v,
                            int32_t *__restrict__ col, double *__restrict__ val, int32_t *rowcnt,
                            unsigned long long *bw) {
    unsigned d = 0;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += gridDim.x * blockDim.x) {
        const int e = idx[q];
        const int r = static_cast<int>(rsorted[q]), c = static_cast<int>(ckey[e]);
        col[q] = c;
        val[q] = v[e];
        atomicAdd(&rowcnt[r], 1);
        d = max(d, static_cast<unsigned>(r - c));
    }
    d = __reduce_max_sync(0xffffffffu, d);
    if ((threadIdx.x & 31) == 0 && d) atomicMax(bw, static_cast<unsigned long long>(d));
}

// Class of every sorted entry for the cut (T, W): 0 middle-local (i - j <= W
// and j in i's tile), 1 middle-halo (i - j <= W, j in an earlier tile), 2
// outer.  mflag / oflag mark middle / outer positions; tcnt counts the middle
// entries of each tile.
__global__ void classify_kernel(int nnz, int T, int W, const uint32_t *__restrict__ rsorted,
                                const int32_t *__restrict__ col, uint8_t *__restrict__ cls,
                                int32_t *__restrict__ mflag, int32_t *__restrict__ oflag, int32_t *tcnt,
                                unsigned long long *counts) {
    unsigned c0 = 0, c1 = 0, c2 = 0;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += gridDim.x * blockDim.x) {
        const int i = static_cast<int>(rsorted[q]), j = col[q];
        const int r0 = (i / T) * T;
        const int k = (i - j <= W) ? (j >= r0 ? 0 : 1) : 2;
        cls[q] = static_cast<uint8_t>(k);
        mflag[q] = k != 2;
        oflag[q] = k == 2;
        if (k != 2) atomicAdd(&tcnt[i / T], 1);
        c0 += k == 0;
        c1 += k == 1;
        c2 += k == 2;
    }
    c0 = __reduce_add_sync(0xffffffffu, c0);
    c1 = __reduce_add_sync(0xffffffffu, c1);
    c2 = __reduce_add_sync(0xffffffffu, c2);
    if ((threadIdx.x & 31) == 0) {
        if (c0) atomicAdd(&counts[0], static_cast<unsigned long long>(c0));
        if (c1) atomicAdd(&counts[1], static_cast<unsigned long long>(c1));
        if (c2) atomicAdd(&counts[2], static_cast<unsigned long long>(c2));
    }
}

// positions q with flag[q] set, in order: out[pre[q]] = q
__global__ void compact_kernel(int count, const int32_t *__restrict__ flag, const int32_t *__restrict__ pre,
                               int32_t *__restrict__ out) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x)
        if (flag[q]) out[pre[q]] = q;
}

// key[t] = col[list[t]] (shift 0) or row(list[t]) / T (tile)
__global__ void list_key_kernel(int count, const int32_t *__restrict__ list, const int32_t *__restrict__ col,
                                const uint32_t *__restrict__ rsorted, int T, int by_tile,
                                uint32_t *__restrict__ key) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
        const int q = list[t];
        key[t] = by_tile ? rsorted[q] / static_cast<uint32_t>(T) : static_cast<uint32_t>(col[q]);
    }
}

}  // namespace
}  // namespace pars3

namespace pars3 {
namespace {

template <typename T>
int download(std::vector<T> &dst, const T *src, size_t count, cudaStream_t st) {
    dst.resize(count);
    if (count == 0) return PARS3_OK;
    return cuda_status(cudaMemcpyAsync(dst.data(), src, sizeof(T) * count, cudaMemcpyDeviceToHost, st));
}

int split_device(int32_t n, const int32_t *rp, const int32_t *ci, const double *val, const int32_t *perm,
                 const pars3_split_params *p, pars3_handle **out, cudaStream_t st) {
    if (!out || n < 0 || !rp) return PARS3_EINVAL;
    *out = nullptr;
    pars3_split_params prm{};
    if (p) prm = *p;
    if (split_params_normalize(&prm) != PARS3_OK) return PARS3_EINVAL;
    int32_t nnz = 0;
    int rc = fetch(&nnz, rp + n, sizeof(int32_t), st);
    if (rc != PARS3_OK) return rc;
    if (nnz < 0 || (n == 0 && nnz != 0)) return PARS3_ENOTSKEW;
    if (nnz > 0 && (!ci || !val)) return PARS3_EINVAL;
    const int G = kThreads;
    const int sym = (prm.flags & PARS3_SPLIT_SYMMETRIC) ? 1 : 0;

    Scratch S;
    int *err = S.get<int>(1);
    int32_t *off = S.get<int32_t>(4), *rowof = S.get<int32_t>(nnz), *deg = S.get<int32_t>(n + 1);
    int32_t *pinv = S.get<int32_t>(n), *seen = S.get<int32_t>(n);
    if (S.err() != cudaSuccess) return PARS3_ENOMEM;
    const int32_t off_h[4] = {0, n, 0, nnz};   // one block: vertices [0, n), entries [0, nnz)
    cudaError_t ce = cudaMemcpyAsync(off, off_h, sizeof(off_h), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (ce != cudaSuccess) return cuda_status(ce);
    int herr = 0;

    // 1. checks: pattern first (it bounds every later index), then values and perm
    validate_kernel<<<grid_for(n, G), G, 0, st>>>(n, Blocks{nullptr, off, off + 2}, rp, ci, rowof, deg, err);
    if ((rc = fetch(&herr, err, sizeof(int), st)) != PARS3_OK) return rc;
    if (herr) return PARS3_ENOTSKEW;
    finite_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, val, err);
    if ((rc = fetch(&herr, err, sizeof(int), st)) != PARS3_OK) return rc;
    if (herr) return PARS3_ENONFINITE;
    if (perm) {
        cudaMemsetAsync(seen, 0, sizeof(int32_t) * n, st);
        perm_count_kernel<<<grid_for(n, G), G, 0, st>>>(n, perm, seen, err);
        perm_inverse_kernel<<<grid_for(n, G), G, 0, st>>>(n, perm, seen, pinv, err);
        if ((rc = fetch(&herr, err, sizeof(int), st)) != PARS3_OK) return rc;
        if (herr) return PARS3_EINVAL;
    } else {
        iota_kernel<<<grid_for(n, G), G, 0, st>>>(n, pinv);
    }

    // 2-3. re-triangularize, then sort by (row, col): by column, then stably by row
    uint32_t *ckey = S.get<uint32_t>(nnz), *rkey = S.get<uint32_t>(nnz);
    uint32_t *ka = S.get<uint32_t>(nnz), *kb = S.get<uint32_t>(nnz);
    int32_t *va = S.get<int32_t>(nnz), *vb = S.get<int32_t>(nnz);
    double *vv = S.get<double>(nnz), *val_s = S.get<double>(nnz);
    int32_t *col_s = S.get<int32_t>(nnz), *rowcnt = S.get<int32_t>(n), *rowptr = S.get<int32_t>(n + 1);
    const int stiles = (nnz + kSortTile - 1) / kSortTile;
    int32_t *hist = S.get<int32_t>(256 * static_cast<size_t>(stiles) + 1);
    int32_t *hoff = S.get<int32_t>(256 * static_cast<size_t>(stiles) + 1);
    unsigned long long *acc = S.get<unsigned long long>(4);   // bandwidth, then the three class counts
    if (S.err() != cudaSuccess) return PARS3_ENOMEM;
    const int nbits = bits_for(n);
    retriangularize_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, rowof, ci, val, pinv, sym, ckey, rkey, va, vv);
    cudaMemcpyAsync(ka, ckey, sizeof(uint32_t) * nnz, cudaMemcpyDeviceToDevice, st);
    uint32_t *ko, *k2;
    int32_t *vo, *v2;
    radix_sort(ka, va, kb, vb, nnz, nbits, hist, hoff, st, &ko, &vo);
    uint32_t *kx = ko == ka ? kb : ka;
    int32_t *vx = vo == va ? vb : va;
    gather_key_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, vo, rkey, kx);
    radix_sort(kx, vo, ko, vx, nnz, nbits, hist, hoff, st, &k2, &v2);
    // the row of every sorted entry gets its own buffer: the sort buffers are reused below
    uint32_t *rsorted = rkey;
    cudaMemcpyAsync(rsorted, k2, sizeof(uint32_t) * nnz, cudaMemcpyDeviceToDevice, st);
    const int32_t *order = v2;   // source entry of every sorted position (read by emit_kernel only)
    cudaMemsetAsync(rowcnt, 0, sizeof(int32_t) * n, st);
    cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 4, st);
    emit_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, order, rsorted, ckey, vv, col_s, val_s, rowcnt, acc);
    scan_kernel<<<1, kScanThreads, 0, st>>>(rowcnt, rowptr, nullptr, n);
    unsigned long long bw = 0;
    if ((rc = fetch(&bw, acc, sizeof(bw), st)) != PARS3_OK) return rc;

    // the cut: given, or the default rule on the reordered bandwidth
    if (prm.T == 0) {
        const int32_t wcap = (prm.dtypes & PARS3_DTYPE_BIT(PARS3_F64)) ? 1024 : 2048;
        auto_cut(static_cast<int64_t>(bw), 32, wcap, 1024, &prm.T, &prm.W);
    }
    if (check_cut(prm.T, prm.W) != PARS3_OK) return PARS3_EINVAL;
    const int T = prm.T, W = prm.W;
    const int ntiles = n > 0 ? (n + T - 1) / T : 0;

    // 4. classes, tile lists in (tile, col, position) order, outer lists
    uint8_t *cls = S.get<uint8_t>(nnz);
    int32_t *mflag = S.get<int32_t>(nnz), *oflag = S.get<int32_t>(nnz);
    int32_t *mpre = S.get<int32_t>(nnz + 1), *opre = S.get<int32_t>(nnz + 1);
    int32_t *tcnt = S.get<int32_t>(ntiles), *tile_ptr = S.get<int32_t>(ntiles + 1);
    int32_t *mlist = S.get<int32_t>(nnz), *olist = S.get<int32_t>(nnz);
    if (S.err() != cudaSuccess) return PARS3_ENOMEM;
    cudaMemsetAsync(tcnt, 0, sizeof(int32_t) * ntiles, st);
    classify_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, T, W, rsorted, col_s, cls, mflag, oflag, tcnt, acc + 1);
    scan_kernel<<<1, kScanThreads, 0, st>>>(mflag, mpre, nullptr, nnz);
    scan_kernel<<<1, kScanThreads, 0, st>>>(oflag, opre, nullptr, nnz);
    scan_kernel<<<1, kScanThreads, 0, st>>>(tcnt, tile_ptr, nullptr, ntiles);
    compact_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, mflag, mpre, mlist);
    compact_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, oflag, opre, olist);
    int32_t M = 0, O = 0;
    unsigned long long cnt3[3] = {0, 0, 0};
    cudaMemcpyAsync(&M, mpre + nnz, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&O, opre + nnz, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if ((rc = fetch(cnt3, acc + 1, sizeof(cnt3), st)) != PARS3_OK) return rc;
    // middle list: positions (in order), stably by column, then stably by tile
    cudaMemcpyAsync(va, mlist, sizeof(int32_t) * M, cudaMemcpyDeviceToDevice, st);
    list_key_kernel<<<grid_for(M, G), G, 0, st>>>(M, va, col_s, rsorted, T, 0, ka);
    radix_sort(ka, va, kb, vb, M, nbits, hist, hoff, st, &ko, &vo);
    kx = ko == ka ? kb : ka;
    vx = vo == va ? vb : va;
    list_key_kernel<<<grid_for(M, G), G, 0, st>>>(M, vo, col_s, rsorted, T, 1, kx);
    radix_sort(kx, vo, ko, vx, M, bits_for(ntiles), hist, hoff, st, &k2, &v2);
    int32_t *tile_list = v2;
    pars3_handle *h = nullptr;
    try {
        h = new pars3_handle();
    } catch (const std::bad_alloc &) {
        return PARS3_ENOMEM;
    }
    std::unique_ptr<pars3_handle> hold(h);
    rc = download(h->tile_list, tile_list, M, st);
    if (rc == PARS3_OK) rc = cuda_status(cudaStreamSynchronize(st));   // va / vb are reused below
    if (rc != PARS3_OK) return rc;
    // outer lists: in position order (CSR), and stably by column (CSC)
    cudaMemcpyAsync(va, olist, sizeof(int32_t) * O, cudaMemcpyDeviceToDevice, st);
    list_key_kernel<<<grid_for(O, G), G, 0, st>>>(O, va, col_s, rsorted, T, 0, ka);
    radix_sort(ka, va, kb, vb, O, nbits, hist, hoff, st, &ko, &vo);

    // the handle: canonical arrays from the device, then the host layout
    try {
        h->n = n;
        h->nnz = nnz;
        h->dtypes = prm.dtypes;
        h->symmetric = sym;
        h->T = T;
        h->W = W;
        h->ntiles = ntiles;
        h->bw = static_cast<int64_t>(bw);
        for (int k = 0; k < 3; ++k) h->counts[k] = static_cast<int64_t>(cnt3[k]);
        if (perm) {
            rc = download(h->perm, perm, n, st);
        } else {
            h->perm.resize(n);
            for (int32_t k = 0; k < n; ++k) h->perm[k] = k;
        }
        if (rc == PARS3_OK) rc = download(h->rowptr, rowptr, static_cast<size_t>(n) + 1, st);
        if (rc == PARS3_OK) rc = download(h->col, col_s, nnz, st);
        if (rc == PARS3_OK) rc = download(h->val, val_s, nnz, st);
        if (rc == PARS3_OK) rc = download(h->cls, cls, nnz, st);
        if (rc == PARS3_OK) rc = download(h->tile_ptr, tile_ptr, static_cast<size_t>(ntiles) + 1, st);
        if (rc == PARS3_OK) rc = download(h->outer_csr, olist, O, st);
        if (rc == PARS3_OK) rc = download(h->outer_csc, vo, O, st);
        if (rc == PARS3_OK) rc = cuda_status(cudaStreamSynchronize(st));
        if (rc != PARS3_OK) return rc;
    } catch (const std::bad_alloc &) {
        return PARS3_ENOMEM;
    }
    rc = split_finish(h, prm);
    if (rc != PARS3_OK) return rc;
    *out = hold.release();
    return PARS3_OK;
}

}  // namespace
}  // namespace pars3

extern "C" int pars3_split_device(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                                  const int32_t *perm, const pars3_split_params *p, pars3_handle **out,
                                  void *stream) {
    return pars3::split_device(n, rowptr, col, val, perm, p, out, static_cast<cudaStream_t>(stream));
}
