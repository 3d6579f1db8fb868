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
// The arrays are the same, element for element, as the host split's and are
// copied into the handle.  The device layout is then built from them on the
// GPU (layout_try_device): the per-entry steps run in kernels, the decisions
// over rows and tiles are the host builder's own helpers, so the layout is
// the one pars3_split builds.
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

// ------------------------------------------------------------ layout (GPU side)
//
// The device layout is built from the canonical split as the host builder
// builds it: the decisions over rows and tiles (which tiles keep the half
// path, long rows, slice order, pieces, fold items) are the host builder's
// own helpers, run on per-row and per-tile counts from the device; every
// per-entry step runs here.

// cent = entry positions in column order (row order within a column, a
// stable sort of positions by column); colcnt counts the entries of each column
__global__ void col_count_kernel(int nnz, const int32_t *__restrict__ col, int32_t *colcnt) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += gridDim.x * blockDim.x)
        atomicAdd(&colcnt[col[q]], 1);
}

// half[q]: a middle entry of a tile that keeps the half path
__global__ void half_flag_kernel(int nnz, int T, const uint32_t *__restrict__ rs, const uint8_t *__restrict__ cls,
                                 const uint8_t *__restrict__ tile_on, uint8_t *__restrict__ half,
                                 int32_t *__restrict__ hflag) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += gridDim.x * blockDim.x) {
        const int h = cls[q] != 2 && tile_on[rs[q] / static_cast<uint32_t>(T)];
        half[q] = static_cast<uint8_t>(h);
        hflag[q] = h;
    }
}

// A half entry's slot in its tile's (row, col) list: hoff[t] + its rank
// among the tile's half entries; its window column and source entry there.
__global__ void half_place_kernel(int nnz, int T, int W, const uint32_t *__restrict__ rs,
                                  const int32_t *__restrict__ col, const uint8_t *__restrict__ half,
                                  const int32_t *__restrict__ hscan, const int32_t *__restrict__ rowptr,
                                  const int32_t *__restrict__ hoff, uint16_t *__restrict__ hcol,
                                  int32_t *__restrict__ hsrc, int32_t *__restrict__ hpos) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += gridDim.x * blockDim.x) {
        if (!half[q]) continue;
        const int t = static_cast<int>(rs[q]) / T, r0 = t * T;
        const int pos = hoff[t] + hscan[q] - hscan[rowptr[r0]];
        hpos[q] = pos;
        hcol[pos] = static_cast<uint16_t>(col[q] - (r0 - W));
        hsrc[pos] = q + 1;
    }
}

// tile-local row pointers of the half entries (T + 8 per tile; rows past the
// tile's end repeat its count)
__global__ void half_rowptr_kernel(int n, int nt, int T, const int32_t *__restrict__ rowptr,
                                   const int32_t *__restrict__ hscan, uint16_t *__restrict__ hrp) {
    const int64_t total = static_cast<int64_t>(nt) * (T + 8);
    for (int64_t x = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; x < total;
         x += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int t = static_cast<int>(x / (T + 8)), i = static_cast<int>(x % (T + 8));
        const int r0 = t * T, r1 = min(n, r0 + T), r = min(r0 + i, r1);
        hrp[x] = static_cast<uint16_t>(hscan[rowptr[r]] - hscan[rowptr[r0]]);
    }
}

// Walk of each half tile's (col, row) list: the (col, row) order's slots
// (hcperm), the window position of each entry's row (hrowc), and the first
// entry of every distinct column (a segment; halo segments have a column
// before the tile), counted per tile.
__global__ void segment_kernel(int M, int T, int W, const int32_t *__restrict__ tlist,
                               const int32_t *__restrict__ tile_ptr, const uint32_t *__restrict__ rs,
                               const int32_t *__restrict__ col, const uint8_t *__restrict__ tile_on,
                               const int32_t *__restrict__ hoff, const int32_t *__restrict__ hpos,
                               uint16_t *__restrict__ hcperm, uint16_t *__restrict__ hrowc,
                               int32_t *__restrict__ segflag, int32_t *nseg, int32_t *nhalo) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < M; s += gridDim.x * blockDim.x) {
        const int e = tlist[s];
        const int t = static_cast<int>(rs[e]) / T, r0 = t * T;
        if (!tile_on[t]) {
            segflag[s] = 0;
            continue;
        }
        const int k = s - tile_ptr[t];
        const int pos = hoff[t] + k;
        hcperm[pos] = static_cast<uint16_t>(hpos[e] - hoff[t]);
        hrowc[pos] = static_cast<uint16_t>(static_cast<int>(rs[e]) - (r0 - W));
        const int j = col[e];
        const bool first = k == 0 || col[tlist[s - 1]] != j;
        segflag[s] = first;
        if (first) {
            atomicAdd(&nseg[t], 1);
            if (j < r0) atomicAdd(&nhalo[t], 1);
        }
    }
}

// segment words (window position | first (col, row) index << 16) at the
// segment's rank in its tile; halo segments come first, so a halo
// segment's rank is also its halo target index
__global__ void segment_write_kernel(int M, int T, int W, const int32_t *__restrict__ tlist,
                                     const int32_t *__restrict__ tile_ptr, const uint32_t *__restrict__ rs,
                                     const int32_t *__restrict__ col, const int32_t *__restrict__ segflag,
                                     const int32_t *__restrict__ segscan, const int32_t *__restrict__ hcsoff,
                                     const int32_t *__restrict__ hhoff, uint32_t *__restrict__ hcs,
                                     int32_t *__restrict__ hhrow) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < M; s += gridDim.x * blockDim.x) {
        if (!segflag[s]) continue;
        const int e = tlist[s];
        const int t = static_cast<int>(rs[e]) / T, r0 = t * T;
        const int k = s - tile_ptr[t];
        const int rank = segscan[s] - segscan[tile_ptr[t]];
        const int j = col[e];
        hcs[hcsoff[t] + rank] = static_cast<uint32_t>(j - (r0 - W)) | (static_cast<uint32_t>(k) << 16);
        if (j < r0) hhrow[hhoff[t] + rank] = j;
    }
}

// end words: every word of a tile after its segments is 0xffff | count << 16
__global__ void segment_end_kernel(int nt, const int32_t *__restrict__ hcsoff, const int32_t *__restrict__ nseg,
                                   const int32_t *__restrict__ hcnt, uint32_t *__restrict__ hcs) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x)
        for (int w = hcsoff[t] + nseg[t]; w < hcsoff[t + 1]; ++w)
            hcs[w] = 0xffffu | (static_cast<uint32_t>(hcnt[t]) << 16);
}

// full-path length of every row: its non-half lower entries and the
// non-half entries of its column (mirrored)
__global__ void full_len_kernel(int n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ cptr,
                                const int32_t *__restrict__ cent, const uint8_t *__restrict__ half,
                                int32_t *__restrict__ flen) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int c = 0;
        for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) c += !half[q];
        for (int s = cptr[i]; s < cptr[i + 1]; ++s) c += !half[cent[s]];
        flen[i] = c;
    }
}

// Row i's full-path entries (lower ones in column order, then the mirrored
// ones of its column in row order) at out[base + m * stride]: the column
// and the source (+(q+1) lower, -(q+1) mirrored).  One thread per row.
__device__ __forceinline__ void emit_full_row(int i, const int32_t *__restrict__ rowptr,
                                              const int32_t *__restrict__ col, const int32_t *__restrict__ cptr,
                                              const int32_t *__restrict__ cent, const uint32_t *__restrict__ rs,
                                              const uint8_t *__restrict__ half, int64_t base, int stride,
                                              int32_t *__restrict__ ocol, int32_t *__restrict__ osrc) {
    int64_t o = base;
    for (int q = rowptr[i]; q < rowptr[i + 1]; ++q)
        if (!half[q]) {
            ocol[o] = col[q];
            osrc[o] = q + 1;
            o += stride;
        }
    for (int s = cptr[i]; s < cptr[i + 1]; ++s) {
        const int q = cent[s];
        if (!half[q]) {
            ocol[o] = static_cast<int32_t>(rs[q]);
            osrc[o] = -(q + 1);
            o += stride;
        }
    }
}

__global__ void emit_slices_kernel(int n, const int32_t *__restrict__ row_base, const int32_t *__restrict__ rowptr,
                                   const int32_t *__restrict__ col, const int32_t *__restrict__ cptr,
                                   const int32_t *__restrict__ cent, const uint32_t *__restrict__ rs,
                                   const uint8_t *__restrict__ half, int32_t *__restrict__ fcol,
                                   int32_t *__restrict__ fsrc) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (row_base[i] >= 0) emit_full_row(i, rowptr, col, cptr, cent, rs, half, row_base[i], 32, fcol, fsrc);
}

__global__ void emit_long_kernel(int nlong, const int32_t *__restrict__ lrow, const int32_t *__restrict__ lrp,
                                 const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                 const int32_t *__restrict__ cptr, const int32_t *__restrict__ cent,
                                 const uint32_t *__restrict__ rs, const uint8_t *__restrict__ half,
                                 int32_t *__restrict__ lflat, int32_t *__restrict__ lsflat) {
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nlong; l += gridDim.x * blockDim.x)
        emit_full_row(lrow[l], rowptr, col, cptr, cent, rs, half, lrp[l], 1, lflat, lsflat);
}

// piece p (first entry e0, length len) goes to lane p % 32 of long slice p / 32
__global__ void piece_scatter_kernel(int npieces, const int2 *__restrict__ pieces, const int32_t *__restrict__ ls_ent,
                                     const int32_t *__restrict__ lflat, const int32_t *__restrict__ lsflat,
                                     int32_t *__restrict__ lcol, int32_t *__restrict__ lsrc) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npieces; p += gridDim.x * blockDim.x) {
        const int2 pc = pieces[p];
        const int64_t base = static_cast<int64_t>(ls_ent[p / 32]) + (p % 32);
        for (int m = 0; m < pc.y; ++m) {
            lcol[base + 32LL * m] = lflat[pc.x + m];
            lsrc[base + 32LL * m] = lsflat[pc.x + m];
        }
    }
}

// bf16 bits of an fp32 value, round to nearest even (quiet NaNs keep a payload bit)
__device__ __forceinline__ uint16_t bf16_rne_bits(float f) {
    uint32_t u = __float_as_uint(f);
    if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu)) return static_cast<uint16_t>((u >> 16) | 0x40u);
    u += 0x7fffu + ((u >> 16) & 1u);
    return static_cast<uint16_t>(u >> 16);
}

// values of every slot from its source (+(q+1) lower, -(q+1) mirrored with
// the mirror sign, 0 padding), in each packed precision
__global__ void fill_values_kernel(int64_t m, const int32_t *__restrict__ src, const double *__restrict__ val,
                                   int symmetric, double *__restrict__ v64, float *__restrict__ v32,
                                   uint16_t *__restrict__ v16) {
    for (int64_t x = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; x < m;
         x += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int s = src[x];
        double a = 0.0;
        if (s > 0) a = val[s - 1];
        else if (s < 0) a = symmetric ? val[-s - 1] : -val[-s - 1];
        const float f = static_cast<float>(a);
        if (v64) v64[x] = a;
        if (v32) v32[x] = f;
        if (v16) v16[x] = s == 0 ? 0 : bf16_rne_bits(f);
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

template <typename T>
int upload(T *dst, const std::vector<T> &src, cudaStream_t st) {
    if (src.empty()) return PARS3_OK;
    return cuda_status(cudaMemcpyAsync(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, st));
}

// the canonical split in device memory
struct DevCanon {
    const uint32_t *rs;       // row of every sorted entry
    const int32_t *col, *rowptr, *tile_ptr, *tlist;
    const double *val;
    const uint8_t *cls;
    const int32_t *cptr, *cent;   // column view
};

// One attempt of the layout build at half-path capacity mcap (as
// build_layout_try on the host).  Every host vector of h->L is filled.
int layout_try_device(pars3_handle *h, const DevCanon &C, int64_t mcap, cudaStream_t st) {
    Layout &L = h->L;
    L = Layout();
    const int32_t n = h->n, T = h->T, W = h->W, nt = h->ntiles;
    const int nnz = static_cast<int>(h->nnz);
    const int M = h->tile_ptr.empty() ? 0 : h->tile_ptr[nt];
    const int G = kThreads;
    Scratch S;
    int rc;
    // ---- 1. half path
    std::vector<int32_t> tcount(nt);
    for (int32_t t = 0; t < nt; ++t) tcount[t] = h->tile_ptr[t + 1] - h->tile_ptr[t];
    half_tiles(h, mcap, tcount);
    std::vector<uint8_t> on(nt);
    for (int32_t t = 0; t < nt; ++t) on[t] = tcount[t] > 0;
    const int64_t hn = L.hoff[nt];
    const int64_t nrp = static_cast<int64_t>(nt) * (T + 8);
    uint8_t *tile_on = S.get<uint8_t>(nt), *half = S.get<uint8_t>(nnz);
    int32_t *hoff = S.get<int32_t>(nt + 1), *hcnt = S.get<int32_t>(nt), *hflag = S.get<int32_t>(nnz);
    int32_t *hscan = S.get<int32_t>(static_cast<size_t>(nnz) + 1), *hpos = S.get<int32_t>(nnz);
    uint16_t *hcol = S.get<uint16_t>(hn), *hcperm = S.get<uint16_t>(hn), *hrowc = S.get<uint16_t>(hn);
    uint16_t *hrp = S.get<uint16_t>(nrp);
    int32_t *hsrc = S.get<int32_t>(hn);
    int32_t *sws = S.get<int32_t>(scan_ws_size(std::max(nnz, M)));
    if (S.err() != cudaSuccess) return PARS3_ENOMEM;
    if ((rc = upload(tile_on, on, st)) != PARS3_OK || (rc = upload(hoff, L.hoff, st)) != PARS3_OK ||
        (rc = upload(hcnt, L.hcnt, st)) != PARS3_OK)
        return rc;
    cudaMemsetAsync(hcol, 0, sizeof(uint16_t) * hn, st);
    cudaMemsetAsync(hcperm, 0, sizeof(uint16_t) * hn, st);
    cudaMemsetAsync(hrowc, 0, sizeof(uint16_t) * hn, st);
    cudaMemsetAsync(hsrc, 0, sizeof(int32_t) * hn, st);
    half_flag_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, T, C.rs, C.cls, tile_on, half, hflag);
    scan_exclusive(hflag, hscan, nnz, sws, st);
    half_place_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, T, W, C.rs, C.col, half, hscan, C.rowptr, hoff, hcol,
                                                      hsrc, hpos);
    half_rowptr_kernel<<<grid_for(nrp, G), G, 0, st>>>(n, nt, T, C.rowptr, hscan, hrp);
    // column segments
    int32_t *segflag = S.get<int32_t>(M), *segscan = S.get<int32_t>(static_cast<size_t>(M) + 1);
    int32_t *nseg = S.get<int32_t>(nt), *nhalo = S.get<int32_t>(nt);
    if (S.err() != cudaSuccess) return PARS3_ENOMEM;
    cudaMemsetAsync(nseg, 0, sizeof(int32_t) * nt, st);
    cudaMemsetAsync(nhalo, 0, sizeof(int32_t) * nt, st);
    segment_kernel<<<grid_for(M, G), G, 0, st>>>(M, T, W, C.tlist, C.tile_ptr, C.rs, C.col, tile_on, hoff, hpos,
                                                 hcperm, hrowc, segflag, nseg, nhalo);
    scan_exclusive(segflag, segscan, M, sws, st);
    std::vector<int32_t> nseg_h, nhalo_h;
    if ((rc = download(nseg_h, nseg, nt, st)) != PARS3_OK || (rc = download(nhalo_h, nhalo, nt, st)) != PARS3_OK ||
        (rc = cuda_status(cudaStreamSynchronize(st))) != PARS3_OK)
        return rc;
    L.hcsoff.assign(static_cast<size_t>(nt) + 1, 0);
    L.hhoff.assign(static_cast<size_t>(nt) + 1, 0);
    L.hcsn.assign(nt, 0);
    L.max_tile_cs = 0;
    for (int32_t t = 0; t < nt; ++t) {
        L.hcsn[t] = nseg_h[t];
        L.hcsoff[t + 1] = static_cast<int32_t>(L.hcsoff[t] + round_up(nseg_h[t] + 1, 4));
        L.hhoff[t + 1] = L.hhoff[t] + nhalo_h[t];
        L.max_tile_cs = std::max(L.max_tile_cs, L.hcsoff[t + 1] - L.hcsoff[t]);
    }
    int32_t *hcsoff = S.get<int32_t>(nt + 1), *hhoff = S.get<int32_t>(nt + 1);
    uint32_t *hcs = S.get<uint32_t>(L.hcsoff[nt]);
    int32_t *hhrow = S.get<int32_t>(L.hhoff[nt]);
    if (S.err() != cudaSuccess) return PARS3_ENOMEM;
    if ((rc = upload(hcsoff, L.hcsoff, st)) != PARS3_OK || (rc = upload(hhoff, L.hhoff, st)) != PARS3_OK) return rc;
    segment_write_kernel<<<grid_for(M, G), G, 0, st>>>(M, T, W, C.tlist, C.tile_ptr, C.rs, C.col, segflag, segscan,
                                                       hcsoff, hhoff, hcs, hhrow);
    segment_end_kernel<<<grid_for(nt, G), G, 0, st>>>(nt, hcsoff, nseg, hcnt, hcs);
    // ---- 2. full-path lengths
    int32_t *flen = S.get<int32_t>(n);
    if (S.err() != cudaSuccess) return PARS3_ENOMEM;
    full_len_kernel<<<grid_for(n, G), G, 0, st>>>(n, C.rowptr, C.cptr, C.cent, half, flen);
    std::vector<int32_t> flen_h;
    if ((rc = download(flen_h, flen, n, st)) != PARS3_OK || (rc = download(L.hhrow, hhrow, L.hhoff[nt], st)) != PARS3_OK ||
        (rc = cuda_status(cudaStreamSynchronize(st))) != PARS3_OK)
        return rc;
    int64_t ftotal = 0;
    for (int32_t i = 0; i < n; ++i) ftotal += flen_h[i];
    // ---- 3. long rows
    std::vector<uint8_t> is_long;
    long_rows(h, flen_h, ftotal, 0, is_long);
    // ---- 4. slices: each tile's rows by full length, longest first, ties by
    // row (a counting sort per tile: short rows have at most kSellMax entries)
    std::vector<int32_t> slen(n), rows(n), row_base;
    for (int32_t i = 0; i < n; ++i) slen[i] = is_long[i] ? 0 : flen_h[i];
    {
        std::vector<int32_t> bucket(kSellMax + 2);
        for (int32_t t = 0; t < nt; ++t) {
            const int32_t r0 = t * T, r1 = std::min(n, r0 + T);
            std::fill(bucket.begin(), bucket.end(), 0);
            for (int32_t i = r0; i < r1; ++i) ++bucket[kSellMax - slen[i] + 1];
            for (int b = 0; b <= kSellMax; ++b) bucket[b + 1] += bucket[b];
            for (int32_t i = r0; i < r1; ++i) rows[r0 + bucket[kSellMax - slen[i]]++] = i;
        }
    }
    if ((rc = slice_rows(h, rows, slen, row_base)) != PARS3_OK) return rc;
    const int64_t fnp = L.sl_ent.back();
    int32_t *rbase = S.get<int32_t>(n), *fcol = S.get<int32_t>(fnp), *fsrc = S.get<int32_t>(fnp);
    if (S.err() != cudaSuccess) return PARS3_ENOMEM;
    if ((rc = upload(rbase, row_base, st)) != PARS3_OK) return rc;
    cudaMemsetAsync(fcol, 0, sizeof(int32_t) * fnp, st);
    cudaMemsetAsync(fsrc, 0, sizeof(int32_t) * fnp, st);
    emit_slices_kernel<<<grid_for(n, G), G, 0, st>>>(n, rbase, C.rowptr, C.col, C.cptr, C.cent, C.rs, half, fcol,
                                                     fsrc);
    // ---- 5. long rows in pieces
    std::vector<PieceRef> pieces;
    if ((rc = long_pieces(h, is_long, flen_h, pieces)) != PARS3_OK) return rc;
    const int nlong = static_cast<int>(L.lrow.size());
    const int64_t ltot = L.lrp.back(), lslots = L.ls_ent.back();
    const int npieces = static_cast<int>(pieces.size());
    std::vector<int2> pc(npieces);
    for (int p = 0; p < npieces; ++p) pc[p] = make_int2(pieces[p].e0, pieces[p].len);
    int32_t *lrow = S.get<int32_t>(nlong), *lrp = S.get<int32_t>(static_cast<size_t>(nlong) + 1);
    int32_t *lflat = S.get<int32_t>(ltot), *lsflat = S.get<int32_t>(ltot), *ls_ent = S.get<int32_t>(L.ls_ent.size());
    int32_t *lcol = S.get<int32_t>(lslots), *lsrc = S.get<int32_t>(lslots);
    int2 *pcs = S.get<int2>(npieces);
    if (S.err() != cudaSuccess) return PARS3_ENOMEM;
    if ((rc = upload(lrow, L.lrow, st)) != PARS3_OK || (rc = upload(lrp, L.lrp, st)) != PARS3_OK ||
        (rc = upload(ls_ent, L.ls_ent, st)) != PARS3_OK || (rc = upload(pcs, pc, st)) != PARS3_OK)
        return rc;
    cudaMemsetAsync(lcol, 0, sizeof(int32_t) * lslots, st);
    cudaMemsetAsync(lsrc, 0, sizeof(int32_t) * lslots, st);
    emit_long_kernel<<<grid_for(nlong, G), G, 0, st>>>(nlong, lrow, lrp, C.rowptr, C.col, C.cptr, C.cent, C.rs, half,
                                                       lflat, lsflat);
    piece_scatter_kernel<<<grid_for(npieces, G), G, 0, st>>>(npieces, pcs, ls_ent, lflat, lsflat, lcol, lsrc);
    // ---- 6. fold items
    fold_items(h);
    // ---- 7. values per precision, then everything to the host
    const bool d64 = h->dtypes & PARS3_DTYPE_BIT(PARS3_F64), d32 = h->dtypes & PARS3_DTYPE_BIT(PARS3_F32),
               d16 = h->dtypes & PARS3_DTYPE_BIT(PARS3_BF16);
    struct Part {
        const int32_t *src;
        int64_t m;
        std::vector<double> *v64;
        std::vector<float> *v32;
        std::vector<uint16_t> *v16;
    } parts[3] = {{hsrc, hn, &L.hval64, &L.hval32, &L.hval16},
                  {fsrc, fnp, &L.fval64, &L.fval32, &L.fval16},
                  {lsrc, lslots, &L.lval64, &L.lval32, &L.lval16}};
    for (const Part &pt : parts) {
        Scratch V;
        double *v64 = d64 ? V.get<double>(pt.m) : nullptr;
        float *v32 = d32 ? V.get<float>(pt.m) : nullptr;
        uint16_t *v16 = d16 ? V.get<uint16_t>(pt.m) : nullptr;
        if (V.err() != cudaSuccess) return PARS3_ENOMEM;
        fill_values_kernel<<<grid_for(pt.m, G), G, 0, st>>>(pt.m, pt.src, C.val, h->symmetric, v64, v32, v16);
        if (d64 && (rc = download(*pt.v64, static_cast<const double *>(v64), pt.m, st)) != PARS3_OK) return rc;
        if (d32 && (rc = download(*pt.v32, static_cast<const float *>(v32), pt.m, st)) != PARS3_OK) return rc;
        if (d16 && (rc = download(*pt.v16, static_cast<const uint16_t *>(v16), pt.m, st)) != PARS3_OK) return rc;
        if ((rc = cuda_status(cudaStreamSynchronize(st))) != PARS3_OK) return rc;   // V is freed next
    }
    if ((rc = download(L.hcol, static_cast<const uint16_t *>(hcol), hn, st)) != PARS3_OK ||
        (rc = download(L.hcperm, static_cast<const uint16_t *>(hcperm), hn, st)) != PARS3_OK ||
        (rc = download(L.hrowc, static_cast<const uint16_t *>(hrowc), hn, st)) != PARS3_OK ||
        (rc = download(L.hrp, static_cast<const uint16_t *>(hrp), nrp, st)) != PARS3_OK ||
        (rc = download(L.hcs, static_cast<const uint32_t *>(hcs), L.hcsoff[nt], st)) != PARS3_OK ||
        (rc = download(L.fcol, static_cast<const int32_t *>(fcol), fnp, st)) != PARS3_OK ||
        (rc = download(L.lcol, static_cast<const int32_t *>(lcol), lslots, st)) != PARS3_OK)
        return rc;
    return cuda_status(cudaStreamSynchronize(st));
}

// The layout search of build_layout with the GPU attempt: start with every
// middle entry of a fitting tile on the half path; while the tile block does
// not fit shared memory, halve the largest half-path tile.
int build_layout_device(pars3_handle *h, const DevCanon &C, cudaStream_t st) {
    int64_t mcap = half_room(h);
    if (mcap < 0) return PARS3_EUNSUPPORTED;
    for (int iter = 0; iter < 40; ++iter) {
        const int rc = layout_try_device(h, C, mcap, st);
        if (rc != PARS3_OK) return rc;
        if (max_smem_all(h) <= kSmemLimit) return PARS3_OK;
        if (h->L.max_tile_half == 0) return PARS3_EUNSUPPORTED;
        mcap = h->L.max_tile_half / 2;
    }
    return PARS3_EUNSUPPORTED;
}

}  // namespace

// The reordered matrix on the device: the stages of the split that do not
// depend on the cut (checks, re-triangularization, (row, col) order, column
// view), kept for any number of cuts (pars3_split_device makes one, the
// autotuner one per candidate).  It owns its device memory.
struct DevBase {
    Scratch S;
    int32_t n = 0, nnz = 0, sym = 0;
    int64_t bw = 0;
    uint32_t *rs = nullptr;   // row of every sorted entry
    int32_t *col = nullptr, *rowptr = nullptr, *cptr = nullptr, *cent = nullptr;
    double *val = nullptr;
    uint32_t *ka = nullptr, *kb = nullptr;   // sort buffers
    int32_t *va = nullptr, *vb = nullptr, *hist = nullptr, *hoff = nullptr;
    int32_t *sws = nullptr;   // prefix-sum workspace
    std::vector<int32_t> perm_h, rowptr_h, col_h;   // host copies for the handles
    std::vector<double> val_h;
};

namespace {

int base_build(DevBase &B, int32_t n, const int32_t *rp, const int32_t *ci, const double *val, const int32_t *perm,
               int sym, cudaStream_t st) {
    int32_t nnz = 0;
    int rc = fetch(&nnz, rp + n, sizeof(int32_t), st);
    if (rc != PARS3_OK) return rc;
    if (nnz < 0 || (n == 0 && nnz != 0)) return PARS3_ENOTSKEW;
    if (nnz > 0 && (!ci || !val)) return PARS3_EINVAL;
    const int G = kThreads;
    B.n = n;
    B.nnz = nnz;
    B.sym = sym;
    Scratch T;   // temporaries of this stage
    Scratch &S = B.S;
    int *err = T.get<int>(1);
    int32_t *off = T.get<int32_t>(4), *rowof = T.get<int32_t>(nnz), *deg = T.get<int32_t>(n + 1);
    int32_t *pinv = T.get<int32_t>(n), *seen = T.get<int32_t>(n);
    if (T.err() != cudaSuccess) return PARS3_ENOMEM;
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
    uint32_t *ckey = T.get<uint32_t>(nnz);
    double *vv = T.get<double>(nnz);
    int32_t *rowcnt = T.get<int32_t>(n), *colcnt = T.get<int32_t>(n);
    unsigned long long *acc = T.get<unsigned long long>(1);
    B.rs = S.get<uint32_t>(nnz);
    B.ka = S.get<uint32_t>(nnz);
    B.kb = S.get<uint32_t>(nnz);
    B.va = S.get<int32_t>(nnz);
    B.vb = S.get<int32_t>(nnz);
    B.val = S.get<double>(nnz);
    B.col = S.get<int32_t>(nnz);
    B.rowptr = S.get<int32_t>(static_cast<size_t>(n) + 1);
    B.cptr = S.get<int32_t>(static_cast<size_t>(n) + 1);
    B.cent = S.get<int32_t>(nnz);
    const int stiles = (nnz + kSortTile - 1) / kSortTile;
    B.hist = S.get<int32_t>(256 * static_cast<size_t>(stiles) + 1);
    B.hoff = S.get<int32_t>(256 * static_cast<size_t>(stiles) + 1);
    B.sws = S.get<int32_t>(scan_ws_size(std::max(std::max(n, nnz), 256 * stiles + 1)));
    if (T.err() != cudaSuccess || S.err() != cudaSuccess) return PARS3_ENOMEM;
    uint32_t *ka = B.ka, *kb = B.kb, *rkey = B.rs;
    int32_t *va = B.va, *vb = B.vb;
    const int nbits = bits_for(n);
    retriangularize_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, rowof, ci, val, pinv, sym, ckey, rkey, va, vv);
    cudaMemcpyAsync(ka, ckey, sizeof(uint32_t) * nnz, cudaMemcpyDeviceToDevice, st);
    uint32_t *ko, *k2;
    int32_t *vo, *v2;
    radix_sort(ka, va, kb, vb, nnz, nbits, B.hist, B.hoff, B.sws, st, &ko, &vo);
    uint32_t *kx = ko == ka ? kb : ka;
    int32_t *vx = vo == va ? vb : va;
    gather_key_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, vo, rkey, kx);
    radix_sort(kx, vo, ko, vx, nnz, nbits, B.hist, B.hoff, B.sws, st, &k2, &v2);
    // the row of every sorted entry gets its own buffer: the sort buffers are reused below
    cudaMemcpyAsync(B.rs, k2, sizeof(uint32_t) * nnz, cudaMemcpyDeviceToDevice, st);
    const int32_t *order = v2;   // source entry of every sorted position (read by emit_kernel only)
    cudaMemsetAsync(rowcnt, 0, sizeof(int32_t) * n, st);
    cudaMemsetAsync(acc, 0, sizeof(unsigned long long), st);
    emit_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, order, B.rs, ckey, vv, B.col, B.val, rowcnt, acc);
    scan_exclusive(rowcnt, B.rowptr, n, B.sws, st);
    // column view for the layout: entries of every column in row order
    cudaMemsetAsync(colcnt, 0, sizeof(int32_t) * n, st);
    col_count_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, B.col, colcnt);
    scan_exclusive(colcnt, B.cptr, n, B.sws, st);
    iota_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, va);
    list_key_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, va, B.col, B.rs, 1, 0, ka);
    radix_sort(ka, va, kb, vb, nnz, nbits, B.hist, B.hoff, B.sws, st, &ko, &vo);
    cudaMemcpyAsync(B.cent, vo, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, st);
    unsigned long long bw = 0;
    cudaMemcpyAsync(&bw, acc, sizeof(bw), cudaMemcpyDeviceToHost, st);
    // host copies
    try {
        if (perm) {
            rc = download(B.perm_h, perm, n, st);
        } else {
            B.perm_h.resize(n);
            for (int32_t k = 0; k < n; ++k) B.perm_h[k] = k;
        }
        if (rc == PARS3_OK) rc = download(B.rowptr_h, static_cast<const int32_t *>(B.rowptr), static_cast<size_t>(n) + 1, st);
        if (rc == PARS3_OK) rc = download(B.col_h, static_cast<const int32_t *>(B.col), nnz, st);
        if (rc == PARS3_OK) rc = download(B.val_h, static_cast<const double *>(B.val), nnz, st);
        if (rc == PARS3_OK) rc = cuda_status(cudaStreamSynchronize(st));   // T is freed next
    } catch (const std::bad_alloc &) {
        return PARS3_ENOMEM;
    }
    B.bw = static_cast<int64_t>(bw);
    return rc;
}

// The cut-dependent stages for the cut (prm.T, prm.W): classes, tile lists
// in (tile, col, position) order, outer lists, then the device layout on the
// GPU.  prm is normalized and its cut valid.
int base_cut(DevBase &B, const pars3_split_params &prm, pars3_handle **out, cudaStream_t st) {
    const int n = B.n, nnz = B.nnz, T = prm.T, W = prm.W;
    const int ntiles = n > 0 ? (n + T - 1) / T : 0;
    const int G = kThreads;
    const int nbits = bits_for(n);
    int rc;
    Scratch S;
    uint8_t *cls = S.get<uint8_t>(nnz);
    int32_t *mflag = S.get<int32_t>(nnz), *oflag = S.get<int32_t>(nnz);
    int32_t *mpre = S.get<int32_t>(static_cast<size_t>(nnz) + 1), *opre = S.get<int32_t>(static_cast<size_t>(nnz) + 1);
    int32_t *tcnt = S.get<int32_t>(ntiles), *tile_ptr = S.get<int32_t>(static_cast<size_t>(ntiles) + 1);
    int32_t *mlist = S.get<int32_t>(nnz), *olist = S.get<int32_t>(nnz);
    unsigned long long *acc = S.get<unsigned long long>(3);
    if (S.err() != cudaSuccess) return PARS3_ENOMEM;
    cudaMemsetAsync(tcnt, 0, sizeof(int32_t) * ntiles, st);
    cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 3, st);
    classify_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, T, W, B.rs, B.col, cls, mflag, oflag, tcnt, acc);
    scan_exclusive(mflag, mpre, nnz, B.sws, st);
    scan_exclusive(oflag, opre, nnz, B.sws, st);
    scan_exclusive(tcnt, tile_ptr, ntiles, B.sws, st);
    compact_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, mflag, mpre, mlist);
    compact_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, oflag, opre, olist);
    int32_t M = 0, O = 0;
    unsigned long long cnt3[3] = {0, 0, 0};
    cudaMemcpyAsync(&M, mpre + nnz, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&O, opre + nnz, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if ((rc = fetch(cnt3, acc, sizeof(cnt3), st)) != PARS3_OK) return rc;
    // middle list: positions (in order), stably by column, then stably by tile
    uint32_t *ka = B.ka, *kb = B.kb, *ko, *k2;
    int32_t *va = B.va, *vb = B.vb, *vo, *v2;
    cudaMemcpyAsync(va, mlist, sizeof(int32_t) * M, cudaMemcpyDeviceToDevice, st);
    list_key_kernel<<<grid_for(M, G), G, 0, st>>>(M, va, B.col, B.rs, T, 0, ka);
    radix_sort(ka, va, kb, vb, M, nbits, B.hist, B.hoff, B.sws, st, &ko, &vo);
    uint32_t *kx = ko == ka ? kb : ka;
    int32_t *vx = vo == va ? vb : va;
    list_key_kernel<<<grid_for(M, G), G, 0, st>>>(M, vo, B.col, B.rs, T, 1, kx);
    radix_sort(kx, vo, ko, vx, M, bits_for(ntiles), B.hist, B.hoff, B.sws, st, &k2, &v2);
    // the tile lists get their own buffer: the sort buffers are reused below
    int32_t *tile_list = S.get<int32_t>(M), *outer_csc = S.get<int32_t>(O);
    if (S.err() != cudaSuccess) return PARS3_ENOMEM;
    cudaMemcpyAsync(tile_list, v2, sizeof(int32_t) * M, cudaMemcpyDeviceToDevice, st);
    // outer lists: in position order (CSR), and stably by column (CSC)
    cudaMemcpyAsync(va, olist, sizeof(int32_t) * O, cudaMemcpyDeviceToDevice, st);
    list_key_kernel<<<grid_for(O, G), G, 0, st>>>(O, va, B.col, B.rs, T, 0, ka);
    radix_sort(ka, va, kb, vb, O, nbits, B.hist, B.hoff, B.sws, st, &ko, &vo);
    cudaMemcpyAsync(outer_csc, vo, sizeof(int32_t) * O, cudaMemcpyDeviceToDevice, st);
    pars3_handle *h = nullptr;
    try {
        h = new pars3_handle();
    } catch (const std::bad_alloc &) {
        return PARS3_ENOMEM;
    }
    std::unique_ptr<pars3_handle> hold(h);
    // the handle: canonical arrays, then the layout built on the GPU
    try {
        h->n = n;
        h->nnz = nnz;
        h->dtypes = prm.dtypes;
        h->symmetric = B.sym;
        h->T = T;
        h->W = W;
        h->ntiles = ntiles;
        h->bw = B.bw;
        for (int k = 0; k < 3; ++k) h->counts[k] = static_cast<int64_t>(cnt3[k]);
        h->perm = B.perm_h;
        h->rowptr = B.rowptr_h;
        h->col = B.col_h;
        h->val = B.val_h;
        rc = download(h->cls, static_cast<const uint8_t *>(cls), nnz, st);
        if (rc == PARS3_OK) rc = download(h->tile_ptr, static_cast<const int32_t *>(tile_ptr), static_cast<size_t>(ntiles) + 1, st);
        if (rc == PARS3_OK) rc = download(h->outer_csr, static_cast<const int32_t *>(olist), O, st);
        if (rc == PARS3_OK) rc = download(h->outer_csc, static_cast<const int32_t *>(outer_csc), O, st);
        if (rc == PARS3_OK) rc = download(h->tile_list, static_cast<const int32_t *>(tile_list), M, st);
        if (rc == PARS3_OK) rc = cuda_status(cudaStreamSynchronize(st));
        if (rc != PARS3_OK) return rc;
    } catch (const std::bad_alloc &) {
        return PARS3_ENOMEM;
    }
    set_layout_params(h, prm);
    const DevCanon C{B.rs, B.col, B.rowptr, tile_ptr, tile_list, B.val, cls, B.cptr, B.cent};
    rc = build_layout_device(h, C, st);
    if (rc != PARS3_OK) return rc;
    *out = hold.release();
    return PARS3_OK;
}

int split_device(int32_t n, const int32_t *rp, const int32_t *ci, const double *val, const int32_t *perm,
                 const pars3_split_params *p, pars3_handle **out, cudaStream_t st) {
    if (!out || n < 0 || !rp) return PARS3_EINVAL;
    *out = nullptr;
    pars3_split_params prm{};
    if (p) prm = *p;
    if (split_params_normalize(&prm) != PARS3_OK) return PARS3_EINVAL;
    DevBase B;
    int rc = base_build(B, n, rp, ci, val, perm, (prm.flags & PARS3_SPLIT_SYMMETRIC) ? 1 : 0, st);
    if (rc != PARS3_OK) return rc;
    // the cut: given, or the default rule on the reordered bandwidth
    if (prm.T == 0) {
        const int32_t wcap = (prm.dtypes & PARS3_DTYPE_BIT(PARS3_F64)) ? 1024 : 2048;
        auto_cut(B.bw, 32, wcap, 1024, &prm.T, &prm.W);
    }
    if (check_cut(prm.T, prm.W) != PARS3_OK) return PARS3_EINVAL;
    return base_cut(B, prm, out, st);
}

}  // namespace
}  // namespace pars3

extern "C" int pars3_split_device(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                                  const int32_t *perm, const pars3_split_params *p, pars3_handle **out,
                                  void *stream) {
    return pars3::split_device(n, rowptr, col, val, perm, p, out, static_cast<cudaStream_t>(stream));
}

namespace pars3 {

int devbase_create(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val, const int32_t *perm,
                   int symmetric, DevBase **out, void *stream) {
    *out = nullptr;
    DevBase *b = nullptr;
    try {
        b = new DevBase();
    } catch (const std::bad_alloc &) {
        return PARS3_ENOMEM;
    }
    const int rc = base_build(*b, n, rowptr, col, val, perm, symmetric, static_cast<cudaStream_t>(stream));
    if (rc != PARS3_OK) {
        delete b;
        return rc;
    }
    *out = b;
    return PARS3_OK;
}

int devbase_cut(DevBase *b, const pars3_split_params &p, pars3_handle **out, void *stream) {
    *out = nullptr;
    pars3_split_params prm = p;
    if (split_params_normalize(&prm) != PARS3_OK || check_cut(prm.T, prm.W) != PARS3_OK) return PARS3_EINVAL;
    if (!!(prm.flags & PARS3_SPLIT_SYMMETRIC) != !!b->sym) return PARS3_EINVAL;
    return base_cut(*b, prm, out, static_cast<cudaStream_t>(stream));
}

int64_t devbase_bandwidth(const DevBase *b) { return b->bw; }

void devbase_free(DevBase *b) { delete b; }

}  // namespace pars3
