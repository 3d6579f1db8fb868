// spmv.cu -- y = (alpha I + S) x on the device for a split handle.
//
// One launch of the tile kernel covers every row tile (block t owns rows
// [tT, tT+T), Sec. 3: block-row ownership, Fig. 2) plus one block per chunk
// of a long row; a second, small launch folds the cross-tile (halo) mirrored
// sums and the long-row partial sums into y in a fixed order.  No atomics:
// every y entry is written by one thread, and every sum runs in an order
// fixed by the layout and the block size, so results are bitwise
// reproducible.
//
// Tile kernel, block t:
//  1. TMA: a 1-D bulk copy stages the x window [tT-W, tT+T) into shared
//     memory (the x slice a row block needs, Sec. 3.1.2; the paper ships it
//     between MPI ranks, here it comes from HBM through the copy engine);
//  2. half pass: each middle entry l_ij of the tile is read once (Eqs. 2-6):
//     l_ij x_j is summed into row i, and the mirrored product l_ij x_i is kept
//     in shared memory;
//  3. full pass: outer rows (both triangles stored) are plain gathers;
//  4. the mirrored products are summed per column in the (column, row) order
//     of the canonical tile list: columns inside the tile complete their row,
//     columns before the tile (conflicting, Fig. 2 R2) go to the halo list.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>

#include "devcommon.cuh"
#include "internal.h"
#include "smem_layout.h"

namespace pars3 {

template <typename VT, typename XT, typename AT>
struct SpmvArgs {
    int32_t n, T, W, ntiles, M;
    const int32_t *hoff, *hcnt;
    const uint16_t *hrp, *hcol, *hcperm;
    const VT *hval;
    const int32_t *hhoff, *hhrow;
    AT *halo;
    const int32_t *frp, *fcol;
    const VT *fval;
    const int32_t *lcbeg, *lcend, *lcol;
    const VT *lval;
    AT *lpart;
    const XT *x;
    XT *y;
    AT alpha;
    int32_t *err;
};

template <typename VT, typename XT, typename AT>
__device__ __forceinline__ void long_chunk(const SpmvArgs<VT, XT, AT> &a, int c, unsigned char *smem) {
    AT *red = reinterpret_cast<AT *>(smem);
    const int tid = threadIdx.x, P = blockDim.x;
    const int beg = a.lcbeg[c], end = a.lcend[c];
    AT acc = AT(0);
    for (int e = beg + tid; e < end; e += P)
        acc += Val<VT>::ld_stream(a.lval + e) * static_cast<AT>(__ldg(a.x + a.lcol[e]));
    red[tid] = acc;
    __syncthreads();
    for (int s = P >> 1; s > 0; s >>= 1) {
        if (tid < s) red[tid] += red[tid + s];
        __syncthreads();
    }
    if (tid == 0) a.lpart[c] = red[0];
}

template <typename VT, typename XT, typename AT>
__global__ void __launch_bounds__(kBlock) tile_kernel(const SpmvArgs<VT, XT, AT> a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, P = blockDim.x;
    const int t = blockIdx.x;
    if (t >= a.ntiles) {
        long_chunk<VT, XT, AT>(a, t - a.ntiles, smem);
        return;
    }
    const SmemLayout L = smem_layout(a.T, a.W, a.M, P, sizeof(XT), sizeof(AT), 1);
    XT *xs = reinterpret_cast<XT *>(smem + L.xs);
    AT *rowacc = reinterpret_cast<AT *>(smem + L.rowacc);
    AT *q = reinterpret_cast<AT *>(smem + L.q);
    uint16_t *hcol_s = reinterpret_cast<uint16_t *>(smem + L.hcol);
    uint16_t *cperm_s = reinterpret_cast<uint16_t *>(smem + L.cperm);
    uint16_t *hrp_s = reinterpret_cast<uint16_t *>(smem + L.hrp);
    int32_t *frp_s = reinterpret_cast<int32_t *>(smem + L.frp);
    uint16_t *cs = reinterpret_cast<uint16_t *>(smem + L.cs);
    uint16_t *ce = reinterpret_cast<uint16_t *>(smem + L.ce);
    int *carry_row = reinterpret_cast<int *>(smem + L.carry_row);
    AT *carry_val = reinterpret_cast<AT *>(smem + L.carry_val);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + L.mbar);

    const int r0 = t * a.T;
    const int r1 = min(r0 + a.T, a.n);
    const int nr = r1 - r0;
    const int wb = r0 - a.W;          // window position p <-> global index wb + p
    const int wlo = max(wb, 0);       // first staged global index
    const int nx = r1 - wlo;
    const uint32_t nbulk = (static_cast<uint32_t>(nx) * sizeof(XT)) & ~15u;

    // 1. x window through the copy engine; the <16-byte tail with plain loads
    if (tid == 0) {
        mbar_init(mbar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0 && nbulk > 0) {
        mbar_arrive_expect_tx(mbar, nbulk);
        bulk_g2s(xs + (wlo - wb), a.x + wlo, nbulk, mbar);
    }
    for (int g = wlo + static_cast<int>(nbulk / sizeof(XT)) + tid; g < r1; g += P) xs[g - wb] = a.x[g];
    // accumulators and tile metadata (overlaps the copy)
    for (int r = tid; r < nr; r += P) rowacc[r] = AT(0);
    const int tw = nr + a.W;
    for (int p = tid; p < tw; p += P) {
        cs[p] = 0;
        ce[p] = 0;
    }
    const int hb = a.hoff[t];
    const int hm = a.hcnt[t];
    const uint16_t *hrp_g = a.hrp + static_cast<size_t>(t) * (a.T + 8);
    for (int r = tid; r <= nr; r += P) hrp_s[r] = hrp_g[r];
    const int f0 = a.frp[r0];
    for (int r = tid; r <= nr; r += P) frp_s[r] = a.frp[r0 + r] - f0;
    for (int k = tid; k < hm; k += P) cperm_s[k] = a.hcperm[hb + k];
    if (nbulk > 0) mbar_wait_bounded(mbar, 0, a.err);
    __syncthreads();

    // 2. half pass: row sums and mirrored products of the middle entries
    merge_rows<AT>(hm, nr, hrp_s,
                   [&](int e, int r) -> AT {
                       const AT v = Val<VT>::ld_stream(a.hval + hb + e);
                       const uint16_t p = __ldcs(a.hcol + hb + e);
                       hcol_s[e] = p;
                       q[e] = v * static_cast<AT>(xs[r + a.W]);
                       return v * static_cast<AT>(xs[p]);
                   },
                   rowacc, carry_row, carry_val);

    // 3. full pass: outer rows, x from the window when it is there
    const int fm = frp_s[nr];
    const unsigned span = static_cast<unsigned>(r1 - wlo);
    merge_rows<AT>(fm, nr, frp_s,
                   [&](int e, int r) -> AT {
                       const int c = __ldcs(a.fcol + f0 + e);
                       const AT v = Val<VT>::ld_stream(a.fval + f0 + e);
                       const unsigned off = static_cast<unsigned>(c - wlo);
                       const AT xv = off < span ? static_cast<AT>(xs[c - wb]) : static_cast<AT>(__ldg(a.x + c));
                       return v * xv;
                   },
                   rowacc, carry_row, carry_val);

    // 4. mirrored sums per column: segment boundaries of the (col,row) list
    for (int k = tid; k < hm; k += P) {
        const int key = hcol_s[cperm_s[k]];
        if (k == 0 || hcol_s[cperm_s[k - 1]] != key) cs[key] = static_cast<uint16_t>(k);
        if (k == hm - 1 || hcol_s[cperm_s[k + 1]] != key) ce[key] = static_cast<uint16_t>(k + 1);
    }
    __syncthreads();
    for (int r = tid; r < nr; r += P) {
        const int p = r + a.W;
        AT c = AT(0);
        for (int k = cs[p]; k < ce[p]; ++k) c += q[cperm_s[k]];
        a.y[r0 + r] = static_cast<XT>((a.alpha * static_cast<AT>(xs[p]) + rowacc[r]) - c);
    }
    const int h0 = a.hhoff[t], h1 = a.hhoff[t + 1];
    for (int h = h0 + tid; h < h1; h += P) {
        const int p = a.hhrow[h] - wb;
        AT c = AT(0);
        for (int k = cs[p]; k < ce[p]; ++k) c += q[cperm_s[k]];
        a.halo[h] = -c;
    }
}

// y[row] += halo sum (each halo target once) and y[long row] += its chunk
// partial sums in chunk order.
template <typename XT, typename AT>
__global__ void __launch_bounds__(256) fold_kernel(int nhalo, const int32_t *__restrict__ hhrow,
                                                   const AT *__restrict__ halo, int nlong,
                                                   const int32_t *__restrict__ lrow,
                                                   const int32_t *__restrict__ lcptr,
                                                   const AT *__restrict__ lpart, XT *__restrict__ y) {
    const int total = nhalo + nlong;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        if (idx < nhalo) {
            const int r = hhrow[idx];
            y[r] = static_cast<XT>(static_cast<AT>(y[r]) + halo[idx]);
        } else {
            const int l = idx - nhalo;
            AT s = AT(0);
            for (int c = lcptr[l]; c < lcptr[l + 1]; ++c) s += lpart[c];
            const int r = lrow[l];
            y[r] = static_cast<XT>(static_cast<AT>(y[r]) + s);
        }
    }
}

template <typename T>
__global__ void permute_kernel(int64_t n, int k, const int32_t *__restrict__ perm, const T *__restrict__ src,
                               T *__restrict__ dst, bool inverse) {
    const int64_t total = n * k;
    for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = idx / k, c = idx - i * k;
        const int64_t o = perm[i];
        if (!inverse) dst[i * k + c] = src[o * k + c];
        else dst[o * k + c] = src[i * k + c];
    }
}

// ------------------------------------------------------------ host side

template <typename VT, typename XT, typename AT>
static int launch_typed(const pars3_handle *h, int dtype, double alpha, const void *x, void *y,
                        cudaStream_t st) {
    const Layout &L = h->L;
    const DevLayout &D = h->D;
    SpmvArgs<VT, XT, AT> a;
    a.n = h->n;
    a.T = h->T;
    a.W = h->W;
    a.ntiles = h->ntiles;
    a.M = L.max_tile_half;
    a.hoff = D.hoff;
    a.hcnt = D.hcnt;
    a.hrp = D.hrp;
    a.hcol = D.hcol;
    a.hcperm = D.hcperm;
    a.hval = static_cast<const VT *>(D.hval[dtype]);
    a.hhoff = D.hhoff;
    a.hhrow = D.hhrow;
    a.halo = static_cast<AT *>(D.halo);
    a.frp = D.frp;
    a.fcol = D.fcol;
    a.fval = static_cast<const VT *>(D.fval[dtype]);
    a.lcbeg = D.lcbeg;
    a.lcend = D.lcend;
    a.lcol = D.lcol;
    a.lval = static_cast<const VT *>(D.lval[dtype]);
    a.lpart = static_cast<AT *>(D.lpart);
    a.x = static_cast<const XT *>(x);
    a.y = static_cast<XT *>(y);
    a.alpha = static_cast<AT>(alpha);
    a.err = D.err;
    const int smem = smem_bytes_for(h, dtype);
    static std::atomic<int> configured{0};
    if (configured.load() < smem) {
        cudaError_t e = cudaFuncSetAttribute(tile_kernel<VT, XT, AT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kSmemLimit);
        if (e != cudaSuccess) return cuda_status(e);
        configured.store(kSmemLimit);
    }
    const int nchunks = static_cast<int>(L.lcbeg.size());
    const int grid = h->ntiles + nchunks;
    if (grid > 0) tile_kernel<VT, XT, AT><<<grid, kBlock, smem, st>>>(a);
    const int nhalo = static_cast<int>(L.hhrow.size());
    const int nlong = static_cast<int>(L.lrow.size());
    if (nhalo + nlong > 0) {
        const int blocks = static_cast<int>(std::min<int64_t>((nhalo + nlong + 255) / 256, 152 * 8));
        fold_kernel<XT, AT><<<blocks, 256, 0, st>>>(nhalo, D.hhrow, static_cast<const AT *>(D.halo), nlong, D.lrow,
                                                    D.lcptr, static_cast<const AT *>(D.lpart), static_cast<XT *>(y));
    }
    return cuda_status(cudaGetLastError());
}

int launch_spmv(const pars3_handle *h, int dtype, double alpha, int k, const void *x, void *y, void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (k != 1) return PARS3_EUNSUPPORTED;
    switch (dtype) {
        case PARS3_F64: return launch_typed<double, double, double>(h, dtype, alpha, x, y, st);
        case PARS3_F32: return launch_typed<float, float, float>(h, dtype, alpha, x, y, st);
        case PARS3_BF16: return launch_typed<uint16_t, float, float>(h, dtype, alpha, x, y, st);
        default: return PARS3_EINVAL;
    }
}

int launch_permute(const pars3_handle *h, int dtype, int k, const void *src, void *dst, bool inverse,
                   void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t total = static_cast<int64_t>(h->n) * k;
    if (total == 0) return PARS3_OK;
    const int blocks = static_cast<int>(std::min<int64_t>((total + 255) / 256, 152 * 16));
    if (dtype == PARS3_F64)
        permute_kernel<double><<<blocks, 256, 0, st>>>(h->n, k, h->D.perm, static_cast<const double *>(src),
                                                       static_cast<double *>(dst), inverse);
    else
        permute_kernel<float><<<blocks, 256, 0, st>>>(h->n, k, h->D.perm, static_cast<const float *>(src),
                                                      static_cast<float *>(dst), inverse);
    return cuda_status(cudaGetLastError());
}

}  // namespace pars3
