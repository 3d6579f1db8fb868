// spmv_kernels.cuh -- device code of the skew product, shared by the
// operator (spmv.cu) and the MRS solver (mrs.cu, which runs the same tile
// kernel in its Lanczos mode).
//
// Two launches per product: the tile kernel (one block per row tile -- the
// block-row ownership of Sec. 3 and Fig. 2 -- after the blocks that sum the
// pieces of long rows) and a small fold kernel that adds the cross-tile
// (halo) mirrored sums and the long-row piece sums to y.  No atomics:
// every y entry has one writer per launch and every sum runs in an order
// fixed by the layout and the block size, so results are bitwise
// reproducible from run to run.
//
// Tile block t (rows [tT, tT+T)):
//  0. one thread issues TMA bulk copies of the x window [tT-W, tT+T) (the x
//     slice a row block needs, Sec. 3.1.2) and of the tile's middle entries
//     (values, window columns, (column,row) order, row pointers);
//  1. meanwhile the full pass streams the tile's full-storage rows in
//     sliced-ELL order (fp32 / bf16: prefetched into L2 by the copy engine
//     at the start of the block; fp64: each warp loads the next slice's
//     columns while it sums the current one): each warp takes 32-row slices,
//     one lane per row (every row of the tile owns a lane), slot m of lane
//     l at 32m+l so that every load instruction reads 32 consecutive
//     entries; a lane's sum starts at alpha x_r and gathers x_j, eight
//     slots in flight;
//  2. half pass: each middle entry l_ij is read once and used twice (Eqs.
//     2-6): l_ij x_j is summed into row i, the mirrored product l_ij x_i is
//     kept in shared memory;
//  3. the mirrored products are summed per column in the (column, row)
//     order of the canonical tile list: columns inside the tile complete
//     their row, columns before the tile (the conflicting region R2 of
//     Fig. 2) go to the halo list that the fold adds to the previous tile.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>

#include "devcommon.cuh"
#include "internal.h"
#include "smem_layout.h"

namespace pars3 {

template <typename VT, typename XT, typename AT>
struct SpmvArgs {
    int32_t n, T, W, ntiles, Mh;
    int32_t nls, nlb, lsb;   // long-row slices, their blocks (launched before the tiles), slices per block
    const int32_t *hoff, *hcnt;
    const uint16_t *hrp, *hcol, *hcperm, *hrowc;
    const int32_t *hcsoff, *hcsn;
    const uint32_t *hcs;
    int32_t CS;         // column segment words of the largest tile
    const VT *hval;
    const int32_t *hhoff, *hhrow;
    AT *halo;
    const int32_t *sl_off, *sl_ent, *sl_e;
    const uint32_t *sl_meta;
    const int32_t *fcol;
    const VT *fval;
    const int32_t *ls_ent;
    const uint16_t *ls_len;
    const int32_t *lcol;
    const VT *lval;
    AT *lpart;
    const XT *x;
    XT *y;
    AT alpha;
    int32_t *err;
    int32_t sym;   // 1: S = L + L^T (mirrored sums added), 0: S = L - L^T (subtracted)
};

template <typename VT> __device__ __forceinline__ typename Val<VT>::acc sval(const VT *p, int e);
template <> __device__ __forceinline__ double sval<double>(const double *p, int e) { return p[e]; }
template <> __device__ __forceinline__ float sval<float>(const float *p, int e) { return p[e]; }
template <> __device__ __forceinline__ float sval<uint16_t>(const uint16_t *p, int e) { return bf16_bits_to_f32(p[e]); }

constexpr int kUnroll = 8;       // independent gathers in flight per lane
constexpr int kShortRow = 16;    // middle rows longer than this are summed by the whole warp

// Sliced-ELL row of lane l: slots base + 32 m + l (m < len) of the global
// value and column arrays, streamed (evict-first); x_j gathered.  The sum
// starts at `start`.
template <typename VT, typename XT, typename AT>
__device__ __forceinline__ AT slice_row_sum(const VT *__restrict__ val, const int32_t *__restrict__ col,
                                            int64_t base, int len, const XT *__restrict__ xg, AT start) {
    AT acc = start;
    for (int m0 = 0; m0 < len; m0 += kUnroll) {
        int c[kUnroll];
        AT v[kUnroll], xv[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            c[u] = 0;
            v[u] = AT(0);
            if (m0 + u < len) {
                const int64_t q = base + static_cast<int64_t>(m0 + u) * kSlice;
                c[u] = __ldcs(col + q);
                v[u] = Val<VT>::ld_stream(val + q);
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) xv[u] = (m0 + u < len) ? static_cast<AT>(__ldg(xg + c[u])) : AT(0);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (m0 + u < len) acc += v[u] * xv[u];
    }
    return acc;
}

// Fp64 variant of the row sum.  The fp64 pipe of this part is narrow, and an
// FMA issued for a slot that no lane of the warp holds still costs its pipe
// time (measured: on the 128^3 + 1% matrix, rounds of a fixed eight slots
// took 56 us per product, rounds sized to the slice took 48 us).  So each
// round covers exactly min(lenw - m0, 8) slots, lenw being the slice's longest
// row (warp-uniform), with lane-level predicates only for shorter rows.  The
// additions happen in the same order as above, so results are identical.
template <int C, typename VT, typename XT, typename AT>
__device__ __forceinline__ AT slice_round(const VT *__restrict__ val, const int32_t *__restrict__ col, int64_t q0,
                                          int rem, const XT *__restrict__ xg, AT acc) {
    int c[C];
    AT v[C], xv[C];
#pragma unroll
    for (int u = 0; u < C; ++u) {
        c[u] = 0;
        v[u] = AT(0);
        if (u < rem) {
            const int64_t q = q0 + static_cast<int64_t>(u) * kSlice;
            c[u] = __ldcs(col + q);
            v[u] = Val<VT>::ld_stream(val + q);
        }
    }
#pragma unroll
    for (int u = 0; u < C; ++u) xv[u] = (u < rem) ? static_cast<AT>(__ldg(xg + c[u])) : AT(0);
#pragma unroll
    for (int u = 0; u < C; ++u)
        if (u < rem) acc += v[u] * xv[u];
    return acc;
}

template <typename VT, typename XT, typename AT>
__device__ __forceinline__ AT slice_row_sum_uniform(const VT *__restrict__ val, const int32_t *__restrict__ col,
                                                    int64_t base, int len, int lenw, const XT *__restrict__ xg,
                                                    AT start) {
    static_assert(kUnroll == 8, "the rounds below assume eight slots");
    AT acc = start;
    for (int m0 = 0; m0 < lenw; m0 += kUnroll) {
        const int rem = len - m0;
        const int64_t q0 = base + static_cast<int64_t>(m0) * kSlice;
        switch (min(lenw - m0, kUnroll)) {
        case 1: acc = slice_round<1, VT, XT, AT>(val, col, q0, rem, xg, acc); break;
        case 2: acc = slice_round<2, VT, XT, AT>(val, col, q0, rem, xg, acc); break;
        case 3: acc = slice_round<3, VT, XT, AT>(val, col, q0, rem, xg, acc); break;
        case 4: acc = slice_round<4, VT, XT, AT>(val, col, q0, rem, xg, acc); break;
        case 5: acc = slice_round<5, VT, XT, AT>(val, col, q0, rem, xg, acc); break;
        case 6: acc = slice_round<6, VT, XT, AT>(val, col, q0, rem, xg, acc); break;
        case 7: acc = slice_round<7, VT, XT, AT>(val, col, q0, rem, xg, acc); break;
        default: acc = slice_round<8, VT, XT, AT>(val, col, q0, rem, xg, acc); break;
        }
    }
    return acc;
}

// First-round columns (slots < kUnroll) of a sliced-ELL row of length len.
__device__ __forceinline__ void slice_cols(const int32_t *__restrict__ col, int64_t base, int len,
                                           int (&c)[kUnroll]) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) c[u] = (u < len) ? __ldcs(col + base + static_cast<int64_t>(u) * kSlice) : 0;
}

// The additions of one round, slots [0, C), in slot order.
template <int C, typename AT>
__device__ __forceinline__ AT slot_sums(const AT (&v)[kUnroll], const AT (&xv)[kUnroll], int rem, AT acc) {
#pragma unroll
    for (int u = 0; u < C; ++u)
        if (u < rem) acc += v[u] * xv[u];
    return acc;
}

// Fp64 full pass of one warp over slices sb, sb + step, ... (< s1).  The
// columns of the next slice's first round are loaded while the current slice
// is summed, so a slice waits on one round trip (values and x gathers
// together) instead of two (columns, then x).  The sums are those of
// slice_row_sum_uniform, in the same order.  Measured per product: 47.9 ->
// 46.2 us on the 128^3 + 1 % matrix, 40.3 -> 37.1 us on the 2048 x 1024 grid.
template <typename VT, typename XT, typename AT, class Epi>
__device__ __forceinline__ void full_pass_pipelined(const int32_t *__restrict__ sl_ent,
                                                    const uint32_t *__restrict__ sl_meta,
                                                    const VT *__restrict__ val, const int32_t *__restrict__ col,
                                                    int sb, int s1, int step, int r0, const XT *__restrict__ xg,
                                                    Epi &epi, AT *rowacc, bool direct) {
    const int lane = threadIdx.x & 31;
    uint32_t meta = 0xffffu;
    int ent = 0;
    if (sb < s1) {
        meta = __ldg(sl_meta + static_cast<int64_t>(sb) * kSlice + lane);
        ent = __ldg(sl_ent + sb);
    }
    int len = (meta & 0xffffu) != 0xffffu ? static_cast<int>(meta >> 16) : 0;
    int c[kUnroll];
    slice_cols(col, static_cast<int64_t>(ent) + lane, len, c);
    for (int s = sb; s < s1; s += step) {
        // the next slice's metadata arrives while this slice's gathers do
        uint32_t meta_n = 0xffffu;
        int ent_n = 0;
        if (s + step < s1) {
            meta_n = __ldg(sl_meta + static_cast<int64_t>(s + step) * kSlice + lane);
            ent_n = __ldg(sl_ent + s + step);
        }
        const int rl = static_cast<int>(meta & 0xffffu);
        const int lenw = __reduce_max_sync(0xffffffffu, len);
        const int64_t q0 = static_cast<int64_t>(ent) + lane;
        AT v[kUnroll], xv[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            v[u] = AT(0);
            xv[u] = AT(0);
            if (u < len) {
                v[u] = Val<VT>::ld_stream(val + q0 + static_cast<int64_t>(u) * kSlice);
                xv[u] = static_cast<AT>(__ldg(xg + c[u]));
            }
        }
        const AT start = rl != 0xffff ? epi.start(xg, r0 + rl) : AT(0);
        const int len_n = (meta_n & 0xffffu) != 0xffffu ? static_cast<int>(meta_n >> 16) : 0;
        slice_cols(col, static_cast<int64_t>(ent_n) + lane, len_n, c);
        AT acc = start;
        switch (min(lenw, kUnroll)) {
        case 0: break;
        case 1: acc = slot_sums<1, AT>(v, xv, len, acc); break;
        case 2: acc = slot_sums<2, AT>(v, xv, len, acc); break;
        case 3: acc = slot_sums<3, AT>(v, xv, len, acc); break;
        case 4: acc = slot_sums<4, AT>(v, xv, len, acc); break;
        case 5: acc = slot_sums<5, AT>(v, xv, len, acc); break;
        case 6: acc = slot_sums<6, AT>(v, xv, len, acc); break;
        case 7: acc = slot_sums<7, AT>(v, xv, len, acc); break;
        default: acc = slot_sums<8, AT>(v, xv, len, acc); break;
        }
        for (int m0 = kUnroll; m0 < lenw; m0 += kUnroll) {   // rows longer than one round
            const int rem = len - m0;
            const int64_t qm = q0 + static_cast<int64_t>(m0) * kSlice;
            switch (min(lenw - m0, kUnroll)) {
            case 1: acc = slice_round<1, VT, XT, AT>(val, col, qm, rem, xg, acc); break;
            case 2: acc = slice_round<2, VT, XT, AT>(val, col, qm, rem, xg, acc); break;
            case 3: acc = slice_round<3, VT, XT, AT>(val, col, qm, rem, xg, acc); break;
            case 4: acc = slice_round<4, VT, XT, AT>(val, col, qm, rem, xg, acc); break;
            case 5: acc = slice_round<5, VT, XT, AT>(val, col, qm, rem, xg, acc); break;
            case 6: acc = slice_round<6, VT, XT, AT>(val, col, qm, rem, xg, acc); break;
            case 7: acc = slice_round<7, VT, XT, AT>(val, col, qm, rem, xg, acc); break;
            default: acc = slice_round<8, VT, XT, AT>(val, col, qm, rem, xg, acc); break;
            }
        }
        if (rl != 0xffff) {
            if (direct) epi.finish(r0 + rl, acc);
            else rowacc[rl] = acc;
        }
        meta = meta_n;
        ent = ent_n;
        len = len_n;
    }
}

// Half-storage row of the middle part: sum_j l_rj x_j over its staged
// entries e0 .. e1-1, x_j from the staged window (one thread, or the whole
// warp for long rows).
template <typename VT, typename XT, typename AT>
__device__ __forceinline__ AT half_row_thread(int e0, int e1, const VT *hval, const uint16_t *hcol, const XT *xs) {
    AT acc = AT(0);
    for (int e = e0; e < e1; ++e) acc += sval<VT>(hval, e) * static_cast<AT>(xs[hcol[e]]);
    return acc;
}

template <typename VT, typename XT, typename AT>
__device__ __forceinline__ AT half_row_warp(int e0, int e1, const VT *hval, const uint16_t *hcol, const XT *xs) {
    const int lane = threadIdx.x & 31;
    AT acc = AT(0);
    for (int e = e0 + lane; e < e1; e += 32) acc += sval<VT>(hval, e) * static_cast<AT>(xs[hcol[e]]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

// Mirrored sum of one column: sum_i l_ij x_i over the column's entries, in
// (column, row) order k0 .. k1-1: the staged value of entry cperm[k] and
// x_i at the window position hrowc[k] of its row -- one FMA per entry, the
// value read a second time from shared memory instead of a stored product.
template <typename VT, typename XT, typename AT>
__device__ __forceinline__ AT half_col_sum(int k0, int k1, const VT *hval, const uint16_t *cperm,
                                           const uint16_t *hrowc, const XT *xs) {
    AT acc = AT(0);
    for (int k = k0; k < k1; ++k) acc += sval<VT>(hval, cperm[k]) * static_cast<AT>(xs[hrowc[k]]);
    return acc;
}

// Row epilogues of the tile block.  Plain product: a row sum starts at
// alpha x_r and is stored as y_r.  PIPE: fp64 tiles load the next slice's
// columns ahead (full_pass_pipelined); the batched kernel, which also holds
// the SpMM path, turns it off to stay within its registers.
template <typename XT, typename AT, bool PIPE = true>
struct EpiSpmv {
    static constexpr bool kStage = false;   // reads no vectors at the end of the tile
    static constexpr bool kPipelined = PIPE;
    static constexpr bool kDirect = true;     // finish() only stores y
    AT alpha;
    XT *y;
    __device__ __forceinline__ AT start(const XT *__restrict__ x, int r) const {
        return alpha * static_cast<AT>(__ldg(x + r));
    }
    __device__ __forceinline__ void finish(int r, AT v) { y[r] = static_cast<XT>(v); }
    __device__ __forceinline__ void invalid(int r) { y[r] = static_cast<XT>(CUDART_NAN); }
    __device__ __forceinline__ void end_block(int, double *) {}
    __device__ __forceinline__ void bind(int, int, unsigned char *) {}
    __device__ __forceinline__ uint32_t stage_bytes(int, int) const { return 0u; }
    __device__ __forceinline__ void stage_issue(int, int, unsigned char *, uint64_t *) {}
    __device__ __forceinline__ void stage_tail(int, int, unsigned char *, int, int) {}
};

// fp64 scalars of the MRS recurrence, kept on the device.  Per-iteration
// values sit in rings of four indexed by j & 3.
struct MrsState {
    double beta[4], rho[4], c[4], s[4], tau[4];
    double gamma;      // gamma_{j+1}
    double t;          // t_{j+1}
    double alpha, tol;
    // epilogue coefficients of the next iteration (see mrs_next_coeffs)
    double e_scale, e_coef, e_inv_b2, e_r3, e_inv_rho, e_tau;
    int32_t j;         // last completed iteration
    int32_t jmax, done, pad;
    uint32_t ticket, pad2;
};

// Scalars of iteration j = st->j + 1, computed once by the thread that
// finished iteration j - 1 (fp64 division is costly on this part, so no
// other thread repeats them, and the step reuses reciprocals it already
// has): w_j = raw / beta_{j-1} + (beta_{j-1} / beta_{j-2}) w_{j-2}; lagged
// p_{j-1} = (w_{j-2} / beta_{j-2} - R[j-3,j-1] p_{j-3}) / rho_{j-1} with
// R[j-3,j-1] = -s_{j-3} beta_{j-2}; x += tau_{j-1} p_{j-1}.  inv_rho is
// 1 / rho_{j-1} (unused for j = 1); the previous e_scale is 1 / beta_{j-2}.
__device__ __forceinline__ void mrs_next_coeffs(MrsState *st, double inv_rho) {
    const int j = st->j + 1;
    const double b1 = st->beta[(j - 1) & 3];
    const double b2 = j >= 2 ? st->beta[(j - 2) & 3] : 1.0;
    const double inv_b2 = j >= 2 ? st->e_scale : 1.0;
    st->e_scale = 1.0 / b1;
    st->e_coef = j >= 2 ? b1 * inv_b2 : 0.0;
    st->e_inv_b2 = inv_b2;
    st->e_r3 = j >= 4 ? -st->s[(j - 3) & 3] * b2 : 0.0;
    st->e_inv_rho = j >= 2 ? inv_rho : 0.0;
    st->e_tau = j >= 2 ? st->tau[(j - 1) & 3] : 0.0;
}

// deterministic block sum of one double per thread (warp butterflies, then
// warps in order)
__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < nw; ++w) s += red[w];
    return s;   // valid on thread 0
}

// Last block of a grid to arrive: sums part[0..count) in a fixed order.
// Returns true (on every thread of that block) and leaves the sum in *out
// (thread 0).  Each block's partial was written by its thread 0, which
// makes it visible device-wide before taking a ticket.
__device__ __forceinline__ bool last_block_sum(unsigned *ticket, const double *part, int count, double *red,
                                               double *out) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double v = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) v += __ldcg(part + i);
    const double s = block_sum(v, red);
    if (threadIdx.x == 0) {
        *out = s;
        *ticket = 0u;
    }
    return true;
}


// One step of the scalar recurrence after iteration j's norm ||w_j||^2 = tot
// is known (one thread): beta_j, the Givens rotation, tau_j, t_{j+1},
// gamma_{j+1}, the stop test and the next iteration's epilogue scalars; in a
// graph, the while-node condition.
__device__ __forceinline__ void mrs_step(MrsState *st, double tot, cudaGraphConditionalHandle cond, int in_graph) {
    const int j = st->j + 1;
    const double beta = sqrt(tot);
    const double gam = st->gamma;
    const double rho = hypot(gam, beta);
    const double inv_rho = 1.0 / rho;
    const double c = gam * inv_rho, s = beta * inv_rho;
    const int k = j & 3;
    st->beta[k] = beta;
    st->rho[k] = rho;
    st->c[k] = c;
    st->s[k] = s;
    st->tau[k] = c * st->t;
    const double tn = -s * st->t;
    st->t = tn;
    st->gamma = st->alpha / c;
    st->j = j;
    const int done = (fabs(tn) <= st->tol) || (beta == 0.0) || (j >= st->jmax);
    st->done = done;
    mrs_next_coeffs(st, inv_rho);   // also the final lagged update uses them
    if (in_graph) cudaGraphSetConditional(cond, done ? 0u : 1u);
}

// Epilogue parameters of one MRS iteration, written to shared memory by the
// first thread of each block: the epilogue reads them there when a row
// finishes, so none of them occupies registers during the full pass (which
// therefore keeps the fp64 look-ahead of the plain product).
template <typename XT, typename AT>
struct MrsEpiParams {
    XT *y;
    const XT *wpp, *pold;
    XT *pnew, *xsol;
    const uint32_t *fold_bits;
    double *part;
    AT scale, coef, c_w, c_p, tau;   // c_w = 1 / (beta_{j-2} rho_{j-1}), c_p = R[j-3,j-1] / rho_{j-1}
    int lag;
};

template <typename XT, typename AT, bool S>
struct EpiMrs {
    // With S, the tile's slices of w_{j-2}, p_{j-3} and x are bulk-copied
    // into shared memory at the start of the block (with the other staged
    // data), so the epilogue reads them without a round trip to HBM at the
    // end; without S (tiles too large for the extra shared memory) they are
    // read from global memory.
    static constexpr bool kStage = S;
    static constexpr bool kPipelined = true;
    // unstaged, a lane can finish its row as soon as it has the sum (the
    // vectors come from global memory); staged, only after the copies land
    static constexpr bool kDirect = !S;
    const MrsEpiParams<XT, AT> *p;            // shared memory
    unsigned char *area;                      // staged slices
    double nrm;
    int r0, T;
    static PARS3_HD uint32_t slice_bytes(int T) {
        return (static_cast<uint32_t>(T) * sizeof(XT) + 127u) & ~127u;
    }
    __device__ __forceinline__ const XT *s_wpp() const {
        return S ? reinterpret_cast<const XT *>(area) : p->wpp + r0;
    }
    __device__ __forceinline__ const XT *s_pold() const {
        return S ? reinterpret_cast<const XT *>(area + slice_bytes(T)) : p->pold + r0;
    }
    __device__ __forceinline__ const XT *s_x() const {
        return S ? reinterpret_cast<const XT *>(area + 2u * slice_bytes(T)) : p->xsol + r0;
    }
    // bytes the bulk copies move (16-byte multiple of each slice)
    __device__ __forceinline__ uint32_t stage_bytes(int, int nr) const {
        const uint32_t b = (static_cast<uint32_t>(nr) * sizeof(XT)) & ~15u;
        return (p->lag ? 3u : 1u) * b;
    }
    __device__ __forceinline__ void bind(int rr0, int TT, unsigned char *ar) {
        r0 = rr0;
        T = TT;
        area = ar;
    }
    __device__ __forceinline__ void stage_issue(int rr0, int nr, unsigned char *, uint64_t *mbar) {
        const uint32_t b = (static_cast<uint32_t>(nr) * sizeof(XT)) & ~15u;
        if (b == 0) return;
        bulk_g2s(const_cast<XT *>(s_wpp()), p->wpp + rr0, b, mbar);
        if (p->lag) {
            bulk_g2s(const_cast<XT *>(s_pold()), p->pold + rr0, b, mbar);
            bulk_g2s(const_cast<XT *>(s_x()), p->xsol + rr0, b, mbar);
        }
    }
    // rows past the last 16-byte boundary of the slice: plain loads
    __device__ __forceinline__ void stage_tail(int rr0, int nr, unsigned char *, int tid, int P) {
        const int first = static_cast<int>(((static_cast<uint32_t>(nr) * sizeof(XT)) & ~15u) / sizeof(XT));
        for (int q = first + tid; q < nr; q += P) {
            const_cast<XT *>(s_wpp())[q] = p->wpp[rr0 + q];
            if (p->lag) {
                const_cast<XT *>(s_pold())[q] = p->pold[rr0 + q];
                const_cast<XT *>(s_x())[q] = p->xsol[rr0 + q];
            }
        }
    }
    __device__ __forceinline__ AT start(const XT *__restrict__, int) const { return AT(0); }
    __device__ __forceinline__ void finish(int r, AT raw) {
        const int q = r - r0;
        AT w = raw * p->scale;
        const AT wp = static_cast<AT>(s_wpp()[q]);
        if (p->coef != AT(0)) w += p->coef * wp;
        const XT wx = static_cast<XT>(w);
        p->y[r] = wx;
        if (!((__ldg(p->fold_bits + (r >> 5)) >> (r & 31)) & 1u))
            nrm += static_cast<double>(wx) * static_cast<double>(wx);
        if (p->lag) {
            // p_{j-1} = (w_{j-2} / beta_{j-2} - R[j-3,j-1] p_{j-3}) / rho_{j-1}, with both
            // quotients folded into the two coefficients once per iteration
            const AT pv = wp * p->c_w - p->c_p * static_cast<AT>(s_pold()[q]);
            p->pnew[r] = static_cast<XT>(pv);
            p->xsol[r] = static_cast<XT>(static_cast<AT>(s_x()[q]) + p->tau * pv);
        }
    }
    // an output that could not be computed (the norm then is NaN as well)
    __device__ __forceinline__ void invalid(int r) {
        p->y[r] = static_cast<XT>(CUDART_NAN);
        nrm = CUDART_NAN;
    }
    // fixed-order block sum of the thread norms into part[t]
    __device__ __forceinline__ void end_block(int t, double *red) {
        double v = nrm;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[warp] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += red[w];
            p->part[t] = s;
        }
    }
};

// The parameters of iteration j = st->j + 1 (one thread); *xop is the
// operand w_{j-1}.
template <typename XT, typename AT>
__device__ __forceinline__ void fill_mrs_params(MrsEpiParams<XT, AT> *e, const MrsState *st, XT *const *wr,
                                                XT *const *pr, XT *xsol, const uint32_t *fold_bits, double *part) {
    const int j = st->j + 1;
    e->y = wr[j % 3];
    e->wpp = wr[(j + 1) % 3];
    e->pold = pr[j % 3];
    e->pnew = pr[(j + 2) % 3];
    e->xsol = xsol;
    e->fold_bits = fold_bits;
    e->part = part;
    e->scale = static_cast<AT>(st->e_scale);
    e->coef = static_cast<AT>(st->e_coef);
    e->lag = j >= 2;
    e->c_w = static_cast<AT>(st->e_inv_b2 * st->e_inv_rho);
    e->c_p = static_cast<AT>(st->e_r3 * st->e_inv_rho);
    e->tau = static_cast<AT>(st->e_tau);
}

// L2 prefetch of slices [s0, s1): their values, columns and metadata.  A
// slice's entries start at a multiple of 32 slots, so every range starts and
// ends on a 16-byte boundary.  At most kTilePrefetch bytes of values (and the
// matching columns) are requested, so that the blocks resident at one time
// cannot claim more than a fraction of L2.
//
// Used for fp32 and bf16 values, where it measured 10-14 % faster on the
// 128^3 + 1 % and 2048 x 1024 grid matrices.  For fp64 it measured 5-17 %
// slower on those two (with or without an evict-first policy, at 16 KB to
// 256 KB per tile; 2-3 % faster on R-MAT), so fp64 tiles instead load the
// next slice's columns ahead in registers (full_pass_pipelined).
constexpr int64_t kTilePrefetch = 256 << 10;
template <typename AT>
constexpr bool tile_prefetch() { return sizeof(AT) == 4; }
template <typename VT, typename XT, typename AT>
__device__ __forceinline__ void prefetch_slices(const SpmvArgs<VT, XT, AT> &a, int s0, int s1) {
    const int64_t e0 = a.sl_ent[s0], e1 = a.sl_ent[s1];
    const int64_t ne = min(e1 - e0, kTilePrefetch / static_cast<int64_t>(sizeof(VT)));
    if (ne > 0) {
        bulk_prefetch_l2(a.fval + e0, static_cast<uint64_t>(ne) * sizeof(VT));
        bulk_prefetch_l2(a.fcol + e0, static_cast<uint64_t>(ne) * 4u);
    }
    bulk_prefetch_l2(a.sl_meta + static_cast<int64_t>(s0) * kSlice, static_cast<uint64_t>(s1 - s0) * kSlice * 4u);
}

// LA: fp32 / bf16 tiles use the fp64 tiles' look-ahead full pass and
// direct stores (the kernel variant compiled for two blocks per SM, whose
// registers hold them)
template <typename VT, typename XT, typename AT, class Epi, bool LA = false>
__device__ __forceinline__ void tile_block(const SpmvArgs<VT, XT, AT> &a, int t, unsigned char *smem,
                                           const XT *__restrict__ xop, Epi &epi) {
    const SmemLayout L = smem_layout(a.T, a.W, a.Mh, a.CS, sizeof(VT), sizeof(XT), sizeof(AT));
    XT *xs = reinterpret_cast<XT *>(smem + L.xs);
    AT *rowacc = reinterpret_cast<AT *>(smem + L.rowacc);
    AT *colacc = reinterpret_cast<AT *>(smem + L.colacc);
    VT *hval = reinterpret_cast<VT *>(smem + L.hval);
    uint16_t *hcol = reinterpret_cast<uint16_t *>(smem + L.hcol);
    uint16_t *cperm = reinterpret_cast<uint16_t *>(smem + L.cperm);
    uint16_t *hrowc = reinterpret_cast<uint16_t *>(smem + L.hrowc);
    uint16_t *hrp = reinterpret_cast<uint16_t *>(smem + L.hrp);
    uint32_t *hcs = reinterpret_cast<uint32_t *>(smem + L.hcs);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + L.mbar);
    const int tid = threadIdx.x, P = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = P >> 5;
    const int r0 = t * a.T, r1 = min(r0 + a.T, a.n), nr = r1 - r0;
    const int wb = r0 - a.W, wlo = max(wb, 0);
    const uint32_t nbulk = (static_cast<uint32_t>(r1 - wlo) * sizeof(XT)) & ~15u;
    const int hb = a.hoff[t], hm = a.hcnt[t];
    const uint32_t hmp = static_cast<uint32_t>((hm + kAlignHalf - 1) / kAlignHalf * kAlignHalf);
    const uint32_t rpb = static_cast<uint32_t>(a.T + 8) * 2u;
    const int cs0 = a.hcsoff[t];
    const uint32_t csb = static_cast<uint32_t>(a.hcsoff[t + 1] - cs0) * 4u;

    // 0. with fp32 / bf16 values the copy engine prefetches the tile's
    // sliced-ELL rows into L2 (the warps' loads then wait on L2, not on HBM);
    // it stages the x window and the middle entries (a tile without middle
    // entries needs neither) and the vectors the epilogue reads (Lanczos mode)
    const int s0 = a.sl_off[t], s1 = a.sl_off[t + 1];
    if (tile_prefetch<AT>() && tid == P - 1 && s1 > s0) prefetch_slices(a, s0, s1);
    const bool stage_half = hm > 0;
    const bool staged = stage_half || Epi::kStage;   // block-uniform
    // A tile without middle entries whose epilogue only stores y: each lane
    // stores its row's sum as soon as it has it, and the block needs neither
    // the row sums in shared memory nor a barrier.  fp64 only: with fp32 /
    // bf16 the three-blocks-per-SM register budget would spill.
    const bool direct = (sizeof(AT) == 8 || LA) && !staged && Epi::kDirect;
    epi.bind(r0, a.T, smem + align128(L.total));
    if (staged && tid == 0) {
        mbar_init(mbar, 1);
        fence_mbar_init();
        uint32_t tx = epi.stage_bytes(r0, nr);
        if (stage_half) tx += nbulk + rpb + hmp * (sizeof(VT) + 6u) + csb;
        mbar_arrive_expect_tx(mbar, tx);
        if (stage_half) {
            if (nbulk > 0) bulk_g2s(xs + (wlo - wb), xop + wlo, nbulk, mbar);
            bulk_g2s(hrp, a.hrp + static_cast<size_t>(t) * (a.T + 8), rpb, mbar);
            bulk_g2s(hval, a.hval + hb, hmp * sizeof(VT), mbar);
            bulk_g2s(hcol, a.hcol + hb, hmp * 2u, mbar);
            bulk_g2s(cperm, a.hcperm + hb, hmp * 2u, mbar);
            bulk_g2s(hrowc, a.hrowc + hb, hmp * 2u, mbar);
            bulk_g2s(hcs, a.hcs + cs0, csb, mbar);
        }
        if constexpr (Epi::kStage) epi.stage_issue(r0, nr, smem + align128(L.total), mbar);
    }
    if (stage_half) {
        for (int g = wlo + static_cast<int>(nbulk / sizeof(XT)) + tid; g < r1; g += P) xs[g - wb] = xop[g];
        for (int r = tid; r < nr; r += P) colacc[r] = AT(0);
    }
    if constexpr (Epi::kStage) epi.stage_tail(r0, nr, smem + align128(L.total), tid, P);
    __syncthreads();   // the barrier is initialised before anyone waits on it

    const int se = a.sl_e[t];
    // rows without full-path entries (the slices se .. s1-1, width 0: on a
    // power-law graph most rows of a tile): their start value, by all
    // threads at once with coalesced metadata loads, instead of a warp per
    // slice
    for (int q = tid; q < (s1 - se) * kSlice; q += P) {
        const uint32_t meta = __ldg(a.sl_meta + static_cast<int64_t>(se) * kSlice + q);
        const int rl = static_cast<int>(meta & 0xffffu);
        if (rl != 0xffff) {
            const AT v0 = epi.start(xop, r0 + rl);
            if (direct) epi.finish(r0 + rl, v0);
            else rowacc[rl] = v0;
        }
    }
    // 1. full pass (sliced ELL) while the copy runs, over the slices that
    // hold entries (s0 .. se-1)
    if constexpr ((sizeof(AT) == 8 || LA) && Epi::kPipelined) {
        full_pass_pipelined<VT, XT, AT, Epi>(a.sl_ent, a.sl_meta, a.fval, a.fcol, s0 + warp, se, nwarps, r0, xop,
                                             epi, rowacc, direct);
    } else {
        // the next slice's metadata is fetched while the current one runs
        int s = s0 + warp;
        uint32_t meta_n = 0u;
        int ent_n = 0;
        if (s < se) {
            meta_n = __ldg(a.sl_meta + static_cast<int64_t>(s) * kSlice + lane);
            ent_n = __ldg(a.sl_ent + s);
        }
        for (; s < se; s += nwarps) {
            const uint32_t meta = meta_n;
            const int ent = ent_n;
            if (s + nwarps < se) {
                meta_n = __ldg(a.sl_meta + static_cast<int64_t>(s + nwarps) * kSlice + lane);
                ent_n = __ldg(a.sl_ent + s + nwarps);
            }
            const int rl = static_cast<int>(meta & 0xffffu);
            if constexpr (sizeof(AT) == 8) {
                const int len = rl != 0xffff ? static_cast<int>(meta >> 16) : 0;
                const int lenw = __reduce_max_sync(0xffffffffu, len);
                const AT start = rl != 0xffff ? epi.start(xop, r0 + rl) : AT(0);
                const AT sum = slice_row_sum_uniform<VT, XT, AT>(a.fval, a.fcol, static_cast<int64_t>(ent) + lane,
                                                                 len, lenw, xop, start);
                if (rl != 0xffff) {
                    if (direct) epi.finish(r0 + rl, sum);
                    else rowacc[rl] = sum;
                }
            } else {
                const int len = static_cast<int>(meta >> 16);
                if (rl != 0xffff) {
                    const AT start = epi.start(xop, r0 + rl);
                    const AT sum = slice_row_sum<VT, XT, AT>(a.fval, a.fcol, static_cast<int64_t>(ent) + lane, len,
                                                           xop, start);
                    if (direct) epi.finish(r0 + rl, sum);
                    else rowacc[rl] = sum;
                }
            }
        }
    }
    if (direct) {   // every row is complete and stored; nothing staged
        __shared__ double red_direct[32];
        epi.end_block(t, red_direct);
        return;
    }
    const bool gave_up = staged && !mbar_wait_bounded(mbar, 0, a.err);
    if (__syncthreads_or(gave_up)) {
        // a staged copy did not arrive in time (the error word says so): the
        // tile's rows and halo sums are marked invalid instead of computed
        // from incomplete data
        for (int r = tid; r < nr; r += P) epi.invalid(r0 + r);
        for (int hh = a.hhoff[t] + tid; hh < a.hhoff[t + 1]; hh += P) a.halo[hh] = static_cast<AT>(CUDART_NAN);
        return;
    }
    if (staged && tid == 0) mbar_inval(mbar);

    double *red = reinterpret_cast<double *>(smem + L.red);
    if (hm == 0) {
        for (int r = tid; r < nr; r += P) epi.finish(r0 + r, rowacc[r]);
        epi.end_block(t, red);
        return;
    }
    // 2. middle entries, each read from HBM once and used twice (Eqs. 2-6)
    // with one FMA per use: row sums (a warp owns 32 consecutive rows; rows
    // longer than kShortRow are summed by the whole warp, one after the
    // other), then, with no barrier in between, mirrored sums per column
    // (one thread per distinct column, its entries in row order).  Columns
    // inside the tile complete their row below; columns before the tile (the
    // conflicting region of Fig. 2) are the first segments and go to the
    // halo list that the fold adds to the previous tile.
    for (int rb = (tid & ~31); rb < nr; rb += P) {
        const int r = rb + lane;
        const bool valid = r < nr;
        const int h0 = valid ? hrp[r] : 0, h1 = valid ? hrp[r + 1] : 0;
        const bool hlong = (h1 - h0) > kShortRow;
        AT hs = AT(0);
        if (valid && !hlong) hs = half_row_thread<VT, XT, AT>(h0, h1, hval, hcol, xs);
        unsigned m = __ballot_sync(0xffffffffu, hlong);
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            const int f0 = __shfl_sync(0xffffffffu, h0, b), f1 = __shfl_sync(0xffffffffu, h1, b);
            const AT s2 = half_row_warp<VT, XT, AT>(f0, f1, hval, hcol, xs);
            if (lane == b) hs = s2;
        }
        if (valid && h1 > h0) rowacc[r] += hs;
    }
    const int g0 = a.hhoff[t], nhalo = a.hhoff[t + 1] - g0;
    for (int sgm = tid; sgm < a.hcsn[t]; sgm += P) {
        const uint32_t w0 = hcs[sgm], w1 = hcs[sgm + 1];
        const AT c = half_col_sum<VT, XT, AT>(static_cast<int>(w0 >> 16), static_cast<int>(w1 >> 16), hval, cperm,
                                              hrowc, xs);
        if (sgm < nhalo) a.halo[g0 + sgm] = a.sym ? c : -c;
        else colacc[static_cast<int>(w0 & 0xffffu) - a.W] = c;
    }
    __syncthreads();
    for (int r = tid; r < nr; r += P) epi.finish(r0 + r, a.sym ? rowacc[r] + colacc[r] : rowacc[r] - colacc[r]);
    epi.end_block(t, red);
}

// Sum of one long-row piece, lane l of a long slice: slots base + 32 m
// (m < len) of lval / lcol, in rounds of eight slots sized to the slice's
// width w (warp-uniform: every piece but the last of each row has the same
// length, so nearly every lane of a round holds an entry).  The next round's
// columns are loaded while this round's values and x gathers are in flight,
// so a round waits on one round trip (fp64: the 64-register budget holds the
// extra columns; fp32 / bf16, compiled for three blocks per SM, load each
// round's columns with its values).  Nothing is staged in shared memory and
// no lanes are combined: each piece is one lane's sequential sum, and the
// fold adds a row's pieces in order.
template <typename VT, typename XT, typename AT>
__device__ __forceinline__ AT piece_sum(const VT *__restrict__ val, const int32_t *__restrict__ col, int64_t base,
                                        int len, int w, const XT *__restrict__ xg) {
    constexpr bool kAhead = sizeof(AT) == 8;
    if constexpr (!kAhead) return slice_row_sum_uniform<VT, XT, AT>(val, col, base, len, w, xg, AT(0));
    int c[kUnroll];
    slice_cols(col, base, len, c);
    AT acc = AT(0);
    for (int m0 = 0; m0 < w; m0 += kUnroll) {
        const int rem = len - m0;
        const int64_t q0 = base + static_cast<int64_t>(m0) * kSlice;
        AT v[kUnroll], xv[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            v[u] = AT(0);
            xv[u] = AT(0);
            if (u < rem) {
                v[u] = Val<VT>::ld_stream(val + q0 + static_cast<int64_t>(u) * kSlice);
                xv[u] = static_cast<AT>(__ldg(xg + c[u]));
            }
        }
        const int64_t q1 = q0 + static_cast<int64_t>(kUnroll) * kSlice;
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) c[u] = (u < rem - kUnroll) ? __ldcs(col + q1 + static_cast<int64_t>(u) * kSlice) : 0;
        switch (min(w - m0, kUnroll)) {
        case 1: acc = slot_sums<1, AT>(v, xv, rem, acc); break;
        case 2: acc = slot_sums<2, AT>(v, xv, rem, acc); break;
        case 3: acc = slot_sums<3, AT>(v, xv, rem, acc); break;
        case 4: acc = slot_sums<4, AT>(v, xv, rem, acc); break;
        case 5: acc = slot_sums<5, AT>(v, xv, rem, acc); break;
        case 6: acc = slot_sums<6, AT>(v, xv, rem, acc); break;
        case 7: acc = slot_sums<7, AT>(v, xv, rem, acc); break;
        default: acc = slot_sums<8, AT>(v, xv, rem, acc); break;
        }
    }
    return acc;
}

// Block b of long-row pieces: long slices [b lsb, (b+1) lsb),
// one per warp in turn; the sum of piece p goes to lpart[p].  Power-law rows
// (R-MAT rows reach 65k entries) thus spread over many lanes of many blocks,
// while a lane's sum stays a plain sequential one.  Not inlined: the tile
// path keeps its own register allocation.
template <typename VT, typename XT, typename AT>
__device__ __noinline__ void long_pieces_block(const SpmvArgs<VT, XT, AT> &a, int b, const XT *__restrict__ xop) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int s1 = min((b + 1) * a.lsb, a.nls);
    for (int s = b * a.lsb + warp; s < s1; s += nw) {
        const int e0 = __ldg(a.ls_ent + s);
        const int w = (__ldg(a.ls_ent + s + 1) - e0) / kSlice;
        const int64_t p = static_cast<int64_t>(s) * kSlice + lane;
        const int len = __ldg(a.ls_len + p);
        a.lpart[p] = piece_sum<VT, XT, AT>(a.lval, a.lcol, static_cast<int64_t>(e0) + lane, len, w, xop);
    }
}

// Blocks per SM the tile kernels are compiled for: fp64 needs its 64
// registers per thread; fp32 / bf16 fit 40 and run three 512-thread blocks.
template <typename AT>
constexpr int tile_min_blocks() { return sizeof(AT) == 8 ? 2 : 3; }

template <typename VT, typename XT, typename AT, bool LA = false>
__global__ void __launch_bounds__(kBlock, LA ? 2 : tile_min_blocks<AT>()) tile_kernel(const SpmvArgs<VT, XT, AT> a) {
    extern __shared__ __align__(128) unsigned char smem[];
    // the fold may be scheduled once every block of this grid has started
    // (it waits for this grid's results before reading them)
    asm volatile("griddepcontrol.launch_dependents;");
    if (static_cast<int>(blockIdx.x) < a.nlb) {
        long_pieces_block<VT, XT, AT>(a, blockIdx.x, a.x);
    } else {
        EpiSpmv<XT, AT> epi{a.alpha, a.y};
        tile_block<VT, XT, AT, EpiSpmv<XT, AT>, LA>(a, blockIdx.x - a.nlb, smem, a.x, epi);
    }
}

// Lanczos step of MRS iteration j = st->j + 1 (see EpiMrs); the operand,
// output and ring slots follow from j, read on the device, so the launch
// can be replayed from a CUDA graph.
template <typename XT>
struct MrsVectors {
    MrsState *st;
    XT *w[3];
    XT *p[3];
    XT *xsol;
    const uint32_t *fold_bits;
    double *part;
};

// The last block of a fused iteration sums the blocks' partial norms and
// runs the scalar step (not inlined, so the tile path keeps its registers).
static __device__ __noinline__ void mrs_fused_tail(MrsState *st, double *part, int ntiles, cudaGraphConditionalHandle cond) {
    __shared__ double red[32];
    double tot = 0.0;
    if (last_block_sum(&st->ticket, part, ntiles, red, &tot) && threadIdx.x == 0) mrs_step(st, tot, cond, 1);
}

// With FUSED (no halo targets and no long rows, so nothing is left for a
// fold), the last tile block to finish also reduces the partial norms and
// runs the scalar step, and the loop body is this one launch.
template <typename VT, typename XT, typename AT, bool S, bool FUSED>
__global__ void __launch_bounds__(kBlock, 2) tile_kernel_mrs(const SpmvArgs<VT, XT, AT> a, const MrsVectors<XT> m,
                                                            cudaGraphConditionalHandle cond) {
    extern __shared__ __align__(128) unsigned char smem[];
    if (m.st->done) {   // an unrolled loop body past convergence (or a solve that starts converged)
        if (FUSED && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
        return;
    }
    __shared__ MrsEpiParams<XT, AT> ep;
    if (threadIdx.x == 0) fill_mrs_params<XT, AT>(&ep, m.st, m.w, m.p, m.xsol, m.fold_bits, m.part);
    __syncthreads();
    const XT *xop = m.w[(m.st->j + 3) % 3];   // w_{j-1} for iteration j = st->j + 1
    EpiMrs<XT, AT, S> epi;
    epi.p = &ep;
    epi.nrm = 0.0;
    if (static_cast<int>(blockIdx.x) < a.nlb) long_pieces_block<VT, XT, AT>(a, blockIdx.x, xop);
    else tile_block<VT, XT, AT>(a, blockIdx.x - a.nlb, smem, xop, epi);
    if constexpr (FUSED) mrs_fused_tail(m.st, m.part, a.ntiles, cond);
}

// Piece sums of a long row in the row's entry order: its np full pieces
// from p0, then its shorter last piece rem (if any).  Loads are issued four
// at a time ahead of the additions, which stay in order.
template <typename AT>
__device__ __forceinline__ AT long_row_sum(int p0, int np, int rem, const AT *__restrict__ lpart, int64_t k, int c,
                                           AT v) {
    int q = 0;
    for (; q + 4 <= np; q += 4) {
        AT t[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) t[u] = lpart[static_cast<int64_t>(p0 + q + u) * k + c];
#pragma unroll
        for (int u = 0; u < 4; ++u) v += t[u];
    }
    for (; q < np; ++q) v += lpart[static_cast<int64_t>(p0 + q) * k + c];
    if (rem >= 0) v += lpart[static_cast<int64_t>(rem) * k + c];
    return v;
}

// The full pieces p0 .. p0+np-1 (column c of k) of a heavy long row (at least
// kFoldHeavy of them; an R-MAT hub row has 257) summed by one warp: lane l
// adds pieces p0 + l, p0 + l + 32, ... in order, then five butterfly steps;
// lane 0's result is used, so the order of every addition is fixed.  A
// thread walking such a row alone made the fold the longest step of the
// product (18 us on the R-MAT matrix).
template <typename AT>
__device__ __forceinline__ AT heavy_pieces_warp(int p0, int np, const AT *__restrict__ lpart, int64_t k, int c) {
    const int lane = threadIdx.x & 31;
    AT s = AT(0);
    for (int q = lane; q < np; q += 32) s += lpart[static_cast<int64_t>(p0 + q) * k + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// The fold lists of a handle (device pointers); items with at least
// kFoldHeavy full pieces are also listed in `heavy` and folded by warps.
struct FoldLists {
    const int32_t *row, *halo, *p0, *np, *rem, *heavy;
    int32_t nheavy;
};

// One thread per receiving row: y[row] += halo sum, then the row's long-row
// piece sums in order.
template <typename XT, typename AT>
__global__ void __launch_bounds__(256) fold_kernel(int nitems, const FoldLists F, const AT *__restrict__ halo,
                                                   const AT *__restrict__ lpart, XT *__restrict__ y) {
    // launched as a programmatic dependent of the tile kernel: wait for its
    // completion (and its writes) before reading y, halo and lpart
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int w = gw; w < F.nheavy; w += nw) {   // heavy rows, a warp each
        const int f = __ldg(F.heavy + w);
        const AT s = heavy_pieces_warp<AT>(__ldg(F.p0 + f), __ldg(F.np + f), lpart, 1, 0);
        if (lane == 0) {
            const int r = __ldg(F.row + f), hi = __ldg(F.halo + f), rem = __ldg(F.rem + f);
            AT v = static_cast<AT>(y[r]);
            if (hi >= 0) v += halo[hi];
            v += s;
            if (rem >= 0) v += lpart[rem];
            y[r] = static_cast<XT>(v);
        }
    }
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nitems; f += gridDim.x * blockDim.x) {
        const int np = __ldg(F.np + f);
        if (np >= kFoldHeavy) continue;
        const int r = __ldg(F.row + f), hi = __ldg(F.halo + f);
        const int p0 = __ldg(F.p0 + f), rem = __ldg(F.rem + f);
        AT v = static_cast<AT>(y[r]);
        if (hi >= 0) v += halo[hi];
        v = long_row_sum<AT>(p0, np, rem, lpart, 1, 0, v);
        y[r] = static_cast<XT>(v);
    }
}

inline FoldLists fold_lists(const DevLayout &D, const Layout &L) {
    return FoldLists{D.fold_row, D.fold_halo, D.fold_p0, D.fold_np, D.fold_rem, D.fold_heavy,
                     static_cast<int32_t>(L.fold_heavy.size())};
}

// Kernel arguments of handle h for precision dtype (values of that
// precision; x, y, alpha and the scratch are set by the caller).
template <typename VT, typename XT, typename AT>
SpmvArgs<VT, XT, AT> make_spmv_args(const pars3_handle *h, int dtype) {
    const Layout &L = h->L;
    const DevLayout &D = h->D;
    SpmvArgs<VT, XT, AT> a;
    a.n = h->n;
    a.T = h->T;
    a.W = h->W;
    a.ntiles = h->ntiles;
    a.Mh = static_cast<int32_t>(round_up(L.max_tile_half, kAlignHalf));
    a.nls = L.nls();
    a.nlb = L.nlong_blocks();
    a.lsb = L.ls_per_block;
    a.hoff = D.hoff;
    a.hcnt = D.hcnt;
    a.hrp = D.hrp;
    a.hcol = D.hcol;
    a.hcperm = D.hcperm;
    a.hrowc = D.hrowc;
    a.hcsoff = D.hcsoff;
    a.hcsn = D.hcsn;
    a.hcs = D.hcs;
    a.CS = L.max_tile_cs;
    a.hval = static_cast<const VT *>(D.hval[dtype]);
    a.hhoff = D.hhoff;
    a.hhrow = D.hhrow;
    a.halo = static_cast<AT *>(D.halo);
    a.sl_off = D.sl_off;
    a.sl_ent = D.sl_ent;
    a.sl_e = D.sl_e;
    a.sl_meta = D.sl_meta;
    a.fcol = D.fcol;
    a.fval = static_cast<const VT *>(D.fval[dtype]);
    a.ls_ent = D.ls_ent;
    a.ls_len = D.ls_len;
    a.lcol = D.lcol;
    a.lval = static_cast<const VT *>(D.lval[dtype]);
    a.lpart = static_cast<AT *>(D.lpart);
    a.x = nullptr;
    a.y = nullptr;
    a.alpha = AT(0);
    a.err = D.err;
    a.sym = h->symmetric;
    return a;
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

}  // namespace pars3
