// spmm_device.cuh -- device code of the multi-right-hand-side product
// Y = (alpha I + S) X (X, Y row-major, k <= 32), shared by the single-matrix
// launch (spmm.cu) and the batched persistent launch (batched.cu).
//
// Lanes run over the k columns: a group of LPR = next_pow2(k) lanes owns one
// row, so every gather of a row of X is a coalesced read of k consecutive
// values.  The x window is not staged (k times T+W values would not fit);
// middle entries gather X rows through L2 like the outer ones.  Each stored
// middle entry is still read once and used twice (Eqs. 2-6): for its row
// and, through the (column, row) list, for the mirrored column sum.  The
// tile's middle entries, row pointers and (column, row) order are staged by
// TMA; a per-entry row index and the row -> sliced-ELL lane map are built in
// shared memory.
#pragma once

#include "spmv_kernels.cuh"

namespace pars3 {

struct SpmmLayout {
    uint32_t hrp, hval, hcol, cperm, hrow, rowpos, cs, ce, mbar, total;
};

// T: tile rows, W: window, Mh: half-path entries of the largest tile
PARS3_HD SpmmLayout spmm_layout(uint32_t T, uint32_t W, uint32_t Mh, uint32_t vsz) {
    SpmmLayout s;
    s.hrp = 0;
    s.hval = align128(s.hrp + (T + 8u) * 2u);
    s.hcol = align128(s.hval + Mh * vsz);
    s.cperm = align128(s.hcol + Mh * 2u);
    s.hrow = align128(s.cperm + Mh * 2u);
    s.rowpos = align128(s.hrow + Mh * 2u);
    s.cs = align128(s.rowpos + T * 4u);
    s.ce = align128(s.cs + (T + W) * 2u);
    s.mbar = align128(s.ce + (T + W) * 2u);
    s.total = align128(s.mbar + 8u);
    return s;
}

template <typename VT, typename XT, typename AT, int LPR>
__device__ __forceinline__ void spmm_tile(const SpmvArgs<VT, XT, AT> &a, int k, int t, unsigned char *smem) {
    const SpmmLayout L = spmm_layout(a.T, a.W, a.Mh, sizeof(VT));
    uint16_t *hrp = reinterpret_cast<uint16_t *>(smem + L.hrp);
    VT *hval = reinterpret_cast<VT *>(smem + L.hval);
    uint16_t *hcol = reinterpret_cast<uint16_t *>(smem + L.hcol);
    uint16_t *cperm = reinterpret_cast<uint16_t *>(smem + L.cperm);
    uint16_t *hrow = reinterpret_cast<uint16_t *>(smem + L.hrow);
    uint32_t *rowpos = reinterpret_cast<uint32_t *>(smem + L.rowpos);
    uint16_t *cs = reinterpret_cast<uint16_t *>(smem + L.cs);
    uint16_t *ce = reinterpret_cast<uint16_t *>(smem + L.ce);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + L.mbar);
    const int tid = threadIdx.x, P = blockDim.x;
    const int r0 = t * a.T, r1 = min(r0 + a.T, a.n), nr = r1 - r0;
    const int wb = r0 - a.W;
    const int hb = a.hoff[t], hm = a.hcnt[t];
    const uint32_t hmp = static_cast<uint32_t>((hm + kAlignHalf - 1) / kAlignHalf * kAlignHalf);
    const uint32_t rpb = static_cast<uint32_t>(a.T + 8) * 2u;
    if (tid == 0) {
        mbar_init(mbar, 1);
        fence_mbar_init();
        uint32_t tx = rpb + (hm > 0 ? hmp * (sizeof(VT) + 4u) : 0u);
        mbar_arrive_expect_tx(mbar, tx);
        bulk_g2s(hrp, a.hrp + static_cast<size_t>(t) * (a.T + 8), rpb, mbar);
        if (hm > 0) {
            bulk_g2s(hval, a.hval + hb, hmp * sizeof(VT), mbar);
            bulk_g2s(hcol, a.hcol + hb, hmp * 2u, mbar);
            bulk_g2s(cperm, a.hcperm + hb, hmp * 2u, mbar);
        }
    }
    for (int p = tid; p < nr + a.W; p += P) {
        cs[p] = 0;
        ce[p] = 0;
    }
    // row -> (slice, lane) of the sliced-ELL rows of this tile
    const int s0 = a.sl_off[t], s1 = a.sl_off[t + 1];
    for (int q = tid; q < (s1 - s0) * kSlice; q += P) {
        const uint32_t meta = __ldg(a.sl_meta + static_cast<int64_t>(s0) * kSlice + q);
        const uint32_t rl = meta & 0xffffu;
        if (rl != 0xffffu) rowpos[rl] = static_cast<uint32_t>(q);
    }
    __syncthreads();
    mbar_wait_bounded(mbar, 0, a.err);
    __syncthreads();
    if (tid == 0) mbar_inval(mbar);
    for (int r = tid; r < nr; r += P)
        for (int e = hrp[r]; e < hrp[r + 1]; ++e) hrow[e] = static_cast<uint16_t>(r);
    for (int q = tid; q < hm; q += P) {
        const int key = hcol[cperm[q]];
        if (q == 0 || hcol[cperm[q - 1]] != key) cs[key] = static_cast<uint16_t>(q);
        if (q == hm - 1 || hcol[cperm[q + 1]] != key) ce[key] = static_cast<uint16_t>(q + 1);
    }
    __syncthreads();

    const int g = tid / LPR, c = tid % LPR, ng = P / LPR;
    const bool on = c < k;
    for (int r = g; r < nr; r += ng) {
        const int64_t row = static_cast<int64_t>(r0 + r);
        AT acc = on ? a.alpha * static_cast<AT>(a.x[row * k + c]) : AT(0);
        const uint32_t pos = rowpos[r];
        const int s = static_cast<int>(pos >> 5), l = static_cast<int>(pos & 31u);
        const uint32_t meta = __ldg(a.sl_meta + (static_cast<int64_t>(s0) + s) * kSlice + l);
        const int len = static_cast<int>(meta >> 16);
        const int64_t base = static_cast<int64_t>(__ldg(a.sl_ent + s0 + s)) + l;
        for (int m = 0; m < len; ++m) {
            const int64_t q = base + static_cast<int64_t>(m) * kSlice;
            const AT v = Val<VT>::ld(a.fval + q);
            const int j = __ldg(a.fcol + q);
            if (on) acc += v * static_cast<AT>(__ldg(a.x + static_cast<int64_t>(j) * k + c));
        }
        if (hm > 0) {
            for (int e = hrp[r]; e < hrp[r + 1]; ++e) {
                const AT v = sval<VT>(hval, e);
                const int64_t j = wb + hcol[e];
                if (on) acc += v * static_cast<AT>(__ldg(a.x + j * k + c));
            }
            const int p = r + a.W;
            AT cm = AT(0);
            for (int q = cs[p]; q < ce[p]; ++q) {
                const int e = cperm[q];
                const AT v = sval<VT>(hval, e);
                if (on) cm += v * static_cast<AT>(__ldg(a.x + static_cast<int64_t>(r0 + hrow[e]) * k + c));
            }
            if (ce[p] > cs[p]) acc = acc - cm;
        }
        if (on) a.y[row * k + c] = static_cast<XT>(acc);
    }
    const int g0 = a.hhoff[t], g1 = a.hhoff[t + 1];
    for (int h = g0 + g; h < g1; h += ng) {
        const int p = a.hhrow[h] - wb;
        AT cm = AT(0);
        for (int q = cs[p]; q < ce[p]; ++q) {
            const int e = cperm[q];
            const AT v = sval<VT>(hval, e);
            if (on) cm += v * static_cast<AT>(__ldg(a.x + static_cast<int64_t>(r0 + hrow[e]) * k + c));
        }
        if (on) a.halo[static_cast<int64_t>(h) * k + c] = -cm;
    }
}

// Long-row chunk: one lane group per row touched, entries read in order.
template <typename VT, typename XT, typename AT, int LPR>
__device__ __forceinline__ void spmm_long(const SpmvArgs<VT, XT, AT> &a, int k, int cidx) {
    const int tid = threadIdx.x, P = blockDim.x;
    const int beg = a.lcbeg[cidx], end = a.lcend[cidx];
    const int l0 = a.lcfirst[cidx], nrc = a.lcrows[cidx];
    const int g = tid / LPR, c = tid % LPR, ng = P / LPR;
    const bool on = c < k;
    for (int u = g; u < nrc; u += ng) {
        const int e0 = max(a.lrp[l0 + u], beg), e1 = min(a.lrp[l0 + u + 1], end);
        AT acc = AT(0);
        for (int e = e0; e < e1; ++e) {
            const AT v = Val<VT>::ld(a.lval + e);
            const int j = __ldg(a.lcol + e);
            if (on) acc += v * static_cast<AT>(__ldg(a.x + static_cast<int64_t>(j) * k + c));
        }
        if (on) a.lpart[static_cast<int64_t>(a.lcslot[cidx] + u) * k + c] = acc;
    }
}

}  // namespace pars3
