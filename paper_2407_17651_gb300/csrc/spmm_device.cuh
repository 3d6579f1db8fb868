// spmm_device.cuh -- device code of the multi-right-hand-side product
// Y = (alpha I + S) X (X, Y row-major, k <= 32), shared by the single-matrix
// launch (spmm.cu) and the batched persistent launch (batched.cu).
//
// A group of LPR lanes owns one row; each lane holds NV consecutive columns
// (NV = 16 bytes of the vector type when k is a multiple of it, else 1), so a
// row of X is gathered with 16-byte coalesced loads and a warp keeps 32/LPR
// rows in flight.  Groups walk the tile's rows in sliced-ELL order (slice by
// slice, lane by lane), so neighbouring groups read neighbouring slots of the
// full-storage arrays and rows of similar length run side by side.  The x
// window is not staged (k times T+W values would not fit); middle entries
// gather X rows through L2 like the outer ones.  Each stored middle entry is
// still read once and used twice (Eqs. 2-6): for its row and, through the
// (column, row) list, for the mirrored column sum.  The tile's middle
// entries, row pointers and (column, row) order are staged by TMA; a
// per-entry row index is built in shared memory.
#pragma once

#include "spmv_kernels.cuh"

namespace pars3 {

struct SpmmLayout {
    uint32_t hrp, hval, hcol, cperm, hrow, cs, ce, mbar, total;
};

// T: tile rows, W: window, Mh: half-path entries of the largest tile
PARS3_HD SpmmLayout spmm_layout(uint32_t T, uint32_t W, uint32_t Mh, uint32_t vsz) {
    SpmmLayout s;
    s.hrp = 0;
    s.hval = align128(s.hrp + (T + 8u) * 2u);
    s.hcol = align128(s.hval + Mh * vsz);
    s.cperm = align128(s.hcol + Mh * 2u);
    s.hrow = align128(s.cperm + Mh * 2u);
    s.cs = align128(s.hrow + Mh * 2u);
    s.ce = align128(s.cs + (T + W) * 2u);
    s.mbar = align128(s.ce + (T + W) * 2u);
    s.total = align128(s.mbar + 8u);
    return s;
}

// L2 policy for the gathered rows of X: kept (evict-last) while the matrix
// and Y stream through L2 with evict-first, so a row of X that several rows
// of the tile reference is read from HBM once.
__device__ __forceinline__ uint64_t l2_keep_policy() {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// NV consecutive elements of a row of X (a 16-byte vector when NV > 1):
// gathers with the keep policy, stores of Y streaming (evict-first)
template <typename XT, int NV> struct XVec;
template <> struct XVec<float, 1> {
    static __device__ __forceinline__ void ld(const float *p, float *o, uint64_t pol) {
        asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(o[0]) : "l"(p), "l"(pol));
    }
    static __device__ __forceinline__ void st(float *p, const float *o) { __stcs(p, o[0]); }
};
template <> struct XVec<double, 1> {
    static __device__ __forceinline__ void ld(const double *p, double *o, uint64_t pol) {
        asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(o[0]) : "l"(p), "l"(pol));
    }
    static __device__ __forceinline__ void st(double *p, const double *o) { __stcs(p, o[0]); }
};
template <> struct XVec<float, 4> {
    static __device__ __forceinline__ void ld(const float *p, float *o, uint64_t pol) {
        asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                     : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3])
                     : "l"(p), "l"(pol));
    }
    static __device__ __forceinline__ void st(float *p, const float *o) {
        __stcs(reinterpret_cast<float4 *>(p), make_float4(o[0], o[1], o[2], o[3]));
    }
};
template <> struct XVec<double, 2> {
    static __device__ __forceinline__ void ld(const double *p, double *o, uint64_t pol) {
        asm volatile("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
                     : "=d"(o[0]), "=d"(o[1])
                     : "l"(p), "l"(pol));
    }
    static __device__ __forceinline__ void st(double *p, const double *o) {
        __stcs(reinterpret_cast<double2 *>(p), make_double2(o[0], o[1]));
    }
};

// 32-byte lanes: two adjacent 16-byte vectors
template <> struct XVec<float, 8> {
    static __device__ __forceinline__ void ld(const float *p, float *o, uint64_t pol) {
        XVec<float, 4>::ld(p, o, pol);
        XVec<float, 4>::ld(p + 4, o + 4, pol);
    }
    static __device__ __forceinline__ void st(float *p, const float *o) {
        XVec<float, 4>::st(p, o);
        XVec<float, 4>::st(p + 4, o + 4);
    }
};
template <> struct XVec<double, 4> {
    static __device__ __forceinline__ void ld(const double *p, double *o, uint64_t pol) {
        XVec<double, 2>::ld(p, o, pol);
        XVec<double, 2>::ld(p + 2, o + 2, pol);
    }
    static __device__ __forceinline__ void st(double *p, const double *o) {
        XVec<double, 2>::st(p, o);
        XVec<double, 2>::st(p + 2, o + 2);
    }
};

// elements per lane for k columns of XT: 32 bytes (two 16-byte vectors) when
// k is at least 16 and a multiple of it -- fewer lanes per row, more rows in
// flight per warp -- else 16 bytes when that divides k, else one element
template <typename XT>
PARS3_HD int spmm_nv(int k) {
    const int v = 16 / static_cast<int>(sizeof(XT));
    if (k >= 16 && k % (2 * v) == 0) return 2 * v;
    return (k % v == 0) ? v : 1;
}

// elements per lane for a requested lane width (bytes; 0 = the rule above):
// one element, a 16-byte vector or two of them, as far as k and the
// alignment of X and Y allow
template <typename XT>
PARS3_HD int spmm_lane_elems(int k, int lane_bytes, bool aligned) {
    if (!aligned) return 1;
    const int v = 16 / static_cast<int>(sizeof(XT));
    if (lane_bytes == 32 && k % (2 * v) == 0) return 2 * v;
    if (lane_bytes == 16 && k % v == 0) return v;
    if (lane_bytes > 0 && lane_bytes <= 8) return 1;
    return spmm_nv<XT>(k);
}

// lanes per row (a power of two) for k columns held NV to a lane
PARS3_HD int spmm_lpr(int k, int nv) {
    const int lanes = (k + nv - 1) / nv;
    int lpr = 1;
    while (lpr < lanes) lpr <<= 1;
    return lpr;
}

// entries in flight per lane group (fewer with fp64 or vector lanes, which
// need more registers per entry; with 32-byte lanes two, which measured
// faster than four with the spills four needs)
template <typename AT, int NV> constexpr int spmm_unroll() {
    return (NV == 1 && sizeof(AT) == 4) ? 8 : (NV * sizeof(AT) >= 32 ? 2 : 4);
}

// acc[0..NV) += sum_m v[base + m*stride] * X[col[base + m*stride], c0..c0+NV)
// for m < len, in m order.  Every lane of a group loads the same value and
// column (L1 broadcast) and its own NV columns of the X row.
template <typename VT, typename XT, typename AT, int NV>
__device__ __forceinline__ void spmm_strided_sum(const VT *__restrict__ val, const int32_t *__restrict__ col,
                                                 int64_t base, int64_t stride, int len, const XT *__restrict__ X,
                                                 int k, int c0, bool on, AT *acc) {
    constexpr int U = spmm_unroll<AT, NV>();
    const uint64_t pol = l2_keep_policy();
    for (int m0 = 0; m0 < len; m0 += U) {
        AT v[U];
        int j[U];
        XT xv[U][NV];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            v[u] = AT(0);
            j[u] = 0;
            if (m0 + u < len) {
                const int64_t q = base + static_cast<int64_t>(m0 + u) * stride;
                v[u] = static_cast<AT>(Val<VT>::ld_stream(val + q));
                j[u] = __ldcs(col + q);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (on && m0 + u < len) {
                XVec<XT, NV>::ld(X + static_cast<int64_t>(j[u]) * k + c0, xv[u], pol);
            } else {
#pragma unroll
                for (int w = 0; w < NV; ++w) xv[u][w] = XT(0);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (m0 + u < len) {
#pragma unroll
                for (int w = 0; w < NV; ++w) acc[w] += v[u] * static_cast<AT>(xv[u][w]);
            }
    }
}

// acc[w] += hval[e] * X[xbase + xidx[e], c0 + w] over the staged middle
// entries e = order[q] (or e = q when order is null) for q in [q0, q1), in q
// order.
template <typename VT, typename XT, typename AT, int NV>
__device__ __forceinline__ void spmm_smem_sum(const VT *hval, const uint16_t *order, const uint16_t *xidx, int q0,
                                              int q1, int64_t xbase, const XT *__restrict__ X, int k, int c0,
                                              bool on, AT *acc) {
    constexpr int U = spmm_unroll<AT, NV>();
    const uint64_t pol = l2_keep_policy();
    for (int m0 = q0; m0 < q1; m0 += U) {
        AT v[U];
        XT xv[U][NV];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            v[u] = AT(0);
            if (m0 + u < q1) {
                const int e = order ? order[m0 + u] : m0 + u;
                v[u] = sval<VT>(hval, e);
                if (on) XVec<XT, NV>::ld(X + (xbase + xidx[e]) * k + c0, xv[u], pol);
            }
            if (!(on && m0 + u < q1)) {
#pragma unroll
                for (int w = 0; w < NV; ++w) xv[u][w] = XT(0);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (m0 + u < q1) {
#pragma unroll
                for (int w = 0; w < NV; ++w) acc[w] += v[u] * static_cast<AT>(xv[u][w]);
            }
    }
}

template <typename VT, typename XT, typename AT, int LPR, int NV>
__device__ __forceinline__ void spmm_tile(const SpmvArgs<VT, XT, AT> &a, int k, int t, unsigned char *smem) {
    const SpmmLayout L = spmm_layout(a.T, a.W, a.Mh, sizeof(VT));
    uint16_t *hrp = reinterpret_cast<uint16_t *>(smem + L.hrp);
    VT *hval = reinterpret_cast<VT *>(smem + L.hval);
    uint16_t *hcol = reinterpret_cast<uint16_t *>(smem + L.hcol);
    uint16_t *cperm = reinterpret_cast<uint16_t *>(smem + L.cperm);
    uint16_t *hrow = reinterpret_cast<uint16_t *>(smem + L.hrow);
    uint16_t *cs = reinterpret_cast<uint16_t *>(smem + L.cs);
    uint16_t *ce = reinterpret_cast<uint16_t *>(smem + L.ce);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + L.mbar);
    const int tid = threadIdx.x, P = blockDim.x;
    const int r0 = t * a.T, r1 = min(r0 + a.T, a.n), nr = r1 - r0;
    const int wb = r0 - a.W;
    const int hb = a.hoff[t], hm = a.hcnt[t];
    const uint32_t hmp = static_cast<uint32_t>((hm + kAlignHalf - 1) / kAlignHalf * kAlignHalf);
    const uint32_t rpb = static_cast<uint32_t>(a.T + 8) * 2u;
    const bool staged = hm > 0;   // block-uniform
    // the copy engine prefetches the tile's sliced-ELL rows into L2, so the
    // groups' value and column loads wait on L2 instead of HBM (k = 32 fp32
    // on the 128^3 + 1 % matrix: 273 -> 259 us)
    if (tid == P - 1 && a.sl_off[t + 1] > a.sl_off[t]) prefetch_slices(a, a.sl_off[t], a.sl_off[t + 1]);
    if (staged) {
        if (tid == 0) {
            mbar_init(mbar, 1);
            fence_mbar_init();
            mbar_arrive_expect_tx(mbar, rpb + hmp * (sizeof(VT) + 4u));
            bulk_g2s(hrp, a.hrp + static_cast<size_t>(t) * (a.T + 8), rpb, mbar);
            bulk_g2s(hval, a.hval + hb, hmp * sizeof(VT), mbar);
            bulk_g2s(hcol, a.hcol + hb, hmp * 2u, mbar);
            bulk_g2s(cperm, a.hcperm + hb, hmp * 2u, mbar);
        }
        for (int p = tid; p < nr + a.W; p += P) {
            cs[p] = 0;
            ce[p] = 0;
        }
        __syncthreads();   // the barrier is initialised before anyone waits on it
        const bool gave_up = !mbar_wait_bounded(mbar, 0, a.err);
        if (__syncthreads_or(gave_up)) {
            // a staged copy did not arrive in time (the error word says so):
            // the tile's rows and halo sums are marked invalid
            for (int64_t q = tid; q < static_cast<int64_t>(nr) * k; q += P)
                a.y[static_cast<int64_t>(r0) * k + q] = static_cast<XT>(CUDART_NAN);
            for (int64_t q = static_cast<int64_t>(a.hhoff[t]) * k + tid; q < static_cast<int64_t>(a.hhoff[t + 1]) * k;
                 q += P)
                a.halo[q] = static_cast<AT>(CUDART_NAN);
            return;
        }
        if (tid == 0) mbar_inval(mbar);
        for (int r = tid; r < nr; r += P)
            for (int e = hrp[r]; e < hrp[r + 1]; ++e) hrow[e] = static_cast<uint16_t>(r);
        for (int q = tid; q < hm; q += P) {
            const int key = hcol[cperm[q]];
            if (q == 0 || hcol[cperm[q - 1]] != key) cs[key] = static_cast<uint16_t>(q);
            if (q == hm - 1 || hcol[cperm[q + 1]] != key) ce[key] = static_cast<uint16_t>(q + 1);
        }
        __syncthreads();
    }

    const int g = tid / LPR, c0 = (tid % LPR) * NV, ng = P / LPR;
    const bool on = c0 < k;
    const int s0 = a.sl_off[t], s1 = a.sl_off[t + 1];
    const int nslot = (s1 - s0) * kSlice;
    const int gw = g % (32 / LPR);
    for (int qb = g - gw; qb < nslot; qb += ng) {
        const int q = qb + gw;
        const int s = q >> 5, l = q & 31;
        const uint32_t meta = q < nslot ? __ldg(a.sl_meta + static_cast<int64_t>(s0) * kSlice + q) : 0xffffu;
        const int rl = static_cast<int>(meta & 0xffffu);
        const bool valid = rl != 0xffff;   // not a padding lane of the tile's last slice
        const int len = valid ? static_cast<int>(meta >> 16) : 0;
        const int64_t row = static_cast<int64_t>(r0 + (valid ? rl : 0));
        AT acc[NV];
        {
            XT xr[NV];
            if (on && valid) XVec<XT, NV>::ld(a.x + row * k + c0, xr, l2_keep_policy());
#pragma unroll
            for (int w = 0; w < NV; ++w) acc[w] = on && valid ? a.alpha * static_cast<AT>(xr[w]) : AT(0);
        }
        const int64_t base = valid ? static_cast<int64_t>(__ldg(a.sl_ent + s0 + s)) + l : 0;
        spmm_strided_sum<VT, XT, AT, NV>(a.fval, a.fcol, base, kSlice, len, a.x, k, c0, on, acc);
        if (!valid) continue;
        if (staged) {
            spmm_smem_sum<VT, XT, AT, NV>(hval, nullptr, hcol, hrp[rl], hrp[rl + 1], wb, a.x, k, c0, on, acc);
            const int p = rl + a.W;
            if (ce[p] > cs[p]) {
                AT cm[NV];
#pragma unroll
                for (int w = 0; w < NV; ++w) cm[w] = AT(0);
                spmm_smem_sum<VT, XT, AT, NV>(hval, cperm, hrow, cs[p], ce[p], r0, a.x, k, c0, on, cm);
#pragma unroll
                for (int w = 0; w < NV; ++w) acc[w] = a.sym ? acc[w] + cm[w] : acc[w] - cm[w];
            }
        }
        if (on) {
            XT out[NV];
#pragma unroll
            for (int w = 0; w < NV; ++w) out[w] = static_cast<XT>(acc[w]);
            XVec<XT, NV>::st(a.y + row * k + c0, out);
        }
    }
    if (!staged) return;
    const int g0 = a.hhoff[t], g1 = a.hhoff[t + 1];
    for (int h = g0 + g; h < g1; h += ng) {
        const int p = a.hhrow[h] - wb;
        AT cm[NV];
#pragma unroll
        for (int w = 0; w < NV; ++w) cm[w] = AT(0);
        spmm_smem_sum<VT, XT, AT, NV>(hval, cperm, hrow, cs[p], ce[p], r0, a.x, k, c0, on, cm);
        if (on)
#pragma unroll
            for (int w = 0; w < NV; ++w) a.halo[static_cast<int64_t>(h) * k + c0 + w] = a.sym ? cm[w] : -cm[w];
    }
}

// Block b of long-row pieces (long slices [b lsb, (b+1) lsb)):
// a lane group per piece, walking the pieces in slice order so that
// neighbouring groups read neighbouring slots; the k-wide sum of piece p goes
// to lpart[p k ..], and the fold adds a row's pieces in order.  A row of tens
// of thousands of entries thus spreads over hundreds of lane groups.
template <typename VT, typename XT, typename AT, int LPR, int NV>
__device__ __forceinline__ void spmm_long(const SpmvArgs<VT, XT, AT> &a, int k, int b) {
    const int tid = threadIdx.x, P = blockDim.x;
    const int g = tid / LPR, c0 = (tid % LPR) * NV, ng = P / LPR;
    const bool on = c0 < k;
    const int s0 = b * a.lsb, s1 = min(s0 + a.lsb, a.nls);
    const int nslot = (s1 - s0) * kSlice;
    for (int q = g; q < nslot; q += ng) {
        const int64_t p = static_cast<int64_t>(s0) * kSlice + q;
        const int s = static_cast<int>(p / kSlice), l = static_cast<int>(p % kSlice);
        const int len = __ldg(a.ls_len + p);
        AT acc[NV];
#pragma unroll
        for (int w = 0; w < NV; ++w) acc[w] = AT(0);
        spmm_strided_sum<VT, XT, AT, NV>(a.lval, a.lcol, static_cast<int64_t>(__ldg(a.ls_ent + s)) + l, kSlice, len,
                                         a.x, k, c0, on, acc);
        if (on)
#pragma unroll
            for (int w = 0; w < NV; ++w) a.lpart[p * k + c0 + w] = acc[w];
    }
}

}  // namespace pars3
