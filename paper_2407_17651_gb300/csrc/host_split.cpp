// host_split.cpp -- the 3-way band split of Sec. 3.1.2 (Figs. 7-8) and the
// device layout derived from it.
//
// Canonical split (the bit-exact contract, see pars3_canonical):
//   re-triangularize P S P^T (an entry landing above the diagonal is stored
//   mirrored with its sign flipped, Eq. 2), sort by (row, column), classify
//   each stored (i, j): middle-local (i-j <= W, j in i's tile), middle-halo
//   (i-j <= W, j in the previous tile) or outer (i-j > W); per tile the
//   middle entries in (column, row) order; the outer entries in row and in
//   column order.  All orderings are stable counting sorts, linear time.
//
// Device layout (implementation; derived from the canonical split):
//   half path  -- middle entries of ordinary rows: stored once, one block per
//                 row tile uses each twice (row sum and mirrored sum), the
//                 mirrored sums of halo entries go to a compact halo list;
//   full path  -- outer entries, and every entry touching a long row or an
//                 over-full tile, stored in both rows with mirrored sign, so
//                 that each row is a plain gather (no write conflicts);
//   long rows  -- rows whose full-path length exceeds long_row are summed in
//                 chunks of kLongChunk entries and folded in fixed order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"
#include "smem_layout.h"

namespace pars3 {

uint16_t f32_to_bf16_rne(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu)) return static_cast<uint16_t>((u >> 16) | 0x40u);
    // round to nearest, ties to even, on the 16 dropped bits
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    return static_cast<uint16_t>(u >> 16);
}

void auto_cut(int64_t bw, int32_t w_min, int32_t w_cap, int32_t t_min, int32_t *T, int32_t *W) {
    int64_t w = w_min;
    while (w < bw && w < w_cap) w *= 2;
    if (w > w_cap) w = w_cap;
    *W = static_cast<int32_t>(w);
    *T = static_cast<int32_t>(std::max<int64_t>(w, t_min));
}

static bool is_pow2(int32_t v) { return v > 0 && (v & (v - 1)) == 0; }

// stable counting sort of idx[] by key(idx) in [0, nkeys)
template <class Key>
static void counting_sort(std::vector<int32_t> &idx, int64_t nkeys, Key key) {
    std::vector<int64_t> cnt(static_cast<size_t>(nkeys) + 1, 0);
    for (int32_t e : idx) ++cnt[key(e) + 1];
    for (int64_t k = 0; k < nkeys; ++k) cnt[k + 1] += cnt[k];
    std::vector<int32_t> out(idx.size());
    for (int32_t e : idx) out[cnt[key(e)]++] = e;
    idx.swap(out);
}

static int canonical_split(pars3_handle *h, const int32_t *rowptr, const int32_t *col,
                           const double *val) {
    const int32_t n = h->n, T = h->T, W = h->W;
    const int64_t nnz = h->nnz;
    std::vector<int32_t> pinv(n);
    for (int32_t k = 0; k < n; ++k) pinv[h->perm[k]] = k;
    // re-triangularize
    std::vector<int32_t> r(nnz), c(nnz);
    std::vector<double> v(nnz);
    for (int32_t i = 0, e = 0; i < n; ++i) {
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k, ++e) {
            int32_t a = pinv[i], b = pinv[col[k]];
            if (a > b) { r[e] = a; c[e] = b; v[e] = val[k]; }
            else       { r[e] = b; c[e] = a; v[e] = -val[k]; }
        }
    }
    // sort by (row, col): stable by col, then stable by row
    std::vector<int32_t> ord(nnz);
    for (int64_t e = 0; e < nnz; ++e) ord[e] = static_cast<int32_t>(e);
    counting_sort(ord, n, [&](int32_t e) { return c[e]; });
    counting_sort(ord, n, [&](int32_t e) { return r[e]; });
    h->rowptr.assign(static_cast<size_t>(n) + 1, 0);
    h->col.resize(nnz);
    h->val.resize(nnz);
    std::vector<int32_t> row_of(nnz);
    for (int64_t q = 0; q < nnz; ++q) {
        int32_t e = ord[q];
        h->col[q] = c[e];
        h->val[q] = v[e];
        row_of[q] = r[e];
        ++h->rowptr[r[e] + 1];
    }
    for (int32_t i = 0; i < n; ++i) h->rowptr[i + 1] += h->rowptr[i];
    { std::vector<int32_t>().swap(r); std::vector<int32_t>().swap(c); std::vector<double>().swap(v); }
    // classify
    h->cls.resize(nnz);
    h->counts[0] = h->counts[1] = h->counts[2] = 0;
    for (int64_t e = 0; e < nnz; ++e) {
        int32_t i = row_of[e], j = h->col[e];
        int32_t r0 = (i / T) * T;
        uint8_t k = (i - j <= W) ? (j >= r0 ? 0 : 1) : 2;
        h->cls[e] = k;
        ++h->counts[k];
    }
    // per-tile middle lists in (col, row) order: CSR order is (row, col);
    // stable by col gives (col, row), stable by tile gives (tile, col, row)
    std::vector<int32_t> mid, outer;
    mid.reserve(h->counts[0] + h->counts[1]);
    outer.reserve(h->counts[2]);
    for (int64_t e = 0; e < nnz; ++e) {
        if (h->cls[e] != 2) mid.push_back(static_cast<int32_t>(e));
        else outer.push_back(static_cast<int32_t>(e));
    }
    counting_sort(mid, n, [&](int32_t e) { return h->col[e]; });
    counting_sort(mid, h->ntiles, [&](int32_t e) { return row_of[e] / T; });
    h->tile_ptr.assign(static_cast<size_t>(h->ntiles) + 1, 0);
    for (int32_t e : mid) ++h->tile_ptr[row_of[e] / T + 1];
    for (int32_t t = 0; t < h->ntiles; ++t) h->tile_ptr[t + 1] += h->tile_ptr[t];
    h->tile_list.swap(mid);
    h->outer_csr = outer;
    counting_sort(outer, n, [&](int32_t e) { return h->col[e]; });
    h->outer_csc.swap(outer);
    h->bw = 0;
    for (int64_t e = 0; e < nnz; ++e) h->bw = std::max<int64_t>(h->bw, row_of[e] - h->col[e]);
    return PARS3_OK;
}

static int primary_dtype(int32_t dtypes) {
    return (dtypes & PARS3_DTYPE_BIT(PARS3_F64)) ? PARS3_F64 : PARS3_F32;
}

static void dtype_sizes(int dtype, uint32_t *xsz, uint32_t *asz) {
    if (dtype == PARS3_F64) { *xsz = 8; *asz = 8; }
    else { *xsz = 4; *asz = 4; }
}

int smem_bytes_for(const pars3_handle *h, int dtype) {
    uint32_t xsz, asz;
    dtype_sizes(dtype, &xsz, &asz);
    SmemLayout s = smem_layout(h->T, h->W, static_cast<uint32_t>(h->L.max_tile_half), kBlock, xsz, asz, 1);
    return static_cast<int>(s.total);
}

// Largest half-path tile (entries) that still fits in shared memory.
static int32_t half_cap(const pars3_handle *h) {
    uint32_t xsz, asz;
    dtype_sizes(primary_dtype(h->dtypes), &xsz, &asz);
    SmemLayout s0 = smem_layout(h->T, h->W, 0, kBlock, xsz, asz, 1);
    int64_t room = static_cast<int64_t>(kSmemLimit) - s0.total - 64;
    int64_t per = asz + 4;
    int64_t cap = room > 0 ? room / per : 0;
    cap = std::min<int64_t>(cap, 65535 - kAlignEntries);
    return static_cast<int32_t>(std::max<int64_t>(cap, 0));
}

int build_layout(pars3_handle *h) {
    Layout &L = h->L;
    const int32_t n = h->n, T = h->T, W = h->W, nt = h->ntiles;
    const int64_t nnz = h->nnz;
    const std::vector<int32_t> &rp = h->rowptr;
    const std::vector<int32_t> &ci = h->col;
    std::vector<int32_t> row_of(nnz);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) row_of[e] = i;
    // column-major view of the band CSR: entries of column j in increasing row
    std::vector<int32_t> cptr(static_cast<size_t>(n) + 1, 0);
    for (int64_t e = 0; e < nnz; ++e) ++cptr[ci[e] + 1];
    for (int32_t j = 0; j < n; ++j) cptr[j + 1] += cptr[j];
    std::vector<int32_t> cent(nnz);
    {
        std::vector<int32_t> fill(cptr.begin(), cptr.end() - 1);
        for (int64_t e = 0; e < nnz; ++e) cent[fill[ci[e]]++] = static_cast<int32_t>(e);
    }
    // long rows: full degree above the threshold
    std::vector<uint8_t> is_long(n, 0);
    for (int32_t i = 0; i < n; ++i) {
        int64_t d = (rp[i + 1] - rp[i]) + (cptr[i + 1] - cptr[i]);
        if (d > h->long_row) is_long[i] = 1;
    }
    // routing: half if middle, both ends ordinary and the tile fits
    const int32_t cap = half_cap(h);
    std::vector<uint8_t> half(nnz, 0);
    std::vector<int32_t> tcount(nt, 0);
    for (int64_t e = 0; e < nnz; ++e) {
        if (h->cls[e] != 2 && !is_long[row_of[e]] && !is_long[ci[e]]) {
            half[e] = 1;
            ++tcount[row_of[e] / T];
        }
    }
    for (int32_t t = 0; t < nt; ++t) {
        if (tcount[t] > cap) {
            int32_t r0 = t * T, r1 = std::min(n, r0 + T);
            for (int64_t e = rp[r0]; e < rp[r1]; ++e) half[e] = 0;
            tcount[t] = 0;
        }
    }
    // half path arrays
    L.hoff.assign(static_cast<size_t>(nt) + 1, 0);
    L.hcnt.assign(nt, 0);
    for (int32_t t = 0; t < nt; ++t) {
        L.hcnt[t] = tcount[t];
        L.hoff[t + 1] = static_cast<int32_t>(L.hoff[t] + round_up(tcount[t], kAlignEntries));
    }
    const int64_t hn = L.hoff[nt];
    L.hcol.assign(hn, 0);
    L.hcperm.assign(hn, 0);
    L.hrp.assign(static_cast<size_t>(nt) * (T + 8), 0);
    std::vector<int32_t> hpos(nnz, -1);  // entry -> global half position
    L.max_tile_half = 0;
    for (int32_t t = 0; t < nt; ++t) {
        int32_t r0 = t * T, r1 = std::min(n, r0 + T);
        int32_t wb = r0 - W;
        int32_t q = 0;
        uint16_t *lrp = &L.hrp[static_cast<size_t>(t) * (T + 8)];
        for (int32_t i = r0; i < r1; ++i) {
            lrp[i - r0] = static_cast<uint16_t>(q);
            for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
                if (!half[e]) continue;
                hpos[e] = L.hoff[t] + q;
                L.hcol[L.hoff[t] + q] = static_cast<uint16_t>(ci[e] - wb);
                ++q;
            }
        }
        for (int32_t i = r1; i <= r0 + T; ++i) lrp[i - r0] = static_cast<uint16_t>(q);
        L.max_tile_half = std::max(L.max_tile_half, q);
    }
    // (col, row) order per tile: the canonical tile lists filtered to half entries
    L.hhoff.assign(static_cast<size_t>(nt) + 1, 0);
    L.hhrow.clear();
    for (int32_t t = 0; t < nt; ++t) {
        int32_t r0 = t * T;
        int32_t q = 0, last = -1;
        for (int32_t s = h->tile_ptr[t]; s < h->tile_ptr[t + 1]; ++s) {
            int32_t e = h->tile_list[s];
            if (!half[e]) continue;
            L.hcperm[L.hoff[t] + q] = static_cast<uint16_t>(hpos[e] - L.hoff[t]);
            ++q;
            int32_t j = ci[e];
            if (j < r0 && j != last) {
                L.hhrow.push_back(j);
                last = j;
            }
        }
        L.hhoff[t + 1] = static_cast<int32_t>(L.hhrow.size());
    }
    // full path: row i = its full lower entries (+a) then the full entries of
    // column i (mirrored, -a), both in increasing column
    L.frp.assign(static_cast<size_t>(n) + 1, 0);
    for (int32_t i = 0; i < n; ++i) {
        int32_t cnt = 0;
        if (!is_long[i]) {
            for (int32_t e = rp[i]; e < rp[i + 1]; ++e) cnt += !half[e];
            for (int32_t s = cptr[i]; s < cptr[i + 1]; ++s) cnt += !half[cent[s]];
        }
        L.frp[i + 1] = L.frp[i] + cnt;
    }
    const int64_t fn = L.frp[n];
    L.fcol.resize(fn);
    std::vector<int32_t> fsrc(fn);   // signed source entry: e+1 (lower) or -(e+1) (mirrored)
    // long rows
    L.lrow.clear();
    L.lcptr.assign(1, 0);
    L.lcbeg.clear();
    L.lcend.clear();
    L.lcol.clear();
    std::vector<int32_t> lsrc;
    for (int32_t i = 0; i < n; ++i) {
        if (is_long[i]) {
            int32_t start = static_cast<int32_t>(L.lcol.size());
            for (int32_t e = rp[i]; e < rp[i + 1]; ++e) { L.lcol.push_back(ci[e]); lsrc.push_back(e + 1); }
            for (int32_t s = cptr[i]; s < cptr[i + 1]; ++s) {
                int32_t e = cent[s];
                L.lcol.push_back(row_of[e]);
                lsrc.push_back(-(e + 1));
            }
            int32_t end = static_cast<int32_t>(L.lcol.size());
            L.lrow.push_back(i);
            for (int32_t b = start; b < end; b += kLongChunk) {
                L.lcbeg.push_back(b);
                L.lcend.push_back(std::min(end, b + kLongChunk));
            }
            L.lcptr.push_back(static_cast<int32_t>(L.lcbeg.size()));
            continue;
        }
        int32_t q = L.frp[i];
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e)
            if (!half[e]) { L.fcol[q] = ci[e]; fsrc[q] = e + 1; ++q; }
        for (int32_t s = cptr[i]; s < cptr[i + 1]; ++s) {
            int32_t e = cent[s];
            if (!half[e]) { L.fcol[q] = row_of[e]; fsrc[q] = -(e + 1); ++q; }
        }
    }
    // values per precision
    auto fill_vals = [&](const std::vector<int32_t> &src, std::vector<double> &v64,
                         std::vector<float> &v32, std::vector<uint16_t> &v16) {
        const size_t m = src.size();
        if (h->dtypes & PARS3_DTYPE_BIT(PARS3_F64)) v64.resize(m);
        if (h->dtypes & PARS3_DTYPE_BIT(PARS3_F32)) v32.resize(m);
        if (h->dtypes & PARS3_DTYPE_BIT(PARS3_BF16)) v16.resize(m);
        for (size_t q = 0; q < m; ++q) {
            int32_t s = src[q];
            double a = s > 0 ? h->val[s - 1] : -h->val[-s - 1];
            if (!v64.empty()) v64[q] = a;
            float f = static_cast<float>(a);
            if (!v32.empty()) v32[q] = f;
            if (!v16.empty()) v16[q] = f32_to_bf16_rne(f);
        }
    };
    std::vector<int32_t> hsrc(hn, 0);
    for (int64_t e = 0; e < nnz; ++e)
        if (half[e]) hsrc[hpos[e]] = static_cast<int32_t>(e + 1);
    // padding slots carry source 0 -> value handled below as 0
    {
        const size_t m = hsrc.size();
        if (h->dtypes & PARS3_DTYPE_BIT(PARS3_F64)) L.hval64.assign(m, 0.0);
        if (h->dtypes & PARS3_DTYPE_BIT(PARS3_F32)) L.hval32.assign(m, 0.0f);
        if (h->dtypes & PARS3_DTYPE_BIT(PARS3_BF16)) L.hval16.assign(m, 0);
        for (size_t q = 0; q < m; ++q) {
            if (hsrc[q] == 0) continue;
            double a = h->val[hsrc[q] - 1];
            float f = static_cast<float>(a);
            if (!L.hval64.empty()) L.hval64[q] = a;
            if (!L.hval32.empty()) L.hval32[q] = f;
            if (!L.hval16.empty()) L.hval16[q] = f32_to_bf16_rne(f);
        }
    }
    fill_vals(fsrc, L.fval64, L.fval32, L.fval16);
    fill_vals(lsrc, L.lval64, L.lval32, L.lval16);
    return PARS3_OK;
}

int64_t model_bytes(const pars3_handle *h, int dtype) {
    if (!(h->dtypes & PARS3_DTYPE_BIT(dtype))) return 0;
    const Layout &L = h->L;
    int64_t sv = dtype == PARS3_F64 ? 8 : (dtype == PARS3_F32 ? 4 : 2);
    int64_t sx = dtype == PARS3_F64 ? 8 : 4;
    int64_t b = 0;
    b += static_cast<int64_t>(L.hcol.size()) * (sv + 2 + 2);             // half values, columns, order
    b += static_cast<int64_t>(h->ntiles) * (h->T + 8) * 2;               // tile row pointers
    b += static_cast<int64_t>(L.fcol.size()) * (sv + 4) + (h->n + 1) * 4; // full rows
    b += static_cast<int64_t>(L.lcol.size()) * (sv + 4);                  // long rows
    b += 2 * static_cast<int64_t>(h->n) * sx;                             // x once, y once
    return b;
}

}  // namespace pars3

using namespace pars3;

extern "C" int pars3_split(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                           const int32_t *perm, const pars3_split_params *p, pars3_handle **out) {
    if (!out || n < 0 || !rowptr) return PARS3_EINVAL;
    *out = nullptr;
    int rc = validate_lower(n, rowptr, col);
    if (rc != PARS3_OK) return rc;
    const int64_t nnz = rowptr[n];
    if (nnz > 0 && !val) return PARS3_EINVAL;
    for (int64_t k = 0; k < nnz; ++k)
        if (!std::isfinite(val[k])) return PARS3_ENONFINITE;
    pars3_split_params prm{};
    if (p) prm = *p;
    if (prm.dtypes == 0) prm.dtypes = PARS3_DTYPE_BIT(PARS3_F64);
    if (prm.dtypes & ~7) return PARS3_EINVAL;
    if ((prm.T == 0) != (prm.W == 0)) return PARS3_EINVAL;
    pars3_handle *h = nullptr;
    try {
        h = new pars3_handle();
        h->n = n;
        h->nnz = nnz;
        h->dtypes = prm.dtypes;
        h->perm.resize(n);
        if (perm) {
            std::vector<uint8_t> seen(n, 0);
            for (int32_t k = 0; k < n; ++k) {
                if (perm[k] < 0 || perm[k] >= n || seen[perm[k]]) { delete h; return PARS3_EINVAL; }
                seen[perm[k]] = 1;
                h->perm[k] = perm[k];
            }
        } else {
            for (int32_t k = 0; k < n; ++k) h->perm[k] = k;
        }
        if (prm.T == 0) {
            std::vector<int32_t> pinv(n);
            for (int32_t k = 0; k < n; ++k) pinv[h->perm[k]] = k;
            int64_t bw = bandwidth(n, rowptr, col, pinv.data());
            int32_t wcap = (prm.dtypes & PARS3_DTYPE_BIT(PARS3_F64)) ? 4096 : 8192;
            auto_cut(bw, 32, wcap, 1024, &prm.T, &prm.W);
        }
        if (!is_pow2(prm.T) || !is_pow2(prm.W) || prm.W < 32 || prm.W > prm.T || prm.T > 32768) {
            delete h;
            return PARS3_EINVAL;
        }
        h->T = prm.T;
        h->W = prm.W;
        h->ntiles = n > 0 ? (n + prm.T - 1) / prm.T : 0;
        h->long_row = prm.long_row > 0 ? prm.long_row : std::max(2048, 4 * prm.T);
        rc = canonical_split(h, rowptr, col, val);
        if (rc == PARS3_OK) rc = build_layout(h);
        if (rc != PARS3_OK) { delete h; return rc; }
    } catch (const std::bad_alloc &) {
        delete h;
        return PARS3_ENOMEM;
    }
    *out = h;
    return PARS3_OK;
}

extern "C" int pars3_split_export(const pars3_handle *h, pars3_canonical *o) {
    if (!h || !o) return PARS3_EINVAL;
    o->n = h->n;
    o->T = h->T;
    o->W = h->W;
    o->ntiles = h->ntiles;
    o->nnz = h->nnz;
    for (int k = 0; k < 3; ++k) o->counts[k] = h->counts[k];
    o->perm = h->perm.data();
    o->rowptr = h->rowptr.data();
    o->col = h->col.data();
    o->val = h->val.data();
    o->cls = h->cls.data();
    o->tile_ptr = h->tile_ptr.data();
    o->tile_list = h->tile_list.data();
    o->outer_csr = h->outer_csr.data();
    o->outer_csc = h->outer_csc.data();
    return PARS3_OK;
}

extern "C" int pars3_info_get(const pars3_handle *h, pars3_info *o) {
    if (!h || !o) return PARS3_EINVAL;
    std::memset(o, 0, sizeof(*o));
    o->n = h->n;
    o->T = h->T;
    o->W = h->W;
    o->ntiles = h->ntiles;
    o->dtypes = h->dtypes;
    o->nnz = h->nnz;
    int64_t hsum = 0;
    for (int32_t c : h->L.hcnt) hsum += c;
    o->half_entries = hsum;
    o->full_entries = static_cast<int64_t>(h->L.fcol.size());
    o->long_entries = static_cast<int64_t>(h->L.lcol.size());
    o->long_rows = static_cast<int32_t>(h->L.lrow.size());
    o->long_chunks = static_cast<int32_t>(h->L.lcbeg.size());
    o->halo_targets = static_cast<int64_t>(h->L.hhrow.size());
    o->max_tile_half = h->L.max_tile_half;
    for (int d = 0; d < kNumDtypes; ++d) {
        o->smem_bytes[d] = (h->dtypes & PARS3_DTYPE_BIT(d)) ? smem_bytes_for(h, d) : 0;
        o->bytes_per_spmv[d] = model_bytes(h, d);
    }
    o->device_bytes = h->D.bytes;
    o->bandwidth = h->bw;
    return PARS3_OK;
}

// Reconstruct the signed entry multiset of every path and compare it with
// the canonical split.
extern "C" int pars3_layout_check(const pars3_handle *h) {
    if (!h) return PARS3_EINVAL;
    const Layout &L = h->L;
    const int32_t n = h->n, T = h->T, W = h->W;
    const double *v64 = L.hval64.empty() ? nullptr : L.hval64.data();
    try {
        // expected multiset: (row, col, value) for every entry and its mirror
        struct E { int32_t r, c; double v; };
        std::vector<E> want, got;
        want.reserve(2 * h->nnz);
        for (int32_t i = 0; i < n; ++i)
            for (int32_t e = h->rowptr[i]; e < h->rowptr[i + 1]; ++e) {
                want.push_back({i, h->col[e], h->val[e]});
                want.push_back({h->col[e], i, -h->val[e]});
            }
        got.reserve(2 * h->nnz);
        for (int32_t t = 0; t < h->ntiles; ++t) {
            int32_t r0 = t * T, r1 = std::min(n, r0 + T), wb = r0 - W;
            const uint16_t *lrp = &L.hrp[static_cast<size_t>(t) * (T + 8)];
            if (lrp[r1 - r0] != L.hcnt[t]) return PARS3_EINVAL;
            std::vector<uint8_t> used(L.hcnt[t], 0);
            for (int32_t i = r0; i < r1; ++i)
                for (int32_t q = lrp[i - r0]; q < lrp[i - r0 + 1]; ++q) {
                    int32_t j = wb + L.hcol[L.hoff[t] + q];
                    if (j < std::max(wb, 0) || j >= i || i - j > W) return PARS3_EINVAL;
                    double a = v64 ? v64[L.hoff[t] + q] : 0.0;
                    got.push_back({i, j, a});
                    got.push_back({j, i, -a});
                }
            for (int32_t q = 0; q < L.hcnt[t]; ++q) {
                uint16_t e = L.hcperm[L.hoff[t] + q];
                if (e >= L.hcnt[t] || used[e]) return PARS3_EINVAL;
                used[e] = 1;
                if (q > 0 && L.hcol[L.hoff[t] + e] < L.hcol[L.hoff[t] + L.hcperm[L.hoff[t] + q - 1]])
                    return PARS3_EINVAL;
            }
        }
        for (int32_t i = 0; i < n; ++i)
            for (int32_t q = L.frp[i]; q < L.frp[i + 1]; ++q)
                got.push_back({i, L.fcol[q], L.fval64.empty() ? 0.0 : L.fval64[q]});
        for (size_t l = 0; l < L.lrow.size(); ++l)
            for (int32_t c = L.lcptr[l]; c < L.lcptr[l + 1]; ++c)
                for (int32_t q = L.lcbeg[c]; q < L.lcend[c]; ++q)
                    got.push_back({L.lrow[l], L.lcol[q], L.lval64.empty() ? 0.0 : L.lval64[q]});
        if (got.size() != want.size()) return PARS3_EINVAL;
        auto key = [](const E &a, const E &b) { return a.r != b.r ? a.r < b.r : a.c < b.c; };
        std::sort(want.begin(), want.end(), key);
        std::sort(got.begin(), got.end(), key);
        for (size_t q = 0; q < got.size(); ++q) {
            if (got[q].r != want[q].r || got[q].c != want[q].c) return PARS3_EINVAL;
            if (v64 && got[q].v != want[q].v) return PARS3_EINVAL;
        }
    } catch (const std::bad_alloc &) {
        return PARS3_ENOMEM;
    }
    return PARS3_OK;
}
