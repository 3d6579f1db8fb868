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
//   full path  -- outer entries, and the middle entries of tiles too large
//                 for shared memory, stored in both rows with mirrored sign,
//                 so that each row is a plain gather (no write conflicts);
//                 sliced ELL: every row of a tile owns one lane of one of
//                 its T/32 slices (long rows with length 0);
//   long rows  -- rows longer than long_row (and the heaviest rows of tiles
//                 whose full-path entries exceed a cap) are cut into pieces
//                 of `piece` entries laid out like the tile slices (one lane
//                 per piece); the piece sums are folded in row order.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"
#include "smem_layout.h"

uint64_t next_handle_serial() {
    static std::atomic<uint64_t> counter{0};
    return ++counter;
}

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

// Stage 1 of the canonical split (independent of the cut points): apply
// the permutation, re-triangularize (an entry whose orientation flips is
// stored negated) and sort by (row, col) into h->rowptr/col/val.
static void canonical_reorder(pars3_handle *h, const int32_t *rowptr, const int32_t *col, const double *val) {
    const int32_t n = h->n;
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
            else       { r[e] = b; c[e] = a; v[e] = h->symmetric ? val[k] : -val[k]; }
        }
    }
    // sort by (row, col): bucket by row (one counting pass), then sort each
    // row's columns (short segments, no duplicates after validation)
    h->rowptr.assign(static_cast<size_t>(n) + 1, 0);
    for (int64_t e = 0; e < nnz; ++e) ++h->rowptr[r[e] + 1];
    for (int32_t i = 0; i < n; ++i) h->rowptr[i + 1] += h->rowptr[i];
    h->col.resize(nnz);
    h->val.resize(nnz);
    {
        // (col, source position) pairs bucketed by row, then each row sorted
        std::vector<std::pair<int32_t, int32_t>> pr(nnz);
        std::vector<int32_t> fill(h->rowptr.begin(), h->rowptr.end() - 1);
        for (int64_t e = 0; e < nnz; ++e) pr[fill[r[e]]++] = {c[e], static_cast<int32_t>(e)};
        for (int32_t i = 0; i < n; ++i) {
            const int32_t b = h->rowptr[i], en = h->rowptr[i + 1];
            if (en - b > 1) std::sort(pr.begin() + b, pr.begin() + en);
        }
        for (int64_t q = 0; q < nnz; ++q) {
            h->col[q] = pr[q].first;
            h->val[q] = v[pr[q].second];
        }
    }
}

// Stage 2 (for the cut points h->T, h->W): class of every stored entry,
// per-tile middle lists in (col, row) order, outer lists in CSR and CSC order.
static void canonical_classify(pars3_handle *h) {
    const int32_t n = h->n, T = h->T, W = h->W;
    const int64_t nnz = h->nnz;
    std::vector<int32_t> row_of(nnz);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t e = h->rowptr[i]; e < h->rowptr[i + 1]; ++e) row_of[e] = i;
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
    // per-tile middle lists in (col, row) order: the middle entries of a tile
    // are a run of CSR positions in (row, col) order; sort each run by
    // (col, row) (positions increase with row inside a column)
    std::vector<int32_t> mid, outer;
    mid.reserve(h->counts[0] + h->counts[1]);
    outer.reserve(h->counts[2]);
    h->tile_ptr.assign(static_cast<size_t>(h->ntiles) + 1, 0);
    for (int32_t t = 0; t < h->ntiles; ++t) {
        const int32_t r0 = t * T, r1 = std::min(n, r0 + T);
        const size_t m0 = mid.size();
        for (int32_t e = h->rowptr[r0]; e < h->rowptr[r1]; ++e) {
            if (h->cls[e] != 2) mid.push_back(e);
            else outer.push_back(e);
        }
        std::sort(mid.begin() + m0, mid.end(), [&](int32_t x, int32_t y) {
            return h->col[x] != h->col[y] ? h->col[x] < h->col[y] : x < y;
        });
        h->tile_ptr[t + 1] = static_cast<int32_t>(mid.size());
    }
    h->tile_list.swap(mid);
    h->outer_csr = outer;
    counting_sort(outer, n, [&](int32_t e) { return h->col[e]; });
    h->outer_csc.swap(outer);
    h->bw = 0;
    for (int64_t e = 0; e < nnz; ++e) h->bw = std::max<int64_t>(h->bw, row_of[e] - h->col[e]);
}

void dtype_sizes(int dtype, uint32_t *vsz, uint32_t *xsz, uint32_t *asz) {
    if (dtype == PARS3_F64) { *vsz = 8; *xsz = 8; *asz = 8; }
    else if (dtype == PARS3_F32) { *vsz = 4; *xsz = 4; *asz = 4; }
    else { *vsz = 2; *xsz = 4; *asz = 4; }
}

static uint32_t smem_total(const pars3_handle *h, int dtype, int64_t Mh, int64_t CS) {
    uint32_t vsz, xsz, asz;
    dtype_sizes(dtype, &vsz, &xsz, &asz);
    return smem_layout(h->T, h->W, static_cast<uint32_t>(round_up(Mh, kAlignHalf)), static_cast<uint32_t>(CS), vsz,
                       xsz, asz).total;
}

int smem_bytes_for(const pars3_handle *h, int dtype) {
    return static_cast<int>(smem_total(h, dtype, h->L.max_tile_half, h->L.max_tile_cs));
}

// Dynamic shared memory of the plain product's tile kernel.  When no tile
// has middle entries on the half path, nothing is staged: fp64 tiles keep
// no row sums in shared memory either (each lane stores its row), fp32 /
// bf16 tiles only their row sums; the rest of the SM's shared memory then
// serves as L1 for the gathers of x.
int spmv_smem_bytes(const pars3_handle *h, int dtype) {
    if (h->L.max_tile_half > 0) return smem_bytes_for(h, dtype);
    if (dtype == PARS3_F64) return 0;
    uint32_t vsz, xsz, asz;
    dtype_sizes(dtype, &vsz, &xsz, &asz);
    const SmemLayout s = smem_layout(h->T, h->W, 0u, 0u, vsz, xsz, asz);
    return static_cast<int>(s.rowacc + static_cast<uint32_t>(h->T) * asz);
}

int max_smem_all(const pars3_handle *h) {
    int m = 0;
    for (int d = 0; d < kNumDtypes; ++d)
        if (h->dtypes & PARS3_DTYPE_BIT(d)) m = std::max(m, smem_bytes_for(h, d));
    return m;
}

// half-path entries a tile may hold, for every packed precision
int64_t half_room(const pars3_handle *h) {
    int64_t best = INT64_MAX;
    for (int d = 0; d < kNumDtypes; ++d) {
        if (!(h->dtypes & PARS3_DTYPE_BIT(d))) continue;
        uint32_t vsz, xsz, asz;
        dtype_sizes(d, &vsz, &xsz, &asz);
        const int64_t base = smem_total(h, d, 8, 8) - 8 * (vsz + 6);   // the fixed part of a half-path layout
        const int64_t per = vsz + 6 + 4;   // value, column, (column, row) order, row, at most a segment word
        const int64_t room = static_cast<int64_t>(kSmemLimit) - base - 1024;
        best = std::min<int64_t>(best, room > 0 ? room / per : -1);
    }
    return std::min<int64_t>(best, 65535 - kAlignHalf);
}

// ---- decisions of the layout build that look at rows and tiles only; the
// host builder below and the GPU builder (device_split.cu) both use them

// Step 1: tcount[t] holds the middle entries of tile t on entry.  A tile
// whose middle entries do not fit shared memory (more than mcap), or are too
// few to repay staging the x window (under 1/kHalfMinFrac of the tile's
// stored entries), takes them on the full path (tcount[t] = 0).  The launch
// reserves the largest tile's staging area for every block, which takes
// that shared memory away from L1 on every SM: when the half path would hold
// under 1/kHalfMinShare of all stored entries it is not used at all.  Fills
// hoff, hcnt and max_tile_half.
void half_tiles(pars3_handle *h, int64_t mcap, std::vector<int32_t> &tcount) {
    Layout &L = h->L;
    const int32_t n = h->n, T = h->T, nt = h->ntiles;
    const std::vector<int32_t> &rp = h->rowptr;
    for (int32_t t = 0; t < nt; ++t) {
        const int32_t r0 = t * T, r1 = std::min(n, r0 + T);
        const int64_t stored = static_cast<int64_t>(rp[r1]) - rp[r0];
        if (tcount[t] > mcap || static_cast<int64_t>(tcount[t]) * kHalfMinFrac < stored) tcount[t] = 0;
    }
    int64_t hsum = 0;
    for (int32_t t = 0; t < nt; ++t) hsum += tcount[t];
    if (hsum * kHalfMinShare < h->nnz) std::fill(tcount.begin(), tcount.end(), 0);
    L.hoff.assign(static_cast<size_t>(nt) + 1, 0);
    L.hcnt.assign(nt, 0);
    for (int32_t t = 0; t < nt; ++t) {
        L.hcnt[t] = tcount[t];
        L.hoff[t + 1] = static_cast<int32_t>(L.hoff[t] + round_up(tcount[t], kAlignHalf));
        L.max_tile_half = std::max(L.max_tile_half, tcount[t]);
    }
}

// Step 3: long rows -- longer than the cap, or the heaviest rows of a tile
// whose full entries exceed the cap (rows of at least kLongMin entries,
// longest first, ties by index).  Sets cap_full.
void long_rows(pars3_handle *h, const std::vector<int32_t> &flen, int64_t ftotal, int64_t cap_in,
               std::vector<uint8_t> &is_long) {
    Layout &L = h->L;
    const int32_t n = h->n, T = h->T, nt = h->ntiles;
    const int64_t avg = nt > 0 ? (ftotal + nt - 1) / nt : 0;
    const int64_t cap = cap_in > 0 ? cap_in : std::max<int64_t>(2048, round_up(2 * avg, kAlignFull));
    L.cap_full = static_cast<int32_t>(std::min<int64_t>(cap, INT32_MAX));
    const int64_t long_thr = std::min<int64_t>(h->long_row > 0 ? h->long_row : kSellMax, kSellMax);
    is_long.assign(n, 0);
    for (int32_t i = 0; i < n; ++i)
        if (flen[i] > long_thr) is_long[i] = 1;
    for (int32_t t = 0; t < nt; ++t) {
        const int32_t r0 = t * T, r1 = std::min(n, r0 + T);
        int64_t f = 0;
        for (int32_t i = r0; i < r1; ++i)
            if (!is_long[i]) f += flen[i];
        if (f <= cap) continue;
        // balance: rows of at least kLongMin entries, longest first (ties by
        // index); then, if the tile is still above the cap, any row
        for (int pass = 0; pass < 2 && f > cap; ++pass) {
            std::vector<int32_t> cand;
            for (int32_t i = r0; i < r1; ++i)
                if (!is_long[i] && flen[i] > 0 && (pass == 1 || flen[i] >= kLongMin)) cand.push_back(i);
            std::sort(cand.begin(), cand.end(), [&](int32_t a, int32_t b) {
                return flen[a] != flen[b] ? flen[a] > flen[b] : a < b;
            });
            for (int32_t i : cand) {
                if (f <= cap) break;
                is_long[i] = 1;
                f -= flen[i];
            }
        }
    }
}

// Step 4: the sliced-ELL slices.  rows[r0 .. r1) lists tile t's rows sorted
// by full-path length slen (longest first, ties by row); every row of a tile
// gets a lane, so the full pass can start each row's sum with alpha x_r.
// row_base[i] receives the slot of row i's first entry (-1 when it has none).
int slice_rows(pars3_handle *h, const std::vector<int32_t> &rows, const std::vector<int32_t> &slen,
               std::vector<int32_t> &row_base) {
    Layout &L = h->L;
    const int32_t n = h->n, T = h->T, nt = h->ntiles;
    L.sl_off.assign(static_cast<size_t>(nt) + 1, 0);
    L.sl_ent.assign(1, 0);
    L.sl_meta.clear();
    L.sl_e.clear();
    row_base.assign(n, -1);
    for (int32_t t = 0; t < nt; ++t) {
        const int32_t r0 = t * T, r1 = std::min(n, r0 + T);
        int64_t tile_ent = 0;
        for (int32_t g = r0; g < r1; g += kSlice) {
            const int32_t width = slen[rows[g]];
            const int64_t start = L.sl_ent.back();
            const int64_t next = start + static_cast<int64_t>(kSlice) * width;
            if (next > INT32_MAX - kSlice) return PARS3_EUNSUPPORTED;   // int32 slot offsets
            L.sl_ent.push_back(static_cast<int32_t>(next));
            for (int l = 0; l < kSlice; ++l) {
                const int32_t k = g + l;
                if (k < r1) {
                    const int32_t i = rows[k];
                    L.sl_meta.push_back(static_cast<uint32_t>(i - r0) | (static_cast<uint32_t>(slen[i]) << 16));
                    if (slen[i] > 0) row_base[i] = static_cast<int32_t>(start + l);
                } else {
                    L.sl_meta.push_back(0xffffu);
                }
            }
            tile_ent += static_cast<int64_t>(kSlice) * width;
        }
        L.sl_off[t + 1] = static_cast<int32_t>(L.sl_ent.size() - 1);
        int32_t se = L.sl_off[t + 1];
        while (se > L.sl_off[t] && L.sl_ent[se] == L.sl_ent[se - 1]) --se;
        L.sl_e.push_back(se);
        L.max_tile_full = static_cast<int32_t>(std::max<int64_t>(L.max_tile_full, tile_ent));
        L.max_tile_slices = std::max(L.max_tile_slices, L.sl_off[t + 1] - L.sl_off[t]);
    }
    return PARS3_OK;
}

// Step 5: long rows in row order (lrow, lrp) and their pieces: full pieces
// in row order, then the shorter last pieces, longest first (ties by row);
// lp0, lrem, the long slices (ls_ent: a slice is as wide as its first, i.e.
// longest, piece) and every piece's length.
int long_pieces(pars3_handle *h, const std::vector<uint8_t> &is_long, const std::vector<int32_t> &flen,
                std::vector<PieceRef> &pieces) {
    Layout &L = h->L;
    const int32_t n = h->n;
    L.lrow.clear();
    L.lrp.assign(1, 0);
    for (int32_t i = 0; i < n; ++i)
        if (is_long[i]) {
            L.lrow.push_back(i);
            L.lrp.push_back(static_cast<int32_t>(std::min<int64_t>(static_cast<int64_t>(L.lrp.back()) + flen[i],
                                                                   INT32_MAX)));
        }
    const size_t nlong = L.lrow.size();
    if (L.lrp.back() >= INT32_MAX / 2) return PARS3_EUNSUPPORTED;   // int32 entry offsets
    const int32_t P = h->piece > 0 ? h->piece : kPieceLen;
    L.piece_len = P;
    std::vector<PieceRef> rest;
    pieces.clear();
    L.lp0.assign(nlong + 1, 0);
    L.lrem.assign(nlong, -1);
    for (size_t l = 0; l < nlong; ++l) {
        const int32_t len = L.lrp[l + 1] - L.lrp[l];
        int32_t q = 0;
        for (; q + P <= len; q += P) pieces.push_back({static_cast<int32_t>(l), L.lrp[l] + q, P});
        L.lp0[l + 1] = static_cast<int32_t>(pieces.size());
        if (q < len) rest.push_back({static_cast<int32_t>(l), L.lrp[l] + q, len - q});
    }
    std::stable_sort(rest.begin(), rest.end(), [](const PieceRef &a, const PieceRef &b) { return a.len > b.len; });
    for (const PieceRef &pc : rest) {
        L.lrem[pc.l] = static_cast<int32_t>(pieces.size());
        pieces.push_back(pc);
    }
    const int64_t npieces = static_cast<int64_t>(pieces.size());
    const int64_t nls = (npieces + kSlice - 1) / kSlice;
    if (nls * kSlice > INT32_MAX / 2) return PARS3_EUNSUPPORTED;
    L.ls_ent.assign(1, 0);
    L.ls_len.assign(static_cast<size_t>(nls) * kSlice, 0);
    for (int64_t sl = 0; sl < nls; ++sl) {
        const int64_t width = pieces[static_cast<size_t>(sl * kSlice)].len;   // the slice's longest piece
        const int64_t next = L.ls_ent.back() + width * kSlice;
        if (next > INT32_MAX - kSlice) return PARS3_EUNSUPPORTED;
        L.ls_ent.push_back(static_cast<int32_t>(next));
    }
    for (int64_t p = 0; p < npieces; ++p) L.ls_len[p] = static_cast<uint16_t>(pieces[static_cast<size_t>(p)].len);
    L.nslots = nls * kSlice;
    L.ls_per_block = h->lsb > 0 ? h->lsb : kLongSlices;
    return PARS3_OK;
}

// Step 6: fold items, each receiving row once, in row order.
void fold_items(pars3_handle *h) {
    Layout &L = h->L;
    const int32_t n = h->n;
    std::vector<int32_t> hidx(n, -1), lidx(n, -1);
    for (size_t k = 0; k < L.hhrow.size(); ++k) hidx[L.hhrow[k]] = static_cast<int32_t>(k);
    for (size_t l = 0; l < L.lrow.size(); ++l) lidx[L.lrow[l]] = static_cast<int32_t>(l);
    L.fold_row.clear();
    L.fold_halo.clear();
    L.fold_p0.clear();
    L.fold_np.clear();
    L.fold_rem.clear();
    L.fold_heavy.clear();
    for (int32_t i = 0; i < n; ++i)
        if (hidx[i] >= 0 || lidx[i] >= 0) {
            const int32_t l = lidx[i];
            L.fold_row.push_back(i);
            L.fold_halo.push_back(hidx[i]);
            L.fold_p0.push_back(l >= 0 ? L.lp0[l] : 0);
            L.fold_np.push_back(l >= 0 ? L.lp0[l + 1] - L.lp0[l] : 0);
            L.fold_rem.push_back(l >= 0 ? L.lrem[l] : -1);
            if (L.fold_np.back() >= kFoldHeavy) L.fold_heavy.push_back(static_cast<int32_t>(L.fold_row.size()) - 1);
        }
}

static int build_layout_try(pars3_handle *h, int64_t mcap_in, int64_t cap_in) {
    Layout &L = h->L;
    L = Layout();
    const int32_t n = h->n, T = h->T, W = h->W, nt = h->ntiles;
    const int64_t nnz = h->nnz;
    const std::vector<int32_t> &rp = h->rowptr;
    const std::vector<int32_t> &ci = h->col;
    std::vector<int32_t> row_of(nnz);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) row_of[e] = i;
    // column view of the band CSR: entries of column j in increasing row
    std::vector<int32_t> cptr(static_cast<size_t>(n) + 1, 0);
    for (int64_t e = 0; e < nnz; ++e) ++cptr[ci[e] + 1];
    for (int32_t j = 0; j < n; ++j) cptr[j + 1] += cptr[j];
    std::vector<int32_t> cent(nnz);
    {
        std::vector<int32_t> fill(cptr.begin(), cptr.end() - 1);
        for (int64_t e = 0; e < nnz; ++e) cent[fill[ci[e]]++] = static_cast<int32_t>(e);
    }
    // ---- 1. half path: middle entries, unless the tile would not fit
    std::vector<int32_t> tcount(nt, 0);
    for (int64_t e = 0; e < nnz; ++e)
        if (h->cls[e] != 2) ++tcount[row_of[e] / T];
    half_tiles(h, mcap_in, tcount);
    std::vector<uint8_t> half(nnz, 0);
    for (int64_t e = 0; e < nnz; ++e) half[e] = h->cls[e] != 2 && tcount[row_of[e] / T] > 0;
    const int64_t hn = L.hoff[nt];
    L.hcol.assign(hn, 0);
    L.hcperm.assign(hn, 0);
    L.hrowc.assign(hn, 0);
    L.hrp.assign(static_cast<size_t>(nt) * (T + 8), 0);
    std::vector<int32_t> hsrc(hn, 0);   // entry + 1 (0 = padding)
    std::vector<int32_t> hpos(nnz, -1);
    for (int32_t t = 0; t < nt; ++t) {
        const int32_t r0 = t * T, r1 = std::min(n, r0 + T), wb = r0 - W;
        int32_t q = 0;
        uint16_t *lrp = &L.hrp[static_cast<size_t>(t) * (T + 8)];
        for (int32_t i = r0; i < r1; ++i) {
            lrp[i - r0] = static_cast<uint16_t>(q);
            for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
                if (!half[e]) continue;
                hpos[e] = L.hoff[t] + q;
                hsrc[L.hoff[t] + q] = e + 1;
                L.hcol[L.hoff[t] + q] = static_cast<uint16_t>(ci[e] - wb);
                ++q;
            }
        }
        for (int32_t i = r1; i <= r0 + T + 7; ++i) lrp[i - r0] = static_cast<uint16_t>(q);
    }
    // (column, row) order of each tile's middle entries, the window position
    // of each one's row, and the column segments: one word per distinct
    // column (window position | first (column, row) index << 16), in column
    // order, then an end word (0xffff | count << 16); the tile's halo columns
    // (positions below W) are its first segments, in the order of its halo
    // targets
    L.hhoff.assign(static_cast<size_t>(nt) + 1, 0);
    L.hcsoff.assign(static_cast<size_t>(nt) + 1, 0);
    L.hcs.clear();
    L.hcsn.clear();
    L.max_tile_cs = 0;
    for (int32_t t = 0; t < nt; ++t) {
        const int32_t r0 = t * T, wb = r0 - W;
        int32_t q = 0, last = -1;
        for (int32_t s = h->tile_ptr[t]; s < h->tile_ptr[t + 1]; ++s) {
            const int32_t e = h->tile_list[s];
            if (!half[e]) continue;
            L.hcperm[L.hoff[t] + q] = static_cast<uint16_t>(hpos[e] - L.hoff[t]);
            L.hrowc[L.hoff[t] + q] = static_cast<uint16_t>(row_of[e] - wb);
            const int32_t j = ci[e];
            if (j != last) L.hcs.push_back(static_cast<uint32_t>(j - wb) | (static_cast<uint32_t>(q) << 16));
            if (j < r0 && j != last) L.hhrow.push_back(j);
            last = j;
            ++q;
        }
        L.hhoff[t + 1] = static_cast<int32_t>(L.hhrow.size());
        L.hcs.push_back(0xffffu | (static_cast<uint32_t>(q) << 16));
        L.hcsn.push_back(static_cast<int32_t>(L.hcs.size()) - L.hcsoff[t] - 1);   // segments (not the end word)
        while (L.hcs.size() % 4) L.hcs.push_back(0xffffu | (static_cast<uint32_t>(q) << 16));
        L.hcsoff[t + 1] = static_cast<int32_t>(L.hcs.size());
        L.max_tile_cs = std::max(L.max_tile_cs, L.hcsoff[t + 1] - L.hcsoff[t]);
    }
    // ---- 2. full-path length of every row: its non-half lower entries and the
    // non-half entries of its column (mirrored)
    std::vector<int32_t> flen(n, 0);
    int64_t ftotal = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t c = 0;
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) c += !half[e];
        for (int32_t s = cptr[i]; s < cptr[i + 1]; ++s) c += !half[cent[s]];
        flen[i] = c;
        ftotal += c;
    }
    // ---- 3. long rows
    std::vector<uint8_t> is_long;
    long_rows(h, flen, ftotal, cap_in, is_long);
    // ---- 4. full path per tile as sliced ELL (rows sorted by length, longest first)
    auto emit_row = [&](int32_t i, int32_t *colp, int32_t *srcp, int64_t stride) {
        int64_t q = 0;
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e)
            if (!half[e]) { colp[q * stride] = ci[e]; srcp[q * stride] = e + 1; ++q; }
        for (int32_t s2 = cptr[i]; s2 < cptr[i + 1]; ++s2) {
            const int32_t e = cent[s2];
            if (!half[e]) { colp[q * stride] = row_of[e]; srcp[q * stride] = -(e + 1); ++q; }
        }
        return q;
    };
    std::vector<int32_t> slen(n), rows(n);
    for (int32_t i = 0; i < n; ++i) slen[i] = is_long[i] ? 0 : flen[i];
    for (int32_t t = 0; t < nt; ++t) {
        const int32_t r0 = t * T, r1 = std::min(n, r0 + T);
        for (int32_t i = r0; i < r1; ++i) rows[i] = i;
        std::sort(rows.begin() + r0, rows.begin() + r1, [&](int32_t a, int32_t b) {
            return slen[a] != slen[b] ? slen[a] > slen[b] : a < b;
        });
    }
    std::vector<int32_t> row_base;
    if (const int rc = slice_rows(h, rows, slen, row_base); rc != PARS3_OK) return rc;
    const int64_t fnp = L.sl_ent.back();
    L.fcol.assign(fnp, 0);
    std::vector<int32_t> fsrc(fnp, 0);  // +(e+1): lower entry, -(e+1): mirrored entry, 0: padding
    for (int32_t t = 0; t < nt; ++t) {
        const int32_t r0 = t * T;
        for (int32_t s2 = L.sl_off[t]; s2 < L.sl_off[t + 1]; ++s2)
            for (int l = 0; l < kSlice; ++l) {
                const uint32_t meta = L.sl_meta[static_cast<size_t>(s2) * kSlice + l];
                if ((meta & 0xffffu) == 0xffffu || (meta >> 16) == 0) continue;
                const int32_t i = r0 + static_cast<int32_t>(meta & 0xffffu);
                emit_row(i, &L.fcol[L.sl_ent[s2] + l], &fsrc[L.sl_ent[s2] + l], kSlice);
            }
    }
    // ---- 5. long rows, concatenated in row order and cut into pieces
    std::vector<PieceRef> pieces;
    if (const int rc = long_pieces(h, is_long, flen, pieces); rc != PARS3_OK) return rc;
    const size_t nlong = L.lrow.size();
    const int64_t ltot = L.lrp.back();
    std::vector<int32_t> lflat(ltot), lsrc_flat(ltot);
    for (size_t l = 0; l < nlong; ++l) emit_row(L.lrow[l], &lflat[L.lrp[l]], &lsrc_flat[L.lrp[l]], 1);
    const int64_t npieces = static_cast<int64_t>(pieces.size());
    L.lcol.assign(static_cast<size_t>(L.ls_ent.back()), 0);
    std::vector<int32_t> lsrc(L.lcol.size(), 0);
    for (int64_t p = 0; p < npieces; ++p) {
        const PieceRef &pc = pieces[static_cast<size_t>(p)];
        const int64_t base = L.ls_ent[p / kSlice] + (p % kSlice);
        for (int32_t m = 0; m < pc.len; ++m) {
            L.lcol[base + static_cast<int64_t>(m) * kSlice] = lflat[pc.e0 + m];
            lsrc[base + static_cast<int64_t>(m) * kSlice] = lsrc_flat[pc.e0 + m];
        }
    }
    // ---- 6. fold items: each receiving row once, in row order
    fold_items(h);
    // ---- 7. values per precision
    auto fill_vals = [&](const std::vector<int32_t> &src, std::vector<double> &v64, std::vector<float> &v32,
                         std::vector<uint16_t> &v16) {
        const size_t m = src.size();
        if (h->dtypes & PARS3_DTYPE_BIT(PARS3_F64)) v64.assign(m, 0.0);
        if (h->dtypes & PARS3_DTYPE_BIT(PARS3_F32)) v32.assign(m, 0.0f);
        if (h->dtypes & PARS3_DTYPE_BIT(PARS3_BF16)) v16.assign(m, 0);
        for (size_t q = 0; q < m; ++q) {
            const int32_t s = src[q];
            if (s == 0) continue;
            const double a = s > 0 ? h->val[s - 1] : (h->symmetric ? h->val[-s - 1] : -h->val[-s - 1]);
            const float f = static_cast<float>(a);
            if (!v64.empty()) v64[q] = a;
            if (!v32.empty()) v32[q] = f;
            if (!v16.empty()) v16[q] = f32_to_bf16_rne(f);
        }
    };
    fill_vals(hsrc, L.hval64, L.hval32, L.hval16);
    fill_vals(fsrc, L.fval64, L.fval32, L.fval16);
    fill_vals(lsrc, L.lval64, L.lval32, L.lval16);
    return PARS3_OK;
}

// Largest layout that fits: start with every middle entry of a fitting tile
// on the half path; while the tile block does not fit in shared memory,
// halve the largest half-path tile (more middle tiles become full storage).
int build_layout(pars3_handle *h) {
    int64_t mcap = half_room(h);
    if (mcap < 0) return PARS3_EUNSUPPORTED;
    for (int iter = 0; iter < 40; ++iter) {
        int rc = build_layout_try(h, mcap, 0);
        if (rc != PARS3_OK) return rc;
        if (max_smem_all(h) <= kSmemLimit) return PARS3_OK;
        if (h->L.max_tile_half == 0) return PARS3_EUNSUPPORTED;
        mcap = h->L.max_tile_half / 2;
    }
    return PARS3_EUNSUPPORTED;
}

int64_t model_bytes(const pars3_handle *h, int dtype) {
    if (!(h->dtypes & PARS3_DTYPE_BIT(dtype))) return 0;
    const Layout &L = h->L;
    const int64_t sv = dtype == PARS3_F64 ? 8 : (dtype == PARS3_F32 ? 4 : 2);
    const int64_t sx = dtype == PARS3_F64 ? 8 : 4;
    int64_t b = 0;
    b += static_cast<int64_t>(L.hcol.size()) * (sv + 2 + 2);               // half values, columns, order
    b += static_cast<int64_t>(L.fcol.size()) * (sv + 4);                   // full rows (sliced ELL)
    b += static_cast<int64_t>(L.sl_meta.size()) * 4 + static_cast<int64_t>(L.sl_ent.size()) * 4;
    b += static_cast<int64_t>(L.lcol.size()) * (sv + 4);                   // long-row pieces
    b += L.nslots * (2 + 2 * (sv == 8 ? 8 : 4));                            // piece lengths, sums out and in
    b += static_cast<int64_t>(h->ntiles) * (h->T + 8) * 2;                 // tile row pointers
    b += 2 * static_cast<int64_t>(h->n) * sx;                              // x once, y once
    return b;
}

}  // namespace pars3

namespace pars3 {

// Layout parameters of a split (everything but the cut points and the
// packed precisions): PARS3_OK or PARS3_EINVAL.
int check_layout_params(const pars3_split_params &p) {
    if (p.long_row < 0 || p.piece < 0 || (p.piece > 0 && (p.piece < 8 || p.piece > kPieceMax))) return PARS3_EINVAL;
    if (p.long_slices < 0 || p.long_slices > 1024) return PARS3_EINVAL;
    if (!(p.lane_bytes == 0 || p.lane_bytes == 4 || p.lane_bytes == 8 || p.lane_bytes == 16 || p.lane_bytes == 32))
        return PARS3_EINVAL;
    if (p.variant != 0 && p.variant != PARS3_VARIANT_LOOKAHEAD) return PARS3_EINVAL;
    return PARS3_OK;
}

void set_layout_params(pars3_handle *h, const pars3_split_params &p) {
    h->long_row = p.long_row > 0 ? p.long_row : 0;
    h->piece = p.piece;
    h->lsb = p.long_slices;
    h->lane_bytes = p.lane_bytes;
    h->variant = p.variant;
}

// Checks and normalises the parameters of a split (dtypes 0 -> F64 only):
// PARS3_OK or PARS3_EINVAL.  T = W = 0, the default cut rule, passes.
int split_params_normalize(pars3_split_params *prm) {
    if (prm->dtypes == 0) prm->dtypes = PARS3_DTYPE_BIT(PARS3_F64);
    if (prm->dtypes & ~7) return PARS3_EINVAL;
    if (prm->flags & ~PARS3_SPLIT_SYMMETRIC) return PARS3_EINVAL;
    if ((prm->T == 0) != (prm->W == 0)) return PARS3_EINVAL;
    return check_layout_params(*prm);
}

int check_cut(int32_t T, int32_t W) {
    return (!is_pow2(T) || !is_pow2(W) || W < 32 || W > T || T > 32768) ? PARS3_EINVAL : PARS3_OK;
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
    if (split_params_normalize(&prm) != PARS3_OK) return PARS3_EINVAL;
    pars3_handle *h = nullptr;
    try {
        h = new pars3_handle();
        h->n = n;
        h->nnz = nnz;
        h->dtypes = prm.dtypes;
        h->symmetric = (prm.flags & PARS3_SPLIT_SYMMETRIC) ? 1 : 0;
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
            int32_t wcap = (prm.dtypes & PARS3_DTYPE_BIT(PARS3_F64)) ? 1024 : 2048;
            auto_cut(bw, 32, wcap, 1024, &prm.T, &prm.W);
        }
        if (check_cut(prm.T, prm.W) != PARS3_OK) {
            delete h;
            return PARS3_EINVAL;
        }
        h->T = prm.T;
        h->W = prm.W;
        h->ntiles = n > 0 ? (n + prm.T - 1) / prm.T : 0;
        set_layout_params(h, prm);
        canonical_reorder(h, rowptr, col, val);
        canonical_classify(h);
        rc = build_layout(h);
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
    int64_t hsum = 0, fsum = 0;
    for (int32_t c : h->L.hcnt) hsum += c;
    for (uint32_t m : h->L.sl_meta)
        if ((m & 0xffffu) != 0xffffu) fsum += m >> 16;
    o->half_entries = hsum;
    o->full_entries = fsum;
    o->long_entries = h->L.lrp.empty() ? 0 : h->L.lrp.back();
    o->long_rows = static_cast<int32_t>(h->L.lrow.size());
    o->long_pieces = h->L.lrow.empty() ? 0 : h->L.lp0.back() + static_cast<int32_t>(
        std::count_if(h->L.lrem.begin(), h->L.lrem.end(), [](int32_t r) { return r >= 0; }));
    o->halo_targets = static_cast<int64_t>(h->L.hhrow.size());
    o->max_tile_half = h->L.max_tile_half;
    for (int d = 0; d < kNumDtypes; ++d) {
        o->smem_bytes[d] = (h->dtypes & PARS3_DTYPE_BIT(d)) ? spmv_smem_bytes(h, d) : 0;
        o->bytes_per_spmv[d] = model_bytes(h, d);
    }
    o->device_bytes = h->D.bytes;
    o->bandwidth = h->bw;
    o->symmetric = h->symmetric;
    return PARS3_OK;
}

// Reconstruct the signed entry multiset of every path and compare it with
// the canonical split.
extern "C" int pars3_layout_check(const pars3_handle *h) {
    if (!h) return PARS3_EINVAL;
    const Layout &L = h->L;
    const int32_t n = h->n, T = h->T, W = h->W;
    const bool has64 = (h->dtypes & PARS3_DTYPE_BIT(PARS3_F64)) != 0;
    const double mirror = h->symmetric ? 1.0 : -1.0;
    try {
        struct E { int32_t r, c; double v; };
        std::vector<E> want, got;
        want.reserve(2 * h->nnz);
        for (int32_t i = 0; i < n; ++i)
            for (int32_t e = h->rowptr[i]; e < h->rowptr[i + 1]; ++e) {
                want.push_back({i, h->col[e], h->val[e]});
                want.push_back({h->col[e], i, mirror * h->val[e]});
            }
        got.reserve(2 * h->nnz);
        for (int32_t t = 0; t < h->ntiles; ++t) {
            const int32_t r0 = t * T, r1 = std::min(n, r0 + T), wb = r0 - W;
            const uint16_t *lrp = &L.hrp[static_cast<size_t>(t) * (T + 8)];
            if (lrp[r1 - r0] != L.hcnt[t] || L.hoff[t] % kAlignHalf) return PARS3_EINVAL;
            std::vector<uint8_t> used(L.hcnt[t], 0);
            for (int32_t i = r0; i < r1; ++i)
                for (int32_t q = lrp[i - r0]; q < lrp[i - r0 + 1]; ++q) {
                    const int32_t j = wb + L.hcol[L.hoff[t] + q];
                    if (j < std::max(wb, 0) || j >= i || i - j > W) return PARS3_EINVAL;
                    const double a = has64 ? L.hval64[L.hoff[t] + q] : 0.0;
                    got.push_back({i, j, a});
                    got.push_back({j, i, mirror * a});
                }
            for (int32_t q = 0; q < L.hcnt[t]; ++q) {
                const uint16_t e = L.hcperm[L.hoff[t] + q];
                if (e >= L.hcnt[t] || used[e]) return PARS3_EINVAL;
                used[e] = 1;
                if (q > 0 && L.hcol[L.hoff[t] + e] < L.hcol[L.hoff[t] + L.hcperm[L.hoff[t] + q - 1]])
                    return PARS3_EINVAL;
            }
            // the row of each (column, row) entry, and the column segments:
            // one per distinct column in order, covering the list, halo
            // columns first (one per halo target)
            {
                std::vector<int32_t> row_of_q(L.hcnt[t]);
                for (int32_t i = r0; i < r1; ++i)
                    for (int32_t q = lrp[i - r0]; q < lrp[i - r0 + 1]; ++q) row_of_q[q] = i;
                for (int32_t q = 0; q < L.hcnt[t]; ++q)
                    if (wb + L.hrowc[L.hoff[t] + q] != row_of_q[L.hcperm[L.hoff[t] + q]]) return PARS3_EINVAL;
                const uint32_t *cs = &L.hcs[L.hcsoff[t]];
                const int32_t ncs = L.hcsoff[t + 1] - L.hcsoff[t];
                int32_t s = 0, k = 0, nhalo = 0;
                for (; s < ncs && (cs[s] & 0xffffu) != 0xffffu; ++s) {
                    const int32_t pos = static_cast<int32_t>(cs[s] & 0xffffu);
                    if (static_cast<int32_t>(cs[s] >> 16) != k) return PARS3_EINVAL;
                    if (s > 0 && pos <= static_cast<int32_t>(cs[s - 1] & 0xffffu)) return PARS3_EINVAL;
                    while (k < L.hcnt[t] && L.hcol[L.hoff[t] + L.hcperm[L.hoff[t] + k]] == pos) ++k;
                    if (k == static_cast<int32_t>(cs[s] >> 16)) return PARS3_EINVAL;   // empty segment
                    if (pos < W) {
                        if (L.hhoff[t] + nhalo >= L.hhoff[t + 1] || L.hhrow[L.hhoff[t] + nhalo] != wb + pos)
                            return PARS3_EINVAL;
                        ++nhalo;
                    }
                }
                if (k != L.hcnt[t] || s >= ncs || static_cast<int32_t>(cs[s] >> 16) != L.hcnt[t]) return PARS3_EINVAL;
                if (nhalo != L.hhoff[t + 1] - L.hhoff[t]) return PARS3_EINVAL;
            }
            std::vector<uint8_t> seen(r1 - r0, 0);
            for (int32_t s2 = L.sl_off[t]; s2 < L.sl_off[t + 1]; ++s2) {
                const int32_t width = (L.sl_ent[s2 + 1] - L.sl_ent[s2]) / kSlice;
                for (int l = 0; l < kSlice; ++l) {
                    const uint32_t meta = L.sl_meta[static_cast<size_t>(s2) * kSlice + l];
                    if ((meta & 0xffffu) == 0xffffu) continue;
                    const int32_t rl = static_cast<int32_t>(meta & 0xffffu), len = static_cast<int32_t>(meta >> 16);
                    if (rl >= r1 - r0 || seen[rl] || len > width || len > kSellMax) return PARS3_EINVAL;
                    seen[rl] = 1;
                    for (int32_t m = 0; m < len; ++m) {
                        const int64_t q = L.sl_ent[s2] + static_cast<int64_t>(m) * kSlice + l;
                        got.push_back({r0 + rl, L.fcol[q], has64 ? L.fval64[q] : 0.0});
                    }
                }
            }
            for (int32_t rl = 0; rl < r1 - r0; ++rl)
                if (!seen[rl]) return PARS3_EINVAL;   // every row owns a lane
            // slices from sl_e[t] on, and only those, have width 0
            if (L.sl_e[t] < L.sl_off[t] || L.sl_e[t] > L.sl_off[t + 1]) return PARS3_EINVAL;
            for (int32_t s2 = L.sl_off[t]; s2 < L.sl_off[t + 1]; ++s2)
                if ((L.sl_ent[s2 + 1] == L.sl_ent[s2]) != (s2 >= L.sl_e[t])) return PARS3_EINVAL;
        }
        // long rows: every piece of row l (its full pieces, then its last
        // piece) lies in the long slices with its length; together they hold
        // the row's entries
        const int64_t nslot = static_cast<int64_t>(L.nls()) * kSlice;
        if (static_cast<int64_t>(L.ls_len.size()) != nslot || L.nslots != nslot) return PARS3_EINVAL;
        std::vector<uint8_t> pseen(static_cast<size_t>(nslot), 0);
        for (size_t l = 0; l < L.lrow.size(); ++l) {
            std::vector<int32_t> ps;
            for (int32_t p = L.lp0[l]; p < L.lp0[l + 1]; ++p) ps.push_back(p);
            if (L.lrem[l] >= 0) ps.push_back(L.lrem[l]);
            int64_t cnt = 0;
            for (size_t u = 0; u < ps.size(); ++u) {
                const int32_t p = ps[u];
                if (p < 0 || p >= nslot || pseen[p]) return PARS3_EINVAL;
                pseen[p] = 1;
                const int32_t len = L.ls_len[p], s2 = p / kSlice, lane = p % kSlice;
                const int32_t width = (L.ls_ent[s2 + 1] - L.ls_ent[s2]) / kSlice;
                if (len < 1 || len > width || len > L.piece_len) return PARS3_EINVAL;
                if (u + 1 < ps.size() && len != L.piece_len) return PARS3_EINVAL;   // only the last is short
                for (int32_t m = 0; m < len; ++m) {
                    const int64_t q = L.ls_ent[s2] + static_cast<int64_t>(m) * kSlice + lane;
                    got.push_back({L.lrow[l], L.lcol[q], has64 ? L.lval64[q] : 0.0});
                }
                cnt += len;
            }
            if (cnt < 1 || cnt != L.lrp[l + 1] - L.lrp[l]) return PARS3_EINVAL;
        }
        for (int64_t p = 0; p < nslot; ++p)
            if (!pseen[p] && L.ls_len[p] != 0) return PARS3_EINVAL;   // padding lanes are empty
        if (got.size() != want.size()) return PARS3_EINVAL;
        auto key = [](const E &a, const E &b) { return a.r != b.r ? a.r < b.r : a.c < b.c; };
        std::sort(want.begin(), want.end(), key);
        std::sort(got.begin(), got.end(), key);
        for (size_t q = 0; q < got.size(); ++q) {
            if (got[q].r != want[q].r || got[q].c != want[q].c) return PARS3_EINVAL;
            if (has64 && got[q].v != want[q].v) return PARS3_EINVAL;
        }
        // fold items: rows strictly increasing, halo targets and long rows each once
        size_t nh = 0, nl = 0;
        for (size_t f = 0; f < L.fold_row.size(); ++f) {
            if (f > 0 && L.fold_row[f] <= L.fold_row[f - 1]) return PARS3_EINVAL;
            nh += L.fold_halo[f] >= 0;
            const bool has_long = L.fold_np[f] > 0 || L.fold_rem[f] >= 0;
            nl += has_long;
            if (has_long) {   // the row's pieces, as the long-row tables give them
                const auto it = std::lower_bound(L.lrow.begin(), L.lrow.end(), L.fold_row[f]);
                if (it == L.lrow.end() || *it != L.fold_row[f]) return PARS3_EINVAL;
                const size_t l = static_cast<size_t>(it - L.lrow.begin());
                if (L.fold_p0[f] != L.lp0[l] || L.fold_np[f] != L.lp0[l + 1] - L.lp0[l] || L.fold_rem[f] != L.lrem[l])
                    return PARS3_EINVAL;
            }
        }
        if (nh != L.hhrow.size() || nl != L.lrow.size()) return PARS3_EINVAL;
        // the heavy list: exactly the items of at least kFoldHeavy full pieces, in order
        {
            size_t q = 0;
            for (size_t f = 0; f < L.fold_row.size(); ++f)
                if (L.fold_np[f] >= kFoldHeavy) {
                    if (q >= L.fold_heavy.size() || L.fold_heavy[q] != static_cast<int32_t>(f)) return PARS3_EINVAL;
                    ++q;
                }
            if (q != L.fold_heavy.size()) return PARS3_EINVAL;
        }
    } catch (const std::bad_alloc &) {
        return PARS3_ENOMEM;
    }
    return PARS3_OK;
}
