// internal.h -- handle layout shared by the host preprocessing (C++) and the
// CUDA launchers of libpars3.  Not part of the public ABI (include/pars3.h).
#pragma once

#include <cstdint>
#include <vector>

#include "pars3.h"

namespace pars3 {

constexpr int kNumDtypes = 3;
constexpr int kAlignHalf = 8;          // half-path tile segments start on 16-byte boundaries (u16, bf16)
constexpr int kAlignFull = 16;         // full-path tile segments: 64 B for int32 columns, 128 B for fp64
constexpr int kBlock = 512;            // threads of the tile kernel (a row tile or a set of long-row slices)
constexpr int kPieceLen = 192;         // default entries per long-row piece
constexpr int kPieceMax = 255;         // longest piece the layout allows
constexpr int kLongSlices = 32;        // long-row slices per block
constexpr int kLongMin = 256;          // shortest row moved to the long path to balance tiles
constexpr int kSellMax = 128;          // longer full-path rows go to the long path
constexpr int kHalfMinFrac = 4;        // a tile keeps its middle entries on the half path only when they
                                       // are at least 1/kHalfMinFrac of its stored entries
constexpr int kHalfMinShare = 16;      // ... and the half path only when it holds 1/kHalfMinShare of all
constexpr int kFoldHeavy = 64;         // long rows of at least this many full pieces are folded by a warp
constexpr int kSlice = 32;             // rows per sliced-ELL slice (one warp)
constexpr int kSmemLimit = 227 * 1024; // opt-in shared memory per block on sm_100/sm_103

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// Device layout on the host side (vectors) and its device mirror.
struct Layout {
    // half path: per tile t, entries [hoff[t], hoff[t] + hcnt[t]) in (row, col) order
    std::vector<int32_t> hoff;      // [ntiles+1] (starts padded to kAlignHalf)
    std::vector<int32_t> hcnt;      // [ntiles]
    std::vector<uint16_t> hrp;      // [ntiles*(T+8)] tile-local row pointers
    std::vector<uint16_t> hcol;     // window position p = j - (tT - W)
    std::vector<uint16_t> hcperm;   // tile-local entry index, (col, row) order
    std::vector<uint16_t> hrowc;    // window position of the row of the k-th (col, row) entry
    std::vector<int32_t> hcsoff;    // [ntiles+1] column segments of tile t: hcs[hcsoff[t] ..]
    std::vector<int32_t> hcsn;      // [ntiles] number of column segments of tile t
    std::vector<uint32_t> hcs;      // window position | (first (col, row) index << 16), end word last
    std::vector<int32_t> hhoff;     // [ntiles+1] halo targets of tile t
    std::vector<int32_t> hhrow;     // global row of each halo target (sorted per tile)
    // full path, sliced ELL: the short rows of tile t, sorted by length
    // (longest first, ties by row), form 32-row slices sl_off[t] .. sl_off[t+1]-1;
    // slice s stores its entries slot-major at [sl_ent[s], sl_ent[s+1]) (slot m
    // of lane l at sl_ent[s] + 32 m + l); sl_meta[32 s + l] = tile-local row
    // | (row length << 16), row 0xffff for an empty lane
    std::vector<int32_t> sl_off;    // [ntiles+1]
    std::vector<int32_t> sl_ent;    // [nslices+1]
    std::vector<uint32_t> sl_meta;  // [nslices*32]
    std::vector<int32_t> fcol;
    std::vector<int32_t> sl_e;      // [ntiles] first slice of tile t whose rows are all empty (width 0);
                                    // slices sl_e[t] .. sl_off[t+1]-1 hold the rows without full entries
    // long rows: long row l is global row lrow[l]; its full-storage entries
    // (in the order of a tile row: lower entries, then mirrored ones), lrp[l]
    // .. lrp[l+1]-1 of the concatenated list (host only), are cut into pieces
    // of piece_len entries and a shorter last piece.  Pieces are laid out
    // like the tile slices: piece p is lane p % 32 of long slice p / 32, its
    // slot m at ls_ent[s] + 32 m + lane of lcol/lval, length ls_len[p].  The
    // full pieces come first, in row order (those of row l are lp0[l] ..
    // lp0[l+1]-1), then the last pieces, longest first (ties by row); lrem[l]
    // is row l's last piece or -1.  The sum of piece p goes to lpart[p].
    std::vector<int32_t> lrow;      // [nlong]
    std::vector<int32_t> lrp;       // [nlong+1] (host only)
    std::vector<int32_t> lp0;       // [nlong+1]
    std::vector<int32_t> lrem;      // [nlong]
    std::vector<int32_t> ls_ent;    // [nls+1]
    std::vector<uint16_t> ls_len;   // [nls*32]
    std::vector<int32_t> lcol;      // slot-major, padded slots hold column 0 and value 0
    int32_t piece_len = 0;
    int32_t ls_per_block = kLongSlices;   // long slices per block
    // fold items: one per row that receives a halo sum and/or long-row piece
    // sums: its halo index (or -1), its full pieces fold_p0 .. fold_p0 +
    // fold_np - 1 and its last piece fold_rem (or -1)
    std::vector<int32_t> fold_row, fold_halo, fold_p0, fold_np, fold_rem;
    std::vector<int32_t> fold_heavy;   // the fold items with at least kFoldHeavy full pieces
    // values per precision (fp64 / fp32 / bf16 bits)
    std::vector<double> hval64, fval64, lval64;
    std::vector<float> hval32, fval32, lval32;
    std::vector<uint16_t> hval16, fval16, lval16;
    int32_t max_tile_half = 0;
    int32_t max_tile_cs = 0;        // column segment words of the largest tile (multiple of 4)
    int32_t max_tile_full = 0;      // sliced-ELL entries (with padding) of the largest tile
    int32_t max_tile_slices = 0;
    int32_t cap_full = 0;
    int64_t nslots = 0;             // long-row piece sums (32 per long slice)
    int32_t nls() const { return ls_ent.empty() ? 0 : static_cast<int32_t>(ls_ent.size()) - 1; }
    int32_t nlong_blocks() const { return (nls() + ls_per_block - 1) / ls_per_block; }
};

struct DevLayout {
    int32_t *hoff = nullptr, *hcnt = nullptr;
    uint16_t *hrp = nullptr, *hcol = nullptr, *hcperm = nullptr, *hrowc = nullptr;
    int32_t *hcsoff = nullptr, *hcsn = nullptr;
    uint32_t *hcs = nullptr;
    int32_t *hhoff = nullptr, *hhrow = nullptr;
    int32_t *sl_off = nullptr, *sl_ent = nullptr, *sl_e = nullptr;
    uint32_t *sl_meta = nullptr;
    int32_t *fcol = nullptr;
    int32_t *ls_ent = nullptr;
    uint16_t *ls_len = nullptr;
    int32_t *lcol = nullptr;
    int32_t *fold_row = nullptr, *fold_halo = nullptr, *fold_p0 = nullptr, *fold_np = nullptr,
            *fold_rem = nullptr, *fold_heavy = nullptr;
    void *hval[kNumDtypes] = {nullptr, nullptr, nullptr};
    void *fval[kNumDtypes] = {nullptr, nullptr, nullptr};
    void *lval[kNumDtypes] = {nullptr, nullptr, nullptr};
    // scratch: halo sums and long-row piece sums (fp64-sized, scratch_k columns)
    void *halo = nullptr;
    void *lpart = nullptr;
    int32_t scratch_k = 0;
    int32_t *perm = nullptr;
    int32_t *err = nullptr;          // device error word
    // staging for pars3_spmv_host
    void *stage_x = nullptr, *stage_y = nullptr, *stage_px = nullptr, *stage_py = nullptr;
    int64_t bytes = 0;
    std::vector<void *> owned;       // everything to cudaFree
};

}  // namespace pars3

uint64_t next_handle_serial();

struct pars3_handle {
    uint64_t serial = next_handle_serial();   // unique per handle for the process lifetime
    int32_t n = 0;
    int64_t nnz = 0;
    int32_t T = 0, W = 0, ntiles = 0;
    int32_t dtypes = 0;
    int32_t long_row = 0;
    int32_t piece = 0;               // entries per long-row piece requested (0 = kPieceLen)
    int32_t lsb = 0;                 // long slices per block requested (0 = kLongSlices)
    int32_t lane_bytes = 0;          // SpMM bytes of X per lane (0 = rule)
    int32_t variant = 0;             // tile kernel variant (PARS3_VARIANT_*)
    int32_t symmetric = 0;           // S = L + L^T instead of L - L^T (mirror sign +1)
    int64_t bw = 0;
    // canonical split (host)
    std::vector<int32_t> perm, rowptr, col;
    std::vector<double> val;
    std::vector<uint8_t> cls;
    std::vector<int32_t> tile_ptr, tile_list, outer_csr, outer_csc;
    int64_t counts[3] = {0, 0, 0};
    // device layout
    pars3::Layout L;
    pars3::DevLayout D;
    bool uploaded = false;
    int device = -1;
    void *graph_cache = nullptr;     // MRS workspace and loop graphs (owned, see mrs.cu)
    void *batch_cache = nullptr;     // batched-launch argument table and graph (owned, see batched.cu)
};

namespace pars3 {

// host_reorder.cpp
int validate_lower(int32_t n, const int32_t *rowptr, const int32_t *col);
int64_t bandwidth(int32_t n, const int32_t *rowptr, const int32_t *col, const int32_t *pinv);

// host_split.cpp
int check_layout_params(const pars3_split_params &p);
int split_params_normalize(pars3_split_params *prm);
int check_cut(int32_t T, int32_t W);
void set_layout_params(pars3_handle *h, const pars3_split_params &p);
// layout-build decisions shared by the host and GPU builders (host_split.cpp)
struct PieceRef {
    int32_t l, e0, len;   // long row, first entry in the concatenated long-row list, length
};
void half_tiles(pars3_handle *h, int64_t mcap, std::vector<int32_t> &tcount);
void long_rows(pars3_handle *h, const std::vector<int32_t> &flen, int64_t ftotal, int64_t cap_in,
               std::vector<uint8_t> &is_long);
int slice_rows(pars3_handle *h, const std::vector<int32_t> &rows, const std::vector<int32_t> &slen,
               std::vector<int32_t> &row_base);
int long_pieces(pars3_handle *h, const std::vector<uint8_t> &is_long, const std::vector<int32_t> &flen,
                std::vector<PieceRef> &pieces);
void fold_items(pars3_handle *h);
int max_smem_all(const pars3_handle *h);
// device_split.cu: the reordered matrix on the device (the cut-independent
// split stages), re-cut on the GPU for any cut (pars3_split_device, the autotuner)
struct DevBase;
int devbase_create(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val, const int32_t *perm,
                   int symmetric, DevBase **out, void *stream);
int devbase_cut(DevBase *b, const pars3_split_params &p, pars3_handle **out, void *stream);
int64_t devbase_bandwidth(const DevBase *b);
void devbase_free(DevBase *b);
int64_t half_room(const pars3_handle *h);
// bit of the calling thread's current CUDA device (kernel attributes are set
// once per device and kernel)
uint64_t device_bit();
// PARS3_OK when h is uploaded and its device is the current one, else PARS3_ESTATE
int ready_on_device(const pars3_handle *h);
void auto_cut(int64_t bw, int32_t w_min, int32_t w_cap, int32_t t_min, int32_t *T, int32_t *W);
int build_layout(pars3_handle *h);
int smem_bytes_for(const pars3_handle *h, int dtype);
int spmv_smem_bytes(const pars3_handle *h, int dtype);

int sm_count();
void dtype_sizes(int dtype, uint32_t *vsz, uint32_t *xsz, uint32_t *asz);
int64_t model_bytes(const pars3_handle *h, int dtype);
uint16_t f32_to_bf16_rne(float f);

// capi.cpp
int cuda_status(int cuda_err);

// spmv.cu
int launch_spmv(const pars3_handle *h, int dtype, double alpha, int k, const void *x, void *y,
                void *stream);
int launch_spmv_scratch(const pars3_handle *h, int dtype, double alpha, const void *x, void *y, void *halo,
                        void *lpart, void *stream);
int launch_permute(const pars3_handle *h, int dtype, int k, const void *src, void *dst, bool inverse,
                   void *stream);
// spmm.cu
int launch_spmm(const pars3_handle *h, int dtype, double alpha, int k, const void *X, void *Y, void *halo,
                void *lpart, void *stream);
int ensure_scratch(pars3_handle *h, int k);
int spmm_smem_bytes(const pars3_handle *h, int dtype);

}  // namespace pars3
