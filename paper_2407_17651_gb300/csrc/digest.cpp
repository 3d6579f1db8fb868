// digest.cpp -- pars3_layout_digest: a 64-bit FNV-1a digest of everything a
// handle's device layout holds (every array of the layout, with its length,
// and the scalars the kernels read), so that two handles can be checked to
// hold the same layout, e.g. one built by pars3_split and one by
// pars3_split_device.  The paper has no counterpart.
#include <cstdint>
#include <cstring>
#include <vector>

#include "internal.h"

namespace pars3 {
namespace {

struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void bytes(const void *p, size_t n) {
        const unsigned char *c = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; ++i) {
            h ^= c[i];
            h *= 1099511628211ull;
        }
    }
    template <typename T>
    void vec(const std::vector<T> &v) {
        const uint64_t n = v.size();
        bytes(&n, sizeof(n));
        if (n) bytes(v.data(), n * sizeof(T));
    }
    template <typename T>
    void val(T v) {
        bytes(&v, sizeof(v));
    }
};

}  // namespace
}  // namespace pars3

extern "C" int pars3_layout_digest(const pars3_handle *h, uint64_t *digest) {
    if (!h || !digest) return PARS3_EINVAL;
    const pars3::Layout &L = h->L;
    pars3::Fnv f;
    f.val(h->n);
    f.val(h->T);
    f.val(h->W);
    f.val(h->ntiles);
    f.val(h->dtypes);
    f.val(h->symmetric);
    f.vec(L.hoff);
    f.vec(L.hcnt);
    f.vec(L.hrp);
    f.vec(L.hcol);
    f.vec(L.hcperm);
    f.vec(L.hrowc);
    f.vec(L.hcsoff);
    f.vec(L.hcsn);
    f.vec(L.hcs);
    f.vec(L.hhoff);
    f.vec(L.hhrow);
    f.vec(L.sl_off);
    f.vec(L.sl_ent);
    f.vec(L.sl_meta);
    f.vec(L.fcol);
    f.vec(L.sl_e);
    f.vec(L.lrow);
    f.vec(L.lrp);
    f.vec(L.lp0);
    f.vec(L.lrem);
    f.vec(L.ls_ent);
    f.vec(L.ls_len);
    f.vec(L.lcol);
    f.val(L.piece_len);
    f.val(L.ls_per_block);
    f.vec(L.fold_row);
    f.vec(L.fold_halo);
    f.vec(L.fold_p0);
    f.vec(L.fold_np);
    f.vec(L.fold_rem);
    f.vec(L.fold_heavy);
    f.vec(L.hval64);
    f.vec(L.fval64);
    f.vec(L.lval64);
    f.vec(L.hval32);
    f.vec(L.fval32);
    f.vec(L.lval32);
    f.vec(L.hval16);
    f.vec(L.fval16);
    f.vec(L.lval16);
    f.val(L.max_tile_half);
    f.val(L.max_tile_cs);
    f.val(L.max_tile_full);
    f.val(L.max_tile_slices);
    f.val(L.cap_full);
    f.val(L.nslots);
    *digest = f.h;
    return PARS3_OK;
}
