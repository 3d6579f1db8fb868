// spmv.cu -- host launchers of the skew product y = (alpha I + S) x (the
// tile and fold kernels of spmv_kernels.cuh) and of the permutation kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "spmv_kernels.cuh"

namespace pars3 {

// ------------------------------------------------------------ host side

int sm_count() {
    static std::atomic<int> cached{0};
    int v = cached.load();
    if (v > 0) return v;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
    cached.store(v);
    return v;
}

template <typename VT, typename XT, typename AT>
static int launch_typed(const pars3_handle *h, int dtype, double alpha, const void *x, void *y, void *halo,
                        void *lpart, cudaStream_t st) {
    const Layout &L = h->L;
    const DevLayout &D = h->D;
    SpmvArgs<VT, XT, AT> a;
    a.n = h->n;
    a.T = h->T;
    a.W = h->W;
    a.ntiles = h->ntiles;
    a.nchunks = static_cast<int32_t>(L.lcbeg.size());
    a.Mh = static_cast<int32_t>(round_up(L.max_tile_half, kAlignHalf));
    a.hoff = D.hoff;
    a.hcnt = D.hcnt;
    a.hrp = D.hrp;
    a.hcol = D.hcol;
    a.hcperm = D.hcperm;
    a.hval = static_cast<const VT *>(D.hval[dtype]);
    a.hhoff = D.hhoff;
    a.hhrow = D.hhrow;
    a.halo = static_cast<AT *>(halo);
    a.sl_off = D.sl_off;
    a.sl_ent = D.sl_ent;
    a.sl_meta = D.sl_meta;
    a.fcol = D.fcol;
    a.fval = static_cast<const VT *>(D.fval[dtype]);
    a.lrp = D.lrp;
    a.lcbeg = D.lcbeg;
    a.lcend = D.lcend;
    a.lcfirst = D.lcfirst;
    a.lcrows = D.lcrows;
    a.lcslot = D.lcslot;
    a.lcol = D.lcol;
    a.lval = static_cast<const VT *>(D.lval[dtype]);
    a.lpart = static_cast<AT *>(lpart);
    a.x = static_cast<const XT *>(x);
    a.y = static_cast<XT *>(y);
    a.alpha = static_cast<AT>(alpha);
    a.err = D.err;
    a.sym = h->symmetric;
    const int smem = smem_bytes_for(h, dtype);
    static std::atomic<uint64_t> configured{0};   // one bit per device
    const uint64_t dbit = device_bit();
    if (!(configured.load() & dbit)) {
        cudaError_t e = cudaFuncSetAttribute(tile_kernel<VT, XT, AT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kSmemLimit);
        if (e != cudaSuccess) return cuda_status(e);
        configured.fetch_or(dbit);
    }
    const int grid = h->ntiles + a.nchunks;
    if (grid > 0) tile_kernel<VT, XT, AT><<<grid, kBlock, smem, st>>>(a);
    const int nf = static_cast<int>(L.fold_row.size());
    if (nf > 0) {
        const int blocks = static_cast<int>(std::min<int64_t>((nf + 255) / 256, 152 * 8));
        fold_kernel<XT, AT><<<blocks, 256, 0, st>>>(nf, D.fold_row, D.fold_halo, D.fold_long,
                                                    static_cast<const AT *>(halo), D.lc0, D.lc1, D.lcfirst, D.lcslot,
                                                    static_cast<const AT *>(lpart), static_cast<XT *>(y));
    }
    return cuda_status(cudaGetLastError());
}

int launch_spmv_scratch(const pars3_handle *h, int dtype, double alpha, const void *x, void *y, void *halo,
                        void *lpart, void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (dtype) {
        case PARS3_F64: return launch_typed<double, double, double>(h, dtype, alpha, x, y, halo, lpart, st);
        case PARS3_F32: return launch_typed<float, float, float>(h, dtype, alpha, x, y, halo, lpart, st);
        case PARS3_BF16: return launch_typed<uint16_t, float, float>(h, dtype, alpha, x, y, halo, lpart, st);
        default: return PARS3_EINVAL;
    }
}

int launch_spmv(const pars3_handle *h, int dtype, double alpha, int k, const void *x, void *y, void *stream) {
    if (k != 1) return PARS3_EUNSUPPORTED;
    return launch_spmv_scratch(h, dtype, alpha, x, y, h->D.halo, h->D.lpart, stream);
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
