// spmv.cu -- host launchers of the skew product y = (alpha I + S) x (the
// tile and fold kernels of spmv_kernels.cuh) and of the permutation kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "spmv_kernels.cuh"

namespace pars3 {

// ------------------------------------------------------------ host side

// SM count of the current device, cached per device
int sm_count() {
    constexpr int kMaxDev = 64;
    static std::atomic<int> cached[kMaxDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev < 0 || dev >= kMaxDev) {
        int v = 0;
        return cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0 ? v : 1;
    }
    int v = cached[dev].load();
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 1;
    cached[dev].store(v);
    return v;
}

template <typename VT, typename XT, typename AT>
static int launch_typed(const pars3_handle *h, int dtype, double alpha, const void *x, void *y, void *halo,
                        void *lpart, cudaStream_t st) {
    const Layout &L = h->L;
    const DevLayout &D = h->D;
    SpmvArgs<VT, XT, AT> a = make_spmv_args<VT, XT, AT>(h, dtype);
    a.halo = static_cast<AT *>(halo);
    a.lpart = static_cast<AT *>(lpart);
    a.x = static_cast<const XT *>(x);
    a.y = static_cast<XT *>(y);
    a.alpha = static_cast<AT>(alpha);
    const int smem = spmv_smem_bytes(h, dtype);
    static std::atomic<uint64_t> configured{0};   // one bit per device
    const uint64_t dbit = device_bit();
    if (!(configured.load() & dbit)) {
        cudaError_t e = cudaFuncSetAttribute(tile_kernel<VT, XT, AT, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
        if constexpr (sizeof(AT) == 4) {
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(tile_kernel<VT, XT, AT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSmemLimit);
        }
        if (e != cudaSuccess) return cuda_status(e);
        configured.fetch_or(dbit);
    }
    const int grid = a.nlb + h->ntiles;
    // fp32 / bf16 look-ahead variant: direct stores, nothing staged unless
    // the tile has middle entries
    const bool la = sizeof(AT) == 4 && h->variant == PARS3_VARIANT_LOOKAHEAD;
    const int smem_la = L.max_tile_half > 0 ? smem : 0;
    if (grid > 0) {
        if constexpr (sizeof(AT) == 4) {
            if (la) tile_kernel<VT, XT, AT, true><<<grid, kBlock, smem_la, st>>>(a);
            else tile_kernel<VT, XT, AT, false><<<grid, kBlock, smem, st>>>(a);
        } else {
            tile_kernel<VT, XT, AT, false><<<grid, kBlock, smem, st>>>(a);
        }
    }
    const int nf = static_cast<int>(L.fold_row.size());
    if (nf > 0) {
        const int blocks = static_cast<int>(std::min<int64_t>((nf + 255) / 256, 8LL * sm_count()));
        // a programmatic dependent launch: the fold's blocks are scheduled
        // during the tile kernel's tail and wait for its results on the device
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(blocks);
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const cudaError_t e = cudaLaunchKernelEx(&cfg, fold_kernel<XT, AT>, nf, fold_lists(D, L),
                                                 static_cast<const AT *>(halo), static_cast<const AT *>(lpart),
                                                 static_cast<XT *>(y));
        if (e != cudaSuccess) return cuda_status(e);
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
    const int blocks = static_cast<int>(std::min<int64_t>((total + 255) / 256, 16LL * sm_count()));
    if (dtype == PARS3_F64)
        permute_kernel<double><<<blocks, 256, 0, st>>>(h->n, k, h->D.perm, static_cast<const double *>(src),
                                                       static_cast<double *>(dst), inverse);
    else
        permute_kernel<float><<<blocks, 256, 0, st>>>(h->n, k, h->D.perm, static_cast<const float *>(src),
                                                      static_cast<float *>(dst), inverse);
    return cuda_status(cudaGetLastError());
}

}  // namespace pars3
