// spmm.cu -- Y = (alpha I + S) X for k right-hand sides (X, Y row-major,
// 1 <= k <= 32) on the split layout of the skew product.
//
// Same decomposition as the single product (blocks of long-row pieces, then
// one block per row tile, then a fold); the device code is in
// spmm_device.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "spmm_device.cuh"

namespace pars3 {

template <typename VT, typename XT, typename AT, int LPR, int NV>
__global__ void __launch_bounds__(kBlock, 2) spmm_kernel(const SpmvArgs<VT, XT, AT> a, int k) {
    extern __shared__ __align__(128) unsigned char smem[];
    if (static_cast<int>(blockIdx.x) < a.nlb) spmm_long<VT, XT, AT, LPR, NV>(a, k, blockIdx.x);
    else spmm_tile<VT, XT, AT, LPR, NV>(a, k, blockIdx.x - a.nlb, smem);
}

// y[row, c] += halo sum + long-row piece sums (in the row's order), one
// thread per (receiving row, column)
template <typename XT, typename AT>
__global__ void __launch_bounds__(256) fold_spmm_kernel(int nitems, int k, const FoldLists F,
                                                        const AT *__restrict__ halo, const AT *__restrict__ lpart,
                                                        XT *__restrict__ y) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t w = gw; w < static_cast<int64_t>(F.nheavy) * k; w += nw) {   // heavy (row, column), a warp each
        const int f = __ldg(F.heavy + w / k), c = static_cast<int>(w % k);
        const AT s = heavy_pieces_warp<AT>(__ldg(F.p0 + f), __ldg(F.np + f), lpart, k, c);
        if (lane == 0) {
            const int64_t r = __ldg(F.row + f);
            const int hi = __ldg(F.halo + f), rem = __ldg(F.rem + f);
            AT v = static_cast<AT>(y[r * k + c]);
            if (hi >= 0) v += halo[static_cast<int64_t>(hi) * k + c];
            v += s;
            if (rem >= 0) v += lpart[static_cast<int64_t>(rem) * k + c];
            y[r * k + c] = static_cast<XT>(v);
        }
    }
    const int64_t total = static_cast<int64_t>(nitems) * k;
    for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < total;
         q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int f = static_cast<int>(q / k), c = static_cast<int>(q - static_cast<int64_t>(f) * k);
        const int np = __ldg(F.np + f);
        if (np >= kFoldHeavy) continue;
        const int64_t r = __ldg(F.row + f);
        const int hi = __ldg(F.halo + f);
        AT v = static_cast<AT>(y[r * k + c]);
        if (hi >= 0) v += halo[static_cast<int64_t>(hi) * k + c];
        v = long_row_sum<AT>(__ldg(F.p0 + f), np, __ldg(F.rem + f), lpart, k, c, v);
        y[r * k + c] = static_cast<XT>(v);
    }
}

// ------------------------------------------------------------------ host

int spmm_smem_bytes(const pars3_handle *h, int dtype) {
    uint32_t vsz, xsz, asz;
    dtype_sizes(dtype, &vsz, &xsz, &asz);
    return static_cast<int>(
        spmm_layout(h->T, h->W, static_cast<uint32_t>(round_up(h->L.max_tile_half, kAlignHalf)), vsz).total);
}

template <typename VT, typename XT, typename AT, int LPR, int NV>
static int launch_spmm_lpr(const pars3_handle *h, int dtype, double alpha, int k, const void *X, void *Y,
                           void *halo, void *lpart, cudaStream_t st) {
    const Layout &L = h->L;
    const DevLayout &D = h->D;
    SpmvArgs<VT, XT, AT> a = make_spmv_args<VT, XT, AT>(h, dtype);
    a.halo = static_cast<AT *>(halo);
    a.lpart = static_cast<AT *>(lpart);
    a.x = static_cast<const XT *>(X);
    a.y = static_cast<XT *>(Y);
    a.alpha = static_cast<AT>(alpha);
    const int smem = spmm_smem_bytes(h, dtype);
    static std::atomic<uint64_t> configured{0};   // one bit per device
    const uint64_t dbit = device_bit();
    if (!(configured.load() & dbit)) {
        cudaError_t e = cudaFuncSetAttribute(spmm_kernel<VT, XT, AT, LPR, NV>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
        if (e != cudaSuccess) return cuda_status(e);
        configured.fetch_or(dbit);
    }
    const int grid = a.nlb + h->ntiles;
    if (grid > 0) spmm_kernel<VT, XT, AT, LPR, NV><<<grid, kBlock, smem, st>>>(a, k);
    const int nf = static_cast<int>(L.fold_row.size());
    if (nf > 0) {
        const int64_t total = static_cast<int64_t>(nf) * k;
        const int blocks = static_cast<int>(std::min<int64_t>((total + 255) / 256, 8LL * sm_count()));
        fold_spmm_kernel<XT, AT><<<blocks, 256, 0, st>>>(nf, k, fold_lists(D, L), static_cast<const AT *>(halo),
                                                         static_cast<const AT *>(lpart), static_cast<XT *>(Y));
    }
    return cuda_status(cudaGetLastError());
}

template <typename VT, typename XT, typename AT, int NV>
static int launch_spmm_nv(const pars3_handle *h, int dtype, double alpha, int k, const void *X, void *Y,
                          void *halo, void *lpart, cudaStream_t st) {
    switch (spmm_lpr(k, NV)) {
        case 1: return launch_spmm_lpr<VT, XT, AT, 1, NV>(h, dtype, alpha, k, X, Y, halo, lpart, st);
        case 2: return launch_spmm_lpr<VT, XT, AT, 2, NV>(h, dtype, alpha, k, X, Y, halo, lpart, st);
        case 4: return launch_spmm_lpr<VT, XT, AT, 4, NV>(h, dtype, alpha, k, X, Y, halo, lpart, st);
        case 8:
            if constexpr (NV <= 4) return launch_spmm_lpr<VT, XT, AT, 8, NV>(h, dtype, alpha, k, X, Y, halo, lpart, st);
            return PARS3_EINVAL;
        case 16:
            if constexpr (NV <= 2) return launch_spmm_lpr<VT, XT, AT, 16, NV>(h, dtype, alpha, k, X, Y, halo, lpart, st);
            return PARS3_EINVAL;
        case 32:
            if constexpr (NV == 1) return launch_spmm_lpr<VT, XT, AT, 32, NV>(h, dtype, alpha, k, X, Y, halo, lpart, st);
            return PARS3_EINVAL;
        default: return PARS3_EINVAL;
    }
}

// 32- or 16-byte lanes (spmm_nv) when X and Y are 16-byte aligned
template <typename VT, typename XT, typename AT>
static int launch_spmm_typed(const pars3_handle *h, int dtype, double alpha, int k, const void *X, void *Y,
                             void *halo, void *lpart, cudaStream_t st) {
    const bool aligned = ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) & 15u) == 0;
    constexpr int V = 16 / static_cast<int>(sizeof(XT));
    const int nv = spmm_lane_elems<XT>(k, h->lane_bytes, aligned);
    if (nv == 2 * V) return launch_spmm_nv<VT, XT, AT, 2 * V>(h, dtype, alpha, k, X, Y, halo, lpart, st);
    if (nv == V) return launch_spmm_nv<VT, XT, AT, V>(h, dtype, alpha, k, X, Y, halo, lpart, st);
    return launch_spmm_nv<VT, XT, AT, 1>(h, dtype, alpha, k, X, Y, halo, lpart, st);
}

int launch_spmm(const pars3_handle *h, int dtype, double alpha, int k, const void *X, void *Y, void *halo,
                void *lpart, void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (dtype) {
        case PARS3_F64: return launch_spmm_typed<double, double, double>(h, dtype, alpha, k, X, Y, halo, lpart, st);
        case PARS3_F32: return launch_spmm_typed<float, float, float>(h, dtype, alpha, k, X, Y, halo, lpart, st);
        case PARS3_BF16: return launch_spmm_typed<uint16_t, float, float>(h, dtype, alpha, k, X, Y, halo, lpart, st);
        default: return PARS3_EINVAL;
    }
}

// Scratch for k right-hand sides: grown (and kept) on the first call that
// needs more than the handle holds.
int ensure_scratch(pars3_handle *h, int k) {
    DevLayout &D = h->D;
    if (D.scratch_k >= k) return PARS3_OK;
    void *halo = nullptr, *lpart = nullptr;
    cudaError_t e = cudaMalloc(&halo, std::max<size_t>(16, h->L.hhrow.size() * 8ull * k));
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaMalloc(&lpart, std::max<size_t>(16, static_cast<size_t>(h->L.nslots) * 8ull * k));
    if (e != cudaSuccess) {
        cudaFree(halo);
        return cuda_status(e);
    }
    D.owned.push_back(halo);
    D.owned.push_back(lpart);
    D.halo = halo;
    D.lpart = lpart;
    D.scratch_k = k;
    return PARS3_OK;
}

}  // namespace pars3

using namespace pars3;

extern "C" int pars3_spmm(const pars3_handle *hc, int32_t dtype, double alpha, int32_t k, const void *X, void *Y,
                          void *stream) {
    pars3_handle *h = const_cast<pars3_handle *>(hc);
    if (!h || k < 1 || k > 32) return PARS3_EINVAL;
    if (dtype < 0 || dtype >= kNumDtypes) return PARS3_EINVAL;
    if (!(h->dtypes & PARS3_DTYPE_BIT(dtype))) return PARS3_EUNSUPPORTED;
    if (ready_on_device(h) != PARS3_OK) return PARS3_ESTATE;
    if (h->n == 0) return PARS3_OK;
    if (!X || !Y || X == Y) return PARS3_EINVAL;
    if (k == 1) return pars3_spmv(h, dtype, alpha, X, Y, stream);
    int rc = ensure_scratch(h, k);
    if (rc != PARS3_OK) return rc;
    if (spmm_smem_bytes(h, dtype) > kSmemLimit) return PARS3_EUNSUPPORTED;
    return launch_spmm(h, dtype, alpha, k, X, Y, h->D.halo, h->D.lpart, stream);
}
