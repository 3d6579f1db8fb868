// batched.cu -- Y_m = (alpha_m I + S_m) X_m for many split handles of uneven
// sizes in ONE persistent launch: a fixed grid of blocks walks the
// concatenated list of work units (every block of long-row pieces and every
// tile of every matrix) in a static round-robin order, followed by one batched fold
// launch.  Per-matrix kernel arguments live in a device table; with
// capture != 0 the pair of launches is recorded once in a CUDA graph and
// replayed while the arguments stay the same.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>
#include <vector>

#include "spmm_device.cuh"

namespace pars3 {

int spmm_smem_bytes(const pars3_handle *h, int dtype);

// upper bound of the batched kernel's static shared memory (its argument
// copy and item index; ptxas reports 384 bytes), kept out of the dynamic
// shared memory it may request
constexpr int kBatchedStaticSmem = 1024;

// work unit u belongs to matrix m with upre[m] <= u < upre[m+1]
__device__ __forceinline__ int unit_matrix(const int32_t *upre, int count, int u) {
    int lo = 0, hi = count;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (upre[mid] <= u) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <typename VT, typename XT, typename AT, int LPR, int NV>
__global__ void __launch_bounds__(kBlock, 2) batched_kernel(const SpmvArgs<VT, XT, AT> *__restrict__ args,
                                                             const int32_t *__restrict__ upre, int count,
                                                             int total, int k) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ SpmvArgs<VT, XT, AT> a;
    __shared__ int item;
    for (int u = blockIdx.x; u < total; u += gridDim.x) {
        // the previous unit's shared-memory accesses finish before the next
        // unit's bulk copies overwrite the same bytes
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            const int m = unit_matrix(upre, count, u);
            a = args[m];
            item = u - upre[m];
        }
        __syncthreads();
        if (k == 1) {
            if (item < a.nlb) {
                long_pieces_block<VT, XT, AT>(a, item, a.x);
            } else {
                EpiSpmv<XT, AT, false> epi{a.alpha, a.y};
                tile_block<VT, XT, AT>(a, item - a.nlb, smem, a.x, epi);
            }
        } else {
            if (item < a.nlb) spmm_long<VT, XT, AT, LPR, NV>(a, k, item);
            else spmm_tile<VT, XT, AT, LPR, NV>(a, k, item - a.nlb, smem);
        }
    }
}

// fold of all matrices: one thread per (receiving row, column)
struct FoldArgs {
    int32_t nf;
    FoldLists F;
};

template <typename XT, typename AT>
__global__ void __launch_bounds__(256) batched_fold_kernel(const FoldArgs *__restrict__ fa,
                                                           const AT *const *__restrict__ halos,
                                                           const AT *const *__restrict__ lparts,
                                                           XT *const *__restrict__ ys, const int64_t *__restrict__ fpre,
                                                           int count, int64_t total, int k,
                                                           const int2 *__restrict__ heavy, int nheavy) {
    // heavy (matrix, row, column) items first, a warp each, as in the
    // single-matrix folds
    const int lane = threadIdx.x & 31;
    const int64_t gw = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t w = gw; w < static_cast<int64_t>(nheavy) * k; w += nw) {
        const int2 mf = heavy[w / k];
        const int c = static_cast<int>(w % k);
        const FoldLists &F = fa[mf.x].F;
        const int f = mf.y;
        const AT s = heavy_pieces_warp<AT>(F.p0[f], F.np[f], lparts[mf.x], k, c);
        if (lane == 0) {
            const int64_t r = F.row[f];
            XT *y = ys[mf.x];
            AT v = static_cast<AT>(y[r * k + c]);
            const int hh = F.halo[f];
            if (hh >= 0) v += halos[mf.x][static_cast<int64_t>(hh) * k + c];
            v += s;
            const int rem = F.rem[f];
            if (rem >= 0) v += lparts[mf.x][static_cast<int64_t>(rem) * k + c];
            y[r * k + c] = static_cast<XT>(v);
        }
    }
    for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < total;
         q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        int lo = 0, hi = count;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (fpre[mid] <= q) lo = mid;
            else hi = mid;
        }
        const int m = lo;
        const int64_t local = q - fpre[m];
        const int f = static_cast<int>(local / k), c = static_cast<int>(local - static_cast<int64_t>(f) * k);
        const FoldArgs F = fa[m];
        if (F.F.np[f] >= kFoldHeavy) continue;
        const int64_t r = F.F.row[f];
        XT *y = ys[m];
        AT v = static_cast<AT>(y[r * k + c]);
        const int hh = F.F.halo[f];
        if (hh >= 0) v += halos[m][static_cast<int64_t>(hh) * k + c];
        v = long_row_sum<AT>(F.F.p0[f], F.F.np[f], F.F.rem[f], lparts[m], k, c, v);
        y[r * k + c] = static_cast<XT>(v);
    }
}

// ------------------------------------------------------------------ host

struct BatchCache {
    std::vector<uint64_t> serial;   // handle serials: a freed handle never matches again
    std::vector<double> alpha;
    std::vector<const void *> X;
    std::vector<void *> Y;
    int dtype = -1, k = 0;
    void *args = nullptr, *upre = nullptr, *fa = nullptr, *halos = nullptr, *lparts = nullptr, *ys = nullptr,
         *fpre = nullptr, *heavy = nullptr;
    int nheavy = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t capture = nullptr;
    void release() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (void *p : {args, upre, fa, halos, lparts, ys, fpre, heavy})
            if (p) cudaFree(p);
        if (capture) cudaStreamDestroy(capture);
        *this = BatchCache();
    }
};

template <typename VT, typename XT, typename AT>
static SpmvArgs<VT, XT, AT> make_args(const pars3_handle *h, int dtype, double alpha, const void *X, void *Y) {
    SpmvArgs<VT, XT, AT> a = make_spmv_args<VT, XT, AT>(h, dtype);
    a.x = static_cast<const XT *>(X);
    a.y = static_cast<XT *>(Y);
    a.alpha = static_cast<AT>(alpha);
    return a;
}

template <typename T>
static int upload_vec(void **dst, const std::vector<T> &v) {
    cudaError_t e = cudaMalloc(dst, std::max<size_t>(16, v.size() * sizeof(T)));
    if (e == cudaSuccess && !v.empty()) e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    return cuda_status(e);
}

template <typename VT, typename XT, typename AT, int LPR, int NV>
static int enqueue(BatchCache &C, int count, int64_t total_units, int64_t total_fold, int smem, int k,
                   cudaStream_t st) {
    static std::atomic<uint64_t> configured{0};   // one bit per device
    const uint64_t dbit = device_bit();
    if (!(configured.load() & dbit)) {
        cudaError_t e = cudaFuncSetAttribute(batched_kernel<VT, XT, AT, LPR, NV>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kSmemLimit - kBatchedStaticSmem);
        if (e != cudaSuccess) return cuda_status(e);
        configured.fetch_or(dbit);
    }
    // Smaller blocks, more of them per SM: a unit (one tile or one block of
    // long-row slices) is short and mostly waits on memory, so more units in
    // flight pay (the kernel's 64 registers a thread fit 1,024 threads an SM
    // however they are split).  Measured on the 64-matrix set against
    // 512-thread blocks, two per SM: 256-thread blocks, four per SM, are
    // faster at every k (fp32 k = 1 / 4 / 32: 362 / 344 / 965 -> 238 / 259 /
    // 873 us); 128-thread blocks, eight per SM, are faster still for fp32 /
    // bf16 up to k = 16 (k = 1: 198 us) and fp64 from k = 4, and slower for
    // fp32 at k = 32 and fp64 at k = 1, where the 256-thread blocks stay.
    const bool quarter = sizeof(AT) == 4 ? k <= 16 : k >= 4;
    const int block = quarter ? kBlock / 4 : kBlock / 2;
    const int per_sm = quarter ? 8 : 4;
    const int grid = static_cast<int>(std::min<int64_t>(total_units, static_cast<int64_t>(per_sm) * sm_count()));
    if (grid > 0)
        batched_kernel<VT, XT, AT, LPR, NV><<<grid, block, smem, st>>>(
            static_cast<const SpmvArgs<VT, XT, AT> *>(C.args), static_cast<const int32_t *>(C.upre), count,
            static_cast<int>(total_units), k);
    if (total_fold > 0) {
        const int blocks = static_cast<int>(std::min<int64_t>((total_fold + 255) / 256, 8LL * sm_count()));
        batched_fold_kernel<XT, AT><<<blocks, 256, 0, st>>>(
            static_cast<const FoldArgs *>(C.fa), static_cast<const AT *const *>(C.halos),
            static_cast<const AT *const *>(C.lparts), static_cast<XT *const *>(C.ys),
            static_cast<const int64_t *>(C.fpre), count, total_fold, k, static_cast<const int2 *>(C.heavy),
            C.nheavy);
    }
    return cuda_status(cudaGetLastError());
}

template <typename VT, typename XT, typename AT, int NV>
static int enqueue_lpr(int lpr, BatchCache &C, int count, int64_t nu, int64_t nfold, int smem, int k,
                       cudaStream_t st) {
    switch (lpr) {
        case 1: return enqueue<VT, XT, AT, 1, NV>(C, count, nu, nfold, smem, k, st);
        case 2: return enqueue<VT, XT, AT, 2, NV>(C, count, nu, nfold, smem, k, st);
        case 4: return enqueue<VT, XT, AT, 4, NV>(C, count, nu, nfold, smem, k, st);
        case 8:
            if constexpr (NV <= 4) return enqueue<VT, XT, AT, 8, NV>(C, count, nu, nfold, smem, k, st);
            return PARS3_EINVAL;
        case 16:
            if constexpr (NV <= 2) return enqueue<VT, XT, AT, 16, NV>(C, count, nu, nfold, smem, k, st);
            return PARS3_EINVAL;
        case 32:
            if constexpr (NV == 1) return enqueue<VT, XT, AT, 32, NV>(C, count, nu, nfold, smem, k, st);
            return PARS3_EINVAL;
        default: return PARS3_EINVAL;
    }
}

template <typename VT, typename XT, typename AT>
static int run_batched(BatchCache &C, pars3_handle *const *hs, int count, int dtype, const double *alpha, int k,
                       const void *const *X, void *const *Y, bool capture, cudaStream_t st) {
    bool same = C.dtype == dtype && C.k == k && static_cast<int>(C.serial.size()) == count;
    for (int m = 0; same && m < count; ++m) same = C.serial[m] == hs[m]->serial;
    same = same && std::equal(C.alpha.begin(), C.alpha.end(), alpha) &&
                      std::equal(C.X.begin(), C.X.end(), X) && std::equal(C.Y.begin(), C.Y.end(), Y);
    std::vector<int32_t> upre(1, 0);
    std::vector<int64_t> fpre(1, 0);
    int smem = 0;
    for (int m = 0; m < count; ++m) {
        const pars3_handle *h = hs[m];
        upre.push_back(upre.back() + h->L.nlong_blocks() + h->ntiles);
        fpre.push_back(fpre.back() + static_cast<int64_t>(h->L.fold_row.size()) * k);
        smem = std::max(smem, k == 1 ? smem_bytes_for(h, dtype) : spmm_smem_bytes(h, dtype));
    }
    if (smem + kBatchedStaticSmem > kSmemLimit) return PARS3_EUNSUPPORTED;
    if (!same) {
        C.release();
        std::vector<SpmvArgs<VT, XT, AT>> args;
        std::vector<FoldArgs> fa;
        std::vector<int2> heavy;
        std::vector<const void *> halos, lparts;
        std::vector<void *> ys;
        for (int m = 0; m < count; ++m) {
            const pars3_handle *h = hs[m];
            args.push_back(make_args<VT, XT, AT>(h, dtype, alpha[m], X[m], Y[m]));
            const DevLayout &D = h->D;
            fa.push_back(FoldArgs{static_cast<int32_t>(h->L.fold_row.size()), fold_lists(D, h->L)});
            for (int32_t f : h->L.fold_heavy) heavy.push_back(make_int2(m, f));
            halos.push_back(D.halo);
            lparts.push_back(D.lpart);
            ys.push_back(Y[m]);
        }
        int rc;
        if ((rc = upload_vec(&C.args, args)) != PARS3_OK) return rc;
        if ((rc = upload_vec(&C.upre, upre)) != PARS3_OK) return rc;
        if ((rc = upload_vec(&C.fa, fa)) != PARS3_OK) return rc;
        if ((rc = upload_vec(&C.halos, halos)) != PARS3_OK) return rc;
        if ((rc = upload_vec(&C.lparts, lparts)) != PARS3_OK) return rc;
        if ((rc = upload_vec(&C.ys, ys)) != PARS3_OK) return rc;
        if ((rc = upload_vec(&C.fpre, fpre)) != PARS3_OK) return rc;
        if ((rc = upload_vec(&C.heavy, heavy)) != PARS3_OK) return rc;
        C.nheavy = static_cast<int>(heavy.size());
        for (int m = 0; m < count; ++m) C.serial.push_back(hs[m]->serial);
        C.alpha.assign(alpha, alpha + count);
        C.X.assign(X, X + count);
        C.Y.assign(Y, Y + count);
        C.dtype = dtype;
        C.k = k;
    }
    // 32- or 16-byte lanes (spmm_nv) when every X and Y is 16-byte aligned
    constexpr int V = 16 / static_cast<int>(sizeof(XT));
    bool aligned = true;
    for (int m = 0; m < count; ++m)
        aligned = aligned && ((reinterpret_cast<uintptr_t>(X[m]) | reinterpret_cast<uintptr_t>(Y[m])) & 15u) == 0;
    // one lane width serves every matrix: a tuned width when all handles carry
    // the same one, else the rule
    int lane_bytes = hs[0]->lane_bytes;
    for (int m = 1; m < count; ++m)
        if (hs[m]->lane_bytes != lane_bytes) lane_bytes = 0;
    const int nv = spmm_lane_elems<XT>(k, lane_bytes, aligned);
    const int lpr = spmm_lpr(k, nv);
    const int64_t nu = upre.back(), nfold = fpre.back();
    auto launch = [&](cudaStream_t s) {
        if (nv == 2 * V) return enqueue_lpr<VT, XT, AT, 2 * V>(lpr, C, count, nu, nfold, smem, k, s);
        if (nv == V) return enqueue_lpr<VT, XT, AT, V>(lpr, C, count, nu, nfold, smem, k, s);
        return enqueue_lpr<VT, XT, AT, 1>(lpr, C, count, nu, nfold, smem, k, s);
    };
    if (!capture) return launch(st);
    if (!C.exec) {
        cudaError_t e = cudaStreamCreateWithFlags(&C.capture, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(C.capture, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) return cuda_status(e);
        const int rc = launch(C.capture);
        e = cudaStreamEndCapture(C.capture, &C.graph);
        if (rc != PARS3_OK) return rc;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&C.exec, C.graph, 0);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return cuda_status(cudaGraphLaunch(C.exec, st));
}

}  // namespace pars3

using namespace pars3;

void pars3_release_batch(pars3_handle *h) {
    if (h && h->batch_cache) {
        BatchCache *C = static_cast<BatchCache *>(h->batch_cache);
        C->release();
        delete C;
        h->batch_cache = nullptr;
    }
}

extern "C" int pars3_spmm_batched(pars3_handle *const *hs, int32_t count, int32_t dtype, const double *alpha,
                                  int32_t k, const void *const *X, void *const *Y, int32_t capture, void *stream) {
    if (!hs || !alpha || !X || !Y || count < 1 || k < 1 || k > 32) return PARS3_EINVAL;
    if (dtype < 0 || dtype >= kNumDtypes) return PARS3_EINVAL;
    for (int m = 0; m < count; ++m) {
        pars3_handle *h = hs[m];
        if (!h) return PARS3_EINVAL;
        if (!(h->dtypes & PARS3_DTYPE_BIT(dtype))) return PARS3_EUNSUPPORTED;
        if (ready_on_device(h) != PARS3_OK) return PARS3_ESTATE;
        if (h->n > 0 && (!X[m] || !Y[m] || X[m] == Y[m])) return PARS3_EINVAL;
        if (k == 1 && ((reinterpret_cast<uintptr_t>(X[m]) | reinterpret_cast<uintptr_t>(Y[m])) & 15u))
            return PARS3_EINVAL;
        const int rc = ensure_scratch(h, k);
        if (rc != PARS3_OK) return rc;
    }
    pars3_handle *owner = hs[0];
    if (!owner->batch_cache) owner->batch_cache = new (std::nothrow) BatchCache();
    if (!owner->batch_cache) return PARS3_ENOMEM;
    BatchCache &C = *static_cast<BatchCache *>(owner->batch_cache);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (dtype) {
        case PARS3_F64: return run_batched<double, double, double>(C, hs, count, dtype, alpha, k, X, Y, capture != 0, st);
        case PARS3_F32: return run_batched<float, float, float>(C, hs, count, dtype, alpha, k, X, Y, capture != 0, st);
        case PARS3_BF16:
            return run_batched<uint16_t, float, float>(C, hs, count, dtype, alpha, k, X, Y, capture != 0, st);
        default: return PARS3_EINVAL;
    }
}
