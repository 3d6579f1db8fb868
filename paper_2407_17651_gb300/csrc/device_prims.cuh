// device_prims.cuh -- device building blocks of the GPU preprocessing
// (device_reorder.cu, device_split.cu): single-block prefix sums over sizes
// that live in device memory, a stable LSD radix sort of 32-bit keys with
// 32-bit values, the strict-lower pattern check, small element-wise kernels
// and the host helpers that drive them.  Each translation unit that
// includes this header gets its own copies (internal linkage).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <vector>

#include "internal.h"

namespace pars3 {
namespace {

constexpr int kThreads = 256;                       // block size of the element-wise kernels
constexpr int kSortItems = 16;                      // keys per thread in a sort tile
constexpr int kSortTile = kThreads * kSortItems;    // 4096 keys per tile
constexpr int kSortWarps = kThreads / 32;
constexpr int kSortWarpKeys = kSortTile / kSortWarps;   // 512 consecutive keys per warp
constexpr int kScanThreads = 1024;                  // single-block prefix sums
constexpr int kScanItems = 8;
constexpr int kErrPattern = 1;                      // error bit of validate_kernel: not a strict lower pattern

__device__ __forceinline__ int lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return static_cast<int>(m);
}

// ------------------------------------------------------------ prefix sums

// Exclusive prefix of one value per thread across a block of kScanThreads
// threads; *total receives the block sum.  ws holds 32 partial sums.
template <typename T>
__device__ T block_excl_scan(T v, T *ws, T *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T t = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += t;
    }
    if (lane == 31) ws[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < (kScanThreads >> 5) ? ws[lane] : T(0);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const T t = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += t;
        }
        ws[lane] = w;   // inclusive sums of the warp totals
    }
    __syncthreads();
    const T before = (warp > 0 ? ws[warp - 1] : T(0)) + inc - v;
    *total = ws[31];
    __syncthreads();   // ws is reused by the next call
    return before;
}

// out[0..len) = exclusive prefix sums of in[0..len), out[len] = the total.
// Called by all kScanThreads threads of one block.
__device__ void block_scan_array(const int32_t *in, int32_t *out, int len, int *ws) {
    int carry = 0;
    for (int base = 0; base < len; base += kScanThreads * kScanItems) {
        const int i0 = base + threadIdx.x * kScanItems;
        int v[kScanItems];
        int s = 0;
#pragma unroll
        for (int t = 0; t < kScanItems; ++t) {
            v[t] = i0 + t < len ? in[i0 + t] : 0;
            s += v[t];
        }
        int total;
        int run = carry + block_excl_scan<int>(s, ws, &total);
#pragma unroll
        for (int t = 0; t < kScanItems; ++t) {
            if (i0 + t < len) out[i0 + t] = run;
            run += v[t];
        }
        carry += total;
    }
    if (threadIdx.x == 0) out[len] = carry;
}

// One chunk of kScanThreads * kScanItems values: out[base ..] = carry +
// exclusive prefix sums of in[base ..], up to len; returns the chunk's sum.
__device__ int block_scan_chunk(const int32_t *in, int32_t *out, int base, int len, int carry, int *ws) {
    const int i0 = base + threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int t = 0; t < kScanItems; ++t) {
        v[t] = i0 + t < len ? in[i0 + t] : 0;
        s += v[t];
    }
    int total;
    int run = carry + block_excl_scan<int>(s, ws, &total);
#pragma unroll
    for (int t = 0; t < kScanItems; ++t) {
        if (i0 + t < len) out[i0 + t] = run;
        run += v[t];
    }
    return total;
}

constexpr int kScanChunk = kScanThreads * kScanItems;   // values per block of the multi-block scan

// multi-block scan, pass 1: bsum[b] = sum of chunk b
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const int32_t *__restrict__ in, int len,
                                                                   int32_t *__restrict__ bsum) {
    __shared__ int ws[32];
    const int i0 = blockIdx.x * kScanChunk + threadIdx.x * kScanItems;
    int s = 0;
#pragma unroll
    for (int t = 0; t < kScanItems; ++t) s += i0 + t < len ? in[i0 + t] : 0;
    int total;
    block_excl_scan<int>(s, ws, &total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// multi-block scan, pass 3: every chunk from its offset boff[b]; the last
// block writes the total to out[len]
__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const int32_t *__restrict__ in,
                                                                  int32_t *__restrict__ out, int len,
                                                                  const int32_t *__restrict__ boff) {
    __shared__ int ws[32];
    block_scan_chunk(in, out, blockIdx.x * kScanChunk, len, boff[blockIdx.x], ws);
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[len] = boff[gridDim.x];
}

// Single-block exclusive scan; the length is *len_dev when len_dev is not
// null (a size the host does not know), else len.
__global__ void __launch_bounds__(kScanThreads) scan_kernel(const int32_t *__restrict__ in,
                                                            int32_t *__restrict__ out, const int32_t *len_dev,
                                                            int len) {
    __shared__ int ws[32];
    block_scan_array(in, out, len_dev ? *len_dev : len, ws);
}

// ------------------------------------------------------------ validation

// The pattern may be the block-diagonal union of several matrices: vertex i
// belongs to matrix mid[i] (all to matrix 0 when mid is null), whose
// vertices are [moff[m], moff[m+1]) and entries [eoff[m], eoff[m+1]).
struct Blocks {
    const int32_t *mid;
    const int32_t *moff, *eoff;   // device, count + 1 each
};

// Rows must satisfy eoff[m] <= rowptr[i] <= rowptr[i+1] <= eoff[m+1] (with
// rowptr at the matrix's first row equal to eoff[m]) and hold strictly
// increasing columns in [moff[m], i); entries are read only inside a row
// whose bounds passed.  Also writes the row of every entry and the row
// lengths (the lower part of each degree).
__global__ void validate_kernel(int n, Blocks B, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                int32_t *__restrict__ rowof, int32_t *__restrict__ deg, int *err) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int m = B.mid ? B.mid[i] : 0;
        const int v0 = B.moff[m], e0 = B.eoff[m], e1 = B.eoff[m + 1];
        const int a = rp[i], b = rp[i + 1];
        if ((i == v0 && a != e0) || a < e0 || b < a || b > e1) {
            atomicOr(err, kErrPattern);
            deg[i] = 0;
            continue;
        }
        int prev = v0 - 1;
        bool ok = true;
        for (int k = a; k < b; ++k) {
            const int j = ci[k];
            if (j <= prev || j >= i) ok = false;
            prev = j;
            rowof[k] = i;
        }
        if (!ok) atomicOr(err, kErrPattern);
        deg[i] = b - a;
    }
}


// ------------------------------------------------------------ radix sort

// hist[d * ntiles + t] = keys of tile t whose digit (key >> shift) & 255 is d
__global__ void __launch_bounds__(kThreads) sort_hist_kernel(const uint32_t *__restrict__ key, int count,
                                                             int shift, int ntiles, int32_t *__restrict__ hist) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int t = blockIdx.x;
    const int base = t * kSortTile;
    for (int i = threadIdx.x; i < kSortTile; i += kThreads)
        if (base + i < count) atomicAdd(&h[(key[base + i] >> shift) & 255], 1);
    __syncthreads();
    hist[threadIdx.x * ntiles + t] = h[threadIdx.x];
}

// Stable scatter of one tile: warp w owns keys [base + 512 w, base + 512 (w+1)),
// taken 32 at a time in order; keys with equal digits are ranked by lane
// within a round and by round within the warp, and warps are ranked by
// index, so equal digits keep their input order.
__global__ void __launch_bounds__(kThreads) sort_scatter_kernel(const uint32_t *__restrict__ key,
                                                                const int32_t *__restrict__ val, int count,
                                                                int shift, int ntiles,
                                                                const int32_t *__restrict__ off,
                                                                uint32_t *__restrict__ key_out,
                                                                int32_t *__restrict__ val_out) {
    __shared__ int cnt[kSortWarps][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = lane; d < 256; d += 32) cnt[warp][d] = 0;
    __syncwarp();
    const int t = blockIdx.x;
    const int base = t * kSortTile + warp * kSortWarpKeys;
    for (int r = 0; r < kSortWarpKeys; r += 32) {
        const int i = base + r + lane;
        const bool ok = i < count;
        const int d = ok ? static_cast<int>((key[i] >> shift) & 255) : 256;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (ok && lane == __ffs(peers) - 1) cnt[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        const int d = threadIdx.x;   // kThreads == 256 digits
        int run = off[d * ntiles + t];
        for (int w = 0; w < kSortWarps; ++w) {
            const int c = cnt[w][d];
            cnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int r = 0; r < kSortWarpKeys; r += 32) {
        const int i = base + r + lane;
        const bool ok = i < count;
        const uint32_t k = ok ? key[i] : 0u;
        const int d = ok ? static_cast<int>((k >> shift) & 255) : 256;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (ok) {
            const int p = cnt[warp][d] + __popc(peers & static_cast<unsigned>(lanemask_lt()));
            key_out[p] = k;
            val_out[p] = val[i];
        }
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1) cnt[warp][d] += __popc(peers);
        __syncwarp();
    }
}

// ------------------------------------------------------------ element-wise

// dst[i] = src[idx[i]]
__global__ void gather_kernel(int n, const int32_t *__restrict__ idx, const int32_t *__restrict__ src,
                              int32_t *__restrict__ dst) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[idx[i]];
}

__global__ void iota_kernel(int n, int32_t *__restrict__ a) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = i;
}

__global__ void fill_kernel(int n, int32_t v, int32_t *__restrict__ a) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = v;
}


// ------------------------------------------------------------ host side

// Device scratch of one call, released on every return path.
class Scratch {
public:
    ~Scratch() {
        for (void *p : ptrs_) cudaFree(p);
    }
    template <typename T>
    T *get(size_t count) {
        void *p = nullptr;
        if (err_ == cudaSuccess) err_ = cudaMalloc(&p, std::max<size_t>(16, count * sizeof(T)));
        if (err_ != cudaSuccess) return nullptr;
        ptrs_.push_back(p);
        return static_cast<T *>(p);
    }
    cudaError_t err() const { return err_; }

private:
    std::vector<void *> ptrs_;
    cudaError_t err_ = cudaSuccess;
};

int grid_for(int64_t items, int per_block) {
    const int64_t g = (items + per_block - 1) / per_block;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g, 8LL * sm_count())));
}

int bits_for(int64_t n) {   // bits needed for the values 0 .. n-1
    int b = 0;
    while (b < 31 && (1LL << b) < n) ++b;
    return b;
}

// Scratch words scan_exclusive needs for arrays of up to len values.
inline size_t scan_ws_size(int64_t len) { return 2 * static_cast<size_t>(len / kScanChunk + 2); }

// out[0 .. len) = exclusive prefix sums of in, out[len] = the total (len
// known to the host).  Long arrays take three passes over many blocks
// (chunk sums, their prefix sums, chunk scans from those offsets); ws holds
// scan_ws_size(len) words.
inline void scan_exclusive(const int32_t *in, int32_t *out, int len, int32_t *ws, cudaStream_t st) {
    if (len <= 4 * kScanChunk) {
        scan_kernel<<<1, kScanThreads, 0, st>>>(in, out, nullptr, len);
        return;
    }
    const int nb = (len + kScanChunk - 1) / kScanChunk;
    int32_t *bsum = ws, *boff = ws + nb + 1;
    scan_reduce_kernel<<<nb, kScanThreads, 0, st>>>(in, len, bsum);
    scan_kernel<<<1, kScanThreads, 0, st>>>(bsum, boff, nullptr, nb);
    scan_apply_kernel<<<nb, kScanThreads, 0, st>>>(in, out, len, boff);
}

// Stable sort of (key, val) pairs by the low `bits` bits of key.  The pairs
// start in (k0, v0); on return *ko/*vo point at whichever buffer holds the
// sorted pairs.
// hist and hoff hold 256 * tiles + 1 words, ws scan_ws_size of that.
void radix_sort(uint32_t *k0, int32_t *v0, uint32_t *k1, int32_t *v1, int count, int bits, int32_t *hist,
                int32_t *hoff, int32_t *ws, cudaStream_t st, uint32_t **ko, int32_t **vo) {
    const int ntiles = (count + kSortTile - 1) / kSortTile;
    for (int shift = 0; shift < bits && count > 0; shift += 8) {
        sort_hist_kernel<<<ntiles, kThreads, 0, st>>>(k0, count, shift, ntiles, hist);
        scan_exclusive(hist, hoff, 256 * ntiles, ws, st);
        sort_scatter_kernel<<<ntiles, kThreads, 0, st>>>(k0, v0, count, shift, ntiles, hoff, k1, v1);
        std::swap(k0, k1);
        std::swap(v0, v1);
    }
    *ko = k0;
    *vo = v0;
}

int fetch(void *h, const void *d, size_t bytes, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(h, d, bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return cuda_status(e);
}

}  // namespace
}  // namespace pars3
