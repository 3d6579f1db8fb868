// devcommon.cuh -- device helpers shared by the kernels of libpars3:
// value types, TMA bulk copies with mbarrier completion (inline PTX for
// sm_100-class GPUs), bounded waits that report through an error word, and
// warp helpers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pars3.h"

namespace pars3 {

// error bits written to the handle's device error word
constexpr int kErrTmaTimeout = 1;

// ----------------------------------------------------------- value access
// bf16 values are stored as their 16 high bits of an fp32 value
__device__ __forceinline__ float bf16_bits_to_f32(uint16_t b) { return __uint_as_float(static_cast<uint32_t>(b) << 16); }

template <typename VT> struct Val;
template <> struct Val<double> {
    using acc = double;
    static __device__ __forceinline__ double ld(const double *p) { return __ldg(p); }
    static __device__ __forceinline__ double ld_stream(const double *p) { return __ldcs(p); }
};
template <> struct Val<float> {
    using acc = float;
    static __device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ float ld_stream(const float *p) { return __ldcs(p); }
};
template <> struct Val<uint16_t> {
    using acc = float;
    static __device__ __forceinline__ float ld(const uint16_t *p) { return bf16_bits_to_f32(__ldg(p)); }
    static __device__ __forceinline__ float ld_stream(const uint16_t *p) {
        return bf16_bits_to_f32(__ldcs(reinterpret_cast<const unsigned short *>(p)));
    }
};

// ----------------------------------------------------- mbarrier + bulk copy
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Ends the barrier's life once every thread has passed its last wait, so
// that the shared memory it occupied can hold data (or a new barrier) again.
__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Orders this thread's earlier generic-proxy accesses to shared memory before
// later bulk-copy (async-proxy) writes into it.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared (TMA engine), completion counted on bar.
// dst, src 16-byte aligned, bytes a positive multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// L2 prefetch of [src, src + bytes) by the bulk-copy engine: nothing comes
// back to the SM and no barrier counts it.  src 16-byte aligned, bytes a
// multiple of 16.  Issued in pieces of at most kPrefetchPiece bytes.
constexpr uint32_t kPrefetchPiece = 32u << 10;
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint64_t bytes) {
    const char *p = static_cast<const char *>(src);
    while (bytes > 0) {
        const uint32_t b = bytes > kPrefetchPiece ? kPrefetchPiece : static_cast<uint32_t>(bytes);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(b) : "memory");
        p += b;
        bytes -= b;
    }
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of bar, giving up after ~2^31 SM cycles (about a
// second); on give-up the error word gets kErrTmaTimeout and the wait is
// repeated once more with the same limit so that no copy still in flight
// outlives the block.  Returns false on give-up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int32_t *err) {
    const long long limit = 1ll << 31;
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) {
            if (err) atomicOr(err, kErrTmaTimeout);
            long long t1 = clock64();
            while (!mbar_try_wait(bar, parity)) {
                if (clock64() - t1 > limit) break;
            }
            return false;
        }
    }
    return true;
}

}  // namespace pars3
