// noalloc.cu -- pars3_spmv_noalloc: the skew product with its scratch
// memory in a fixed, library-wide device array, so that the call itself
// allocates nothing.
//
// pars3_spmv keeps its scratch (the cross-tile halo sums and the long-row
// partial sums) in buffers that pars3_upload sizes for the handle.  Some
// callers cannot have the library allocate device memory for that: code
// whose device memory is all handed to another allocator (a framework's
// caching allocator or a pool that reserved the device), or loops running
// under a fixed memory budget where an allocation, or its failure, is not
// acceptable.  This variant uses g_spmv_scratch instead: a file-scope
// __device__ array of kNoAllocScratchBytes that every GPU loading the
// library holds until the process exits.
//
// Host code cannot use the array's name as a device address (it names a
// host-side stand-in), so the address is looked up with
// cudaGetSymbolAddress, once per device, on the first call made with that
// device current.  With CUDA's default lazy loading that lookup may also
// load this file's device code and so reserve the array on the device: the
// first call on each device should come before any stream capture and
// before any memory budget applies.
// Every call shares the array and leaves its contents behind: the kernels
// overwrite every scratch entry before reading it, so nothing needs
// clearing, but two calls that overlap on the GPU (different streams, no
// ordering between them) race on the array.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace pars3 {

constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;   // 4 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_spmv_scratch[kNoAllocScratchBytes];

static void *g_scratch_addr[kMaxDevices] = {};
static std::mutex g_scratch_mu;

// Device address of g_spmv_scratch on the current device.
static int scratch_on_current_device(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= kMaxDevices) return PARS3_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_spmv_scratch);
        if (e != cudaSuccess) return cuda_status(e);
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return PARS3_OK;
}

}  // namespace pars3

using namespace pars3;

extern "C" int pars3_spmv_noalloc(const pars3_handle *h, int32_t dtype, double alpha, const void *x, void *y,
                                  void *stream) {
    if (!h) return PARS3_EINVAL;
    if (dtype < 0 || dtype >= kNumDtypes) return PARS3_EINVAL;
    if (!(h->dtypes & PARS3_DTYPE_BIT(dtype))) return PARS3_EUNSUPPORTED;
    if (ready_on_device(h) != PARS3_OK) return PARS3_ESTATE;
    if (h->n == 0) return PARS3_OK;
    if (!x || !y || x == y) return PARS3_EINVAL;
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15u) return PARS3_EINVAL;
    const size_t asz = dtype == PARS3_F64 ? 8 : 4;
    const size_t halo_bytes = (h->L.hhrow.size() * asz + 255) / 256 * 256;
    const size_t part_bytes = static_cast<size_t>(h->L.nslots) * asz;
    if (halo_bytes + part_bytes > kNoAllocScratchBytes) return PARS3_EUNSUPPORTED;
    void *base = nullptr;
    int rc = scratch_on_current_device(&base);
    if (rc != PARS3_OK) return rc;
    unsigned char *b = static_cast<unsigned char *>(base);
    return launch_spmv_scratch(h, dtype, alpha, x, y, b, b + halo_bytes, stream);
}
