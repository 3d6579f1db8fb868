// capi.cu -- C ABI entry points of libpars3 that manage device state:
// upload, release, status, vector permutation, the operator calls and the
// host-buffer end-to-end product.  Host preprocessing lives in
// host_reorder.cpp / host_split.cpp, kernels in spmv.cu / mrs.cu /
// batched.cu.
#include <cuda_runtime.h>

#include <cstring>
#include <new>

#include "internal.h"

namespace pars3 {

int ready_on_device(const pars3_handle *h) {
    if (!h->uploaded) return PARS3_ESTATE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device) return PARS3_ESTATE;
    return PARS3_OK;
}

uint64_t device_bit() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    return 1ull << (dev & 63);
}

int cuda_status(int e) {
    if (e == cudaSuccess) return PARS3_OK;
    if (e == cudaErrorMemoryAllocation) return PARS3_ENOMEM;
    return PARS3_ECUDA;
}

template <typename T>
static int dev_copy(DevLayout &D, T **dst, const std::vector<T> &src, cudaStream_t st) {
    size_t bytes = src.size() * sizeof(T);
    if (bytes == 0) bytes = 16;  // keep every pointer valid
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, (bytes + 255) / 256 * 256);
    if (e != cudaSuccess) return cuda_status(e);
    D.owned.push_back(p);
    D.bytes += static_cast<int64_t>((bytes + 255) / 256 * 256);
    if (!src.empty()) {
        e = cudaMemcpyAsync(p, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_status(e);
    }
    *dst = static_cast<T *>(p);
    return PARS3_OK;
}

static int dev_alloc(DevLayout &D, void **dst, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, (bytes + 255) / 256 * 256);
    if (e != cudaSuccess) return cuda_status(e);
    D.owned.push_back(p);
    D.bytes += static_cast<int64_t>((bytes + 255) / 256 * 256);
    *dst = p;
    return PARS3_OK;
}

static void release_device(pars3_handle *h) {
    for (void *p : h->D.owned) cudaFree(p);
    h->D = DevLayout();
    h->uploaded = false;
}

static int upload_impl(pars3_handle *h, cudaStream_t st) {
    Layout &L = h->L;
    DevLayout &D = h->D;
    int rc = PARS3_OK;
#define UP(dst, src) \
    if ((rc = dev_copy(D, &(dst), (src), st)) != PARS3_OK) return rc
    UP(D.hoff, L.hoff);
    UP(D.hcnt, L.hcnt);
    UP(D.hrp, L.hrp);
    UP(D.hcol, L.hcol);
    UP(D.hcperm, L.hcperm);
    UP(D.hrowc, L.hrowc);
    UP(D.hcsoff, L.hcsoff);
    UP(D.hcsn, L.hcsn);
    UP(D.hcs, L.hcs);
    UP(D.hhoff, L.hhoff);
    UP(D.hhrow, L.hhrow);
    UP(D.sl_off, L.sl_off);
    UP(D.sl_ent, L.sl_ent);
    UP(D.sl_e, L.sl_e);
    UP(D.sl_meta, L.sl_meta);
    UP(D.fcol, L.fcol);
    UP(D.ls_ent, L.ls_ent);
    UP(D.ls_len, L.ls_len);
    UP(D.lcol, L.lcol);
    UP(D.fold_row, L.fold_row);
    UP(D.fold_halo, L.fold_halo);
    UP(D.fold_p0, L.fold_p0);
    UP(D.fold_np, L.fold_np);
    UP(D.fold_rem, L.fold_rem);
    UP(D.fold_heavy, L.fold_heavy);
    UP(D.perm, h->perm);
    if (h->dtypes & PARS3_DTYPE_BIT(PARS3_F64)) {
        double *a, *b, *c;
        UP(a, L.hval64); UP(b, L.fval64); UP(c, L.lval64);
        D.hval[PARS3_F64] = a; D.fval[PARS3_F64] = b; D.lval[PARS3_F64] = c;
    }
    if (h->dtypes & PARS3_DTYPE_BIT(PARS3_F32)) {
        float *a, *b, *c;
        UP(a, L.hval32); UP(b, L.fval32); UP(c, L.lval32);
        D.hval[PARS3_F32] = a; D.fval[PARS3_F32] = b; D.lval[PARS3_F32] = c;
    }
    if (h->dtypes & PARS3_DTYPE_BIT(PARS3_BF16)) {
        uint16_t *a, *b, *c;
        UP(a, L.hval16); UP(b, L.fval16); UP(c, L.lval16);
        D.hval[PARS3_BF16] = a; D.fval[PARS3_BF16] = b; D.lval[PARS3_BF16] = c;
    }
#undef UP
    // scratch sized for fp64 accumulators and one right-hand side
    if ((rc = dev_alloc(D, &D.halo, L.hhrow.size() * sizeof(double))) != PARS3_OK) return rc;
    if ((rc = dev_alloc(D, &D.lpart, static_cast<size_t>(L.nslots) * sizeof(double))) != PARS3_OK) return rc;
    D.scratch_k = 1;
    void *err = nullptr;
    if ((rc = dev_alloc(D, &err, sizeof(int32_t))) != PARS3_OK) return rc;
    D.err = static_cast<int32_t *>(err);
    cudaError_t e = cudaMemsetAsync(D.err, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaStreamSynchronize(st);
    return cuda_status(e);
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

static int check_call(const pars3_handle *h, int dtype, const void *x, const void *y) {
    if (!h) return PARS3_EINVAL;
    if (dtype < 0 || dtype >= kNumDtypes) return PARS3_EINVAL;
    if (!(h->dtypes & PARS3_DTYPE_BIT(dtype))) return PARS3_EUNSUPPORTED;
    if (ready_on_device(h) != PARS3_OK) return PARS3_ESTATE;
    if (h->n > 0 && (!x || !y || !aligned16(x) || !aligned16(y))) return PARS3_EINVAL;
    if (x == y && h->n > 0) return PARS3_EINVAL;
    return PARS3_OK;
}

}  // namespace pars3

using namespace pars3;

extern "C" const char *pars3_strerror(int code) {
    switch (code) {
        case PARS3_OK: return "ok";
        case PARS3_EINVAL: return "invalid argument";
        case PARS3_ENOTSKEW: return "input is not a strict lower triangle (entry on/above the diagonal, unsorted or duplicate column, bad row pointer)";
        case PARS3_ENOMEM: return "out of memory";
        case PARS3_ECUDA: return "CUDA runtime error";
        case PARS3_ENOCONV: return "MRS did not reach the tolerance within the iteration limit";
        case PARS3_ETIMEOUT: return "a bounded device-side wait gave up";
        case PARS3_EUNSUPPORTED: return "unsupported request (precision not packed or size limit)";
        case PARS3_ESTATE: return "handle not ready (not uploaded)";
        case PARS3_ENONFINITE: return "NaN or Inf in the input values";
        default: return "unknown status";
    }
}

extern "C" int pars3_version(int32_t *major, int32_t *minor, int32_t *arch) {
    if (major) *major = 1;
    if (minor) *minor = 0;
    if (arch) *arch = 103;
    return PARS3_OK;
}

extern "C" int pars3_upload(pars3_handle *h, void *stream) {
    if (!h) return PARS3_EINVAL;
    if (h->uploaded) return PARS3_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    int rc;
    try {
        rc = upload_impl(h, static_cast<cudaStream_t>(stream));
    } catch (const std::bad_alloc &) {
        rc = PARS3_ENOMEM;
    }
    if (rc != PARS3_OK) {
        release_device(h);
        return rc;
    }
    h->uploaded = true;
    h->device = dev;
    return PARS3_OK;
}

void pars3_release_graphs(pars3_handle *h);
void pars3_release_batch(pars3_handle *h);

extern "C" void pars3_free(pars3_handle *h) {
    if (!h) return;
    pars3_release_graphs(h);
    pars3_release_batch(h);
    release_device(h);
    delete h;
}

extern "C" int pars3_check(const pars3_handle *h, void *stream) {
    if (!h) return PARS3_EINVAL;
    if (ready_on_device(h) != PARS3_OK) return PARS3_ESTATE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int32_t v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, h->D.err, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->D.err, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    return v ? PARS3_ETIMEOUT : PARS3_OK;
}

extern "C" int pars3_spmv(const pars3_handle *h, int32_t dtype, double alpha, const void *x, void *y,
                          void *stream) {
    int rc = check_call(h, dtype, x, y);
    if (rc != PARS3_OK) return rc;
    if (h->n == 0) return PARS3_OK;
    return launch_spmv(h, dtype, alpha, 1, x, y, stream);
}

extern "C" int pars3_permute(const pars3_handle *h, int32_t dtype, int32_t k, const void *src, void *dst,
                             void *stream) {
    int rc = check_call(h, dtype, src, dst);
    if (rc != PARS3_OK) return rc;
    if (k < 1) return PARS3_EINVAL;
    return launch_permute(h, dtype, k, src, dst, false, stream);
}

extern "C" int pars3_unpermute(const pars3_handle *h, int32_t dtype, int32_t k, const void *src, void *dst,
                               void *stream) {
    int rc = check_call(h, dtype, src, dst);
    if (rc != PARS3_OK) return rc;
    if (k < 1) return PARS3_EINVAL;
    return launch_permute(h, dtype, k, src, dst, true, stream);
}

extern "C" int pars3_spmv_host(pars3_handle *h, int32_t dtype, double alpha, const void *x_host, void *y_host,
                               void *stream) {
    if (!h || !x_host || !y_host) return PARS3_EINVAL;
    if (dtype < 0 || dtype >= kNumDtypes) return PARS3_EINVAL;
    if (!(h->dtypes & PARS3_DTYPE_BIT(dtype))) return PARS3_EUNSUPPORTED;
    if (ready_on_device(h) != PARS3_OK) return PARS3_ESTATE;
    if (h->n == 0) return PARS3_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bytes = static_cast<size_t>(h->n) * (dtype == PARS3_F64 ? 8 : 4);
    DevLayout &D = h->D;
    int rc;
    if (!D.stage_x) {
        if ((rc = dev_alloc(D, &D.stage_x, 8ull * h->n)) != PARS3_OK) return rc;
        if ((rc = dev_alloc(D, &D.stage_y, 8ull * h->n)) != PARS3_OK) return rc;
        if ((rc = dev_alloc(D, &D.stage_px, 8ull * h->n)) != PARS3_OK) return rc;
        if ((rc = dev_alloc(D, &D.stage_py, 8ull * h->n)) != PARS3_OK) return rc;
    }
    cudaError_t e = cudaMemcpyAsync(D.stage_x, x_host, bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_status(e);
    if ((rc = launch_permute(h, dtype, 1, D.stage_x, D.stage_px, false, st)) != PARS3_OK) return rc;
    if ((rc = launch_spmv(h, dtype, alpha, 1, D.stage_px, D.stage_py, st)) != PARS3_OK) return rc;
    if ((rc = launch_permute(h, dtype, 1, D.stage_py, D.stage_y, true, st)) != PARS3_OK) return rc;
    e = cudaMemcpyAsync(y_host, D.stage_y, bytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaStreamSynchronize(st);
    return cuda_status(e);
}
