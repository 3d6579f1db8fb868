// probe.cu -- pars3_fp64_fma_rate: the device's fp64 fused multiply-add
// throughput, measured with a kernel of independent FMA chains.  A
// measurement helper for reports (the fp64 products are bound by this pipe as
// much as by HBM on parts with a narrow fp64 unit); the paper has no
// counterpart.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace pars3 {

constexpr int kProbeChains = 8;      // independent FMA chains per thread
constexpr int kProbeIters = 2048;    // FMAs per chain
constexpr int kProbeBlock = 512;

// Every thread runs kProbeChains chains a <- a * m + c; the sums are written
// so the compiler keeps every FMA.  m and c come from the host so nothing is
// folded at compile time.
__global__ void __launch_bounds__(kProbeBlock) fma_probe_kernel(double m, double c, double *out) {
    double a[kProbeChains];
#pragma unroll
    for (int q = 0; q < kProbeChains; ++q) a[q] = threadIdx.x * 1e-9 + q;
    for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
        for (int q = 0; q < kProbeChains; ++q) a[q] = fma(a[q], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kProbeChains; ++q) s += a[q];
    if (s == 12345.678) out[0] = s;   // never true for the inputs below; keeps the chains live
}

}  // namespace pars3

using namespace pars3;

extern "C" int pars3_fp64_fma_rate(double *fma_per_s, void *stream) {
    if (!fma_per_s) return PARS3_EINVAL;
    *fma_per_s = 0.0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.f;
    const int grid = 2 * sm_count() * 4;   // several waves of two resident blocks per SM
    for (int rep = 0; e == cudaSuccess && rep < 4; ++rep) {   // the first run warms up
        cudaEventRecord(e0, st);
        fma_probe_kernel<<<grid, kProbeBlock, 0, st>>>(0.999999, 1e-7, out);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    if (e != cudaSuccess) return cuda_status(e);
    const double fmas = static_cast<double>(grid) * kProbeBlock * kProbeChains * kProbeIters;
    *fma_per_s = best > 0.f ? fmas / (1e-3 * best) : 0.0;
    return PARS3_OK;
}
