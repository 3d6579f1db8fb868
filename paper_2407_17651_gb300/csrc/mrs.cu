// mrs.cu -- the minimal residual (MRS) method for (alpha I + S) x = b on the
// device (Sec. 1: MRS needs one product and one inner product per
// iteration), plain in fp64 or as an fp32 / bf16-value inner solver inside
// fp64 iterative refinement.
//
// Recurrence (skew Lanczos + Givens; x_k minimises ||b - A x|| over
// x0 + K_k(S, r0)):
//   v_1 = r0/beta_0, w = S v_j + beta_{j-1} v_{j-1}, beta_j = ||w||,
//   gamma_1 = alpha, rho_j = hypot(gamma_j, beta_j), c_j = gamma_j/rho_j,
//   s_j = beta_j/rho_j, gamma_{j+1} = alpha/c_j, R[j-2,j] = -s_{j-2} beta_{j-1},
//   p_j = (v_j - R[j-2,j] p_{j-2}) / rho_j, tau_j = c_j t_j, t_{j+1} = -s_j t_j,
//   x_j = x_{j-1} + tau_j p_j, ||r_j|| = |t_{j+1}|.
// Only w vectors are stored (v_j = w_{j-1}/beta_{j-1}); iteration j is two
// launches: the tile kernel in Lanczos mode (w_j, its partial norms, and the
// lagged p/x update of iteration j-1) and the fold kernel below (halo and
// long-row sums, the fixed-order norm reduction, the scalar recurrence and
// the loop condition).  The loop runs as a CUDA graph with a device-side
// while-condition; the host syncs once per refinement cycle.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "spmv_kernels.cuh"

namespace pars3 {

constexpr int kRedBlock = 256;
constexpr int kBodyUnroll = 4;   // MRS iterations per pass of the graph's while node
constexpr int kMaxRedBlocks = 1024;

// Fold of MRS iteration j: w_j[r] += (halo + long-row partials) / beta_{j-1}
// for the rows the tile kernel left open, their squared norms, then (last
// block) beta_j from all partial norms and the Givens step.
template <typename XT, typename AT>
__global__ void __launch_bounds__(kRedBlock) fold_mrs_kernel(
    int nitems, const FoldLists F, const AT *__restrict__ halo, const AT *__restrict__ lpart,
    const MrsVectors<XT> m, int ntiles, cudaGraphConditionalHandle cond, int in_graph) {
    __shared__ double red[32];
    MrsState *st = m.st;
    if (st->done) {   // an unrolled loop body past convergence (or a solve that starts converged)
        if (in_graph && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
        return;
    }
    const int j = st->j + 1;
    XT *y = m.w[j % 3];
    const AT scale = static_cast<AT>(st->e_scale);   // 1 / beta_{j-1}
    double nrm = 0.0;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int w = gw; w < F.nheavy; w += nw) {   // heavy rows, a warp each (as in the plain fold)
        const int f = __ldg(F.heavy + w);
        const AT sp = heavy_pieces_warp<AT>(__ldg(F.p0 + f), __ldg(F.np + f), lpart, 1, 0);
        if (lane == 0) {
            const int r = __ldg(F.row + f), hi = __ldg(F.halo + f), rem = __ldg(F.rem + f);
            AT s = AT(0);
            if (hi >= 0) s += halo[hi];
            s += sp;
            if (rem >= 0) s += lpart[rem];
            const XT wx = static_cast<XT>(static_cast<AT>(y[r]) + s * scale);
            y[r] = wx;
            nrm += static_cast<double>(wx) * static_cast<double>(wx);
        }
    }
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nitems; f += gridDim.x * blockDim.x) {
        const int np = __ldg(F.np + f);
        if (np >= kFoldHeavy) continue;
        const int r = __ldg(F.row + f), hi = __ldg(F.halo + f);
        AT s = AT(0);
        if (hi >= 0) s += halo[hi];
        s = long_row_sum<AT>(__ldg(F.p0 + f), np, __ldg(F.rem + f), lpart, 1, 0, s);
        const XT wx = static_cast<XT>(static_cast<AT>(y[r]) + s * scale);
        y[r] = wx;
        nrm += static_cast<double>(wx) * static_cast<double>(wx);
    }
    const double bs = block_sum(nrm, red);
    if (threadIdx.x == 0) m.part[ntiles + blockIdx.x] = bs;
    double tot = 0.0;
    if (!last_block_sum(&st->ticket, m.part, ntiles + gridDim.x, red, &tot)) return;
    if (threadIdx.x == 0) mrs_step(st, tot, cond, in_graph);
}

// Start of an inner solve on rhs r scaled by inv: w_0 = r*inv, w_{-1} = 0,
// p ring = 0, x = 0, beta_0 = ||w_0||, t_1 = beta_0, gamma_1 = alpha.
template <typename XT>
__global__ void __launch_bounds__(kRedBlock) mrs_init_kernel(int n, const double *__restrict__ r, double inv,
                                                            const MrsVectors<XT> m, double alpha, double rel_tol,
                                                            int jmax) {
    __shared__ double red[32];
    double nrm = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const XT w0 = static_cast<XT>(r[i] * inv);
        m.w[0][i] = w0;
        m.w[1][i] = XT(0);
        m.w[2][i] = XT(0);
        m.p[0][i] = XT(0);
        m.p[1][i] = XT(0);
        m.p[2][i] = XT(0);
        m.xsol[i] = XT(0);
        nrm += static_cast<double>(w0) * static_cast<double>(w0);
    }
    const double bs = block_sum(nrm, red);
    if (threadIdx.x == 0) m.part[blockIdx.x] = bs;
    double tot = 0.0;
    MrsState *st = m.st;
    if (!last_block_sum(&st->ticket, m.part, gridDim.x, red, &tot)) return;
    if (threadIdx.x != 0) return;
    const double b0 = sqrt(tot);
    for (int k = 0; k < 4; ++k) {
        st->beta[k] = 0.0;
        st->rho[k] = 1.0;
        st->c[k] = 1.0;
        st->s[k] = 0.0;
        st->tau[k] = 0.0;
    }
    st->beta[0] = b0;
    st->t = b0;
    st->gamma = alpha;
    st->alpha = alpha;
    st->tol = rel_tol * b0;
    st->j = 0;
    st->jmax = jmax;
    st->done = b0 == 0.0;
    mrs_next_coeffs(st, 0.0);
}

// After the last iteration J: p_J = (w_{J-1}/beta_{J-1} - R[J-2,J] p_{J-2}) / rho_J,
// x += tau_J p_J.  These are the lagged-update scalars of iteration J + 1,
// already in the state (mrs_next_coeffs).
template <typename XT, typename AT>
__global__ void mrs_finish_kernel(int n, const MrsVectors<XT> m) {
    const MrsState *st = m.st;
    const int J = st->j;
    if (J < 1) return;
    const AT inv_b = static_cast<AT>(st->e_inv_b2);
    const AT rr = static_cast<AT>(st->e_r3);
    const AT inv_rho = static_cast<AT>(st->e_inv_rho);
    const AT tau = static_cast<AT>(st->e_tau);
    const XT *wv = m.w[(J + 2) % 3];
    const XT *pp = m.p[(J + 1) % 3];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const AT pv = (static_cast<AT>(wv[i]) * inv_b - rr * static_cast<AT>(pp[i])) * inv_rho;
        m.xsol[i] = static_cast<XT>(static_cast<AT>(m.xsol[i]) + tau * pv);
    }
}

// r = b - y and ||r||^2 (fp64); with y == nullptr, ||b||^2.
__global__ void __launch_bounds__(kRedBlock) residual_kernel(int n, const double *__restrict__ b,
                                                             const double *__restrict__ y, double *__restrict__ r,
                                                             double *part, unsigned *ticket, double *out) {
    __shared__ double red[32];
    double nrm = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = y ? b[i] - y[i] : b[i];
        if (r) r[i] = v;
        nrm += v * v;
    }
    const double bs = block_sum(nrm, red);
    if (threadIdx.x == 0) part[blockIdx.x] = bs;
    double tot = 0.0;
    if (!last_block_sum(ticket, part, gridDim.x, red, &tot)) return;
    if (threadIdx.x == 0) *out = tot;
}

// x += scale * d
template <typename XT>
__global__ void axpy_kernel(int n, double scale, const XT *__restrict__ d, double *__restrict__ x) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        x[i] += scale * static_cast<double>(d[i]);
}

// ------------------------------------------------------------------ host

// Device workspace and the captured loop of one inner precision.
struct MrsGraph {
    void *w[3] = {nullptr, nullptr, nullptr}, *p[3] = {nullptr, nullptr, nullptr}, *xsol = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle cond = 0;
};

struct MrsWork {
    bool ready = false;
    double *r = nullptr, *y = nullptr;       // fp64 residual and product
    MrsState *st = nullptr;
    double *part = nullptr;                  // partial norms
    unsigned *ticket = nullptr;              // reduction ticket of residual_kernel
    double *scal = nullptr;                  // reduction results (device)
    uint32_t *fold_bits = nullptr;
    MrsGraph g[kNumDtypes];
    std::vector<void *> owned;
    cudaStream_t capture = nullptr;
};

static int work_alloc(MrsWork &W, void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) return cuda_status(e);
    W.owned.push_back(*p);
    return PARS3_OK;
}

static int fold_blocks(const pars3_handle *h) {
    const int nf = static_cast<int>(h->L.fold_row.size());
    return std::max(1, std::min(kMaxRedBlocks, (nf + kRedBlock - 1) / kRedBlock));
}

static int red_blocks(int n) { return std::max(1, std::min(kMaxRedBlocks, (n + kRedBlock - 1) / kRedBlock)); }

static int ensure_work(pars3_handle *h, MrsWork *&W) {
    if (!h->graph_cache) h->graph_cache = new (std::nothrow) MrsWork();
    if (!h->graph_cache) return PARS3_ENOMEM;
    W = static_cast<MrsWork *>(h->graph_cache);
    if (W->ready) return PARS3_OK;
    const size_t n = static_cast<size_t>(h->n);
    int rc;
    void *p;
    if ((rc = work_alloc(*W, &p, n * 8)) != PARS3_OK) return rc;
    W->r = static_cast<double *>(p);
    if ((rc = work_alloc(*W, &p, n * 8)) != PARS3_OK) return rc;
    W->y = static_cast<double *>(p);
    if ((rc = work_alloc(*W, &p, sizeof(MrsState))) != PARS3_OK) return rc;
    W->st = static_cast<MrsState *>(p);
    const size_t nparts = static_cast<size_t>(h->ntiles) + kMaxRedBlocks + 8;
    if ((rc = work_alloc(*W, &p, nparts * 8)) != PARS3_OK) return rc;
    W->part = static_cast<double *>(p);
    if ((rc = work_alloc(*W, &p, 64)) != PARS3_OK) return rc;
    W->ticket = static_cast<unsigned *>(p);
    if ((rc = work_alloc(*W, &p, 64)) != PARS3_OK) return rc;
    W->scal = static_cast<double *>(p);
    // rows the fold kernel finishes (their norms are taken there)
    std::vector<uint32_t> bits((n + 31) / 32 + 1, 0u);
    for (int32_t r : h->L.fold_row) bits[r >> 5] |= 1u << (r & 31);
    if ((rc = work_alloc(*W, &p, bits.size() * 4)) != PARS3_OK) return rc;
    W->fold_bits = static_cast<uint32_t *>(p);
    cudaError_t e = cudaMemcpy(W->fold_bits, bits.data(), bits.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(W->st, 0, sizeof(MrsState));
    if (e == cudaSuccess) e = cudaMemset(W->ticket, 0, 64);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&W->capture, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_status(e);
    W->ready = true;
    return PARS3_OK;
}

template <typename VT, typename XT, typename AT>
static SpmvArgs<VT, XT, AT> spmv_args(const pars3_handle *h, int dtype) {
    return make_spmv_args<VT, XT, AT>(h, dtype);
}

// largest dynamic shared memory of a launch (the fused kernel also has a
// little static shared memory, which counts against the same per-block limit)
template <typename VT, typename XT, typename AT, bool S, bool F>
static cudaError_t set_mrs_smem(int) {
    return cudaFuncSetAttribute(tile_kernel_mrs<VT, XT, AT, S, F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kSmemLimit - 1024);
}

// Capture the loop body (tile kernel in Lanczos mode + MRS fold) once as
// the body of a while-node; the condition is set by the fold kernel.
template <typename VT, typename XT, typename AT>
static int build_graph(pars3_handle *h, int dtype, MrsWork &W) {
    MrsGraph &G = W.g[dtype];
    if (G.exec) return PARS3_OK;
    const size_t n = static_cast<size_t>(h->n);
    int rc;
    for (int k = 0; k < 3; ++k) {
        if ((rc = work_alloc(W, &G.w[k], n * sizeof(XT))) != PARS3_OK) return rc;
        if ((rc = work_alloc(W, &G.p[k], n * sizeof(XT))) != PARS3_OK) return rc;
    }
    if ((rc = work_alloc(W, &G.xsol, n * sizeof(XT))) != PARS3_OK) return rc;
    MrsVectors<XT> m;
    m.st = W.st;
    for (int k = 0; k < 3; ++k) {
        m.w[k] = static_cast<XT *>(G.w[k]);
        m.p[k] = static_cast<XT *>(G.p[k]);
    }
    m.xsol = static_cast<XT *>(G.xsol);
    m.fold_bits = W.fold_bits;
    m.part = W.part;
    const SpmvArgs<VT, XT, AT> a = spmv_args<VT, XT, AT>(h, dtype);
    // tile kernel with the epilogue vectors staged in shared memory when
    // they fit next to the tile's own staging area, else unstaged
    uint32_t vsz, xsz, asz;
    dtype_sizes(dtype, &vsz, &xsz, &asz);
    const uint32_t tile_total =
        smem_layout(h->T, h->W, static_cast<uint32_t>(round_up(h->L.max_tile_half, kAlignHalf)),
                    static_cast<uint32_t>(h->L.max_tile_cs), vsz, xsz, asz).total;
    const uint32_t staged_bytes = align128(tile_total) + 3u * EpiMrs<XT, AT, true>::slice_bytes(h->T);
    constexpr uint32_t kStaticSlack = 1024;   // static shared memory of the fused kernel
    // fp64 tiles without middle entries finish each row in the full pass
    // itself (no staging, no row sums in shared memory, the most L1 for the
    // gathers of the operand): measured 118 -> see DESIGN; others stage
    const bool direct_fp64 = sizeof(AT) == 8 && h->L.max_tile_half == 0;
    const bool stage = !direct_fp64 && staged_bytes + kStaticSlack <= static_cast<uint32_t>(kSmemLimit);
    const int smem = stage ? std::max(smem_bytes_for(h, dtype), static_cast<int>(staged_bytes)) : smem_bytes_for(h, dtype);
    const Layout &L = h->L;
    // fusing the step into the tile kernel saves a launch per iteration in
    // fp64 (measured 2 %) but costs 8 % in fp32, where the separate fold wins
    const bool fused = sizeof(AT) == 8 && L.fold_row.empty() && L.lrow.empty() &&
                       smem + static_cast<int>(kStaticSlack) <= kSmemLimit;
    cudaError_t e = cudaSuccess;
    if (stage && fused) e = set_mrs_smem<VT, XT, AT, true, true>(smem);
    else if (stage) e = set_mrs_smem<VT, XT, AT, true, false>(smem);
    else if (fused) e = set_mrs_smem<VT, XT, AT, false, true>(smem);
    else e = set_mrs_smem<VT, XT, AT, false, false>(smem);
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaGraphCreate(&G.graph, 0);
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaGraphConditionalHandleCreate(&G.cond, G.graph, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return cuda_status(e);
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = G.cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, G.graph, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) return cuda_status(e);
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(W.capture, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return cuda_status(e);
    const int grid = a.nlb + h->ntiles;
    const DevLayout &D = h->D;
    // kBodyUnroll iterations per pass of the while node (each launch returns
    // at once after convergence), so the node's own cost is paid less often
    for (int u = 0; u < kBodyUnroll; ++u) {
        if (stage && fused) tile_kernel_mrs<VT, XT, AT, true, true><<<grid, kBlock, smem, W.capture>>>(a, m, G.cond);
        else if (stage) tile_kernel_mrs<VT, XT, AT, true, false><<<grid, kBlock, smem, W.capture>>>(a, m, G.cond);
        else if (fused) tile_kernel_mrs<VT, XT, AT, false, true><<<grid, kBlock, smem, W.capture>>>(a, m, G.cond);
        else tile_kernel_mrs<VT, XT, AT, false, false><<<grid, kBlock, smem, W.capture>>>(a, m, G.cond);
        if (!fused)
            fold_mrs_kernel<XT, AT><<<fold_blocks(h), kRedBlock, 0, W.capture>>>(
                static_cast<int>(L.fold_row.size()), fold_lists(D, L), static_cast<const AT *>(D.halo),
                static_cast<const AT *>(D.lpart),
                m, h->ntiles, G.cond, 1);
    }
    cudaGraph_t captured = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(W.capture, &captured);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaGraphInstantiate(&G.exec, G.graph, 0);
    return cuda_status(e);
}

static int inner_graph(pars3_handle *h, int dtype, MrsWork &W) {
    switch (dtype) {
        case PARS3_F64: return build_graph<double, double, double>(h, dtype, W);
        case PARS3_F32: return build_graph<float, float, float>(h, dtype, W);
        case PARS3_BF16: return build_graph<uint16_t, float, float>(h, dtype, W);
        default: return PARS3_EINVAL;
    }
}

template <typename XT>
static MrsVectors<XT> vectors(MrsWork &W, int dtype) {
    MrsVectors<XT> m;
    m.st = W.st;
    for (int k = 0; k < 3; ++k) {
        m.w[k] = static_cast<XT *>(W.g[dtype].w[k]);
        m.p[k] = static_cast<XT *>(W.g[dtype].p[k]);
    }
    m.xsol = static_cast<XT *>(W.g[dtype].xsol);
    m.fold_bits = W.fold_bits;
    m.part = W.part;
    return m;
}

// One inner solve of A d = r/||r|| in precision dtype; d accumulated into x
// with the factor ||r||.  Returns iterations in *iters and the recursive
// estimate |t| / beta_0 in *est.
static int inner_solve(pars3_handle *h, int dtype, MrsWork &W, double alpha, double rnorm, double rel_tol,
                       int jmax, double *x, cudaStream_t st, int *iters, double *est) {
    const int n = h->n;
    const int blocks = red_blocks(n);
    if (dtype == PARS3_F64) {
        MrsVectors<double> m = vectors<double>(W, dtype);
        mrs_init_kernel<double><<<blocks, kRedBlock, 0, st>>>(n, W.r, 1.0 / rnorm, m, alpha, rel_tol, jmax);
    } else {
        MrsVectors<float> m = vectors<float>(W, dtype);
        mrs_init_kernel<float><<<blocks, kRedBlock, 0, st>>>(n, W.r, 1.0 / rnorm, m, alpha, rel_tol, jmax);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaGraphLaunch(W.g[dtype].exec, st);
    if (e != cudaSuccess) return cuda_status(e);
    const int fb = std::min(8 * sm_count(), (n + 255) / 256);
    if (dtype == PARS3_F64) {
        MrsVectors<double> m = vectors<double>(W, dtype);
        mrs_finish_kernel<double, double><<<fb, 256, 0, st>>>(n, m);
        axpy_kernel<double><<<fb, 256, 0, st>>>(n, rnorm, m.xsol, x);
    } else {
        MrsVectors<float> m = vectors<float>(W, dtype);
        mrs_finish_kernel<float, float><<<fb, 256, 0, st>>>(n, m);
        axpy_kernel<float><<<fb, 256, 0, st>>>(n, rnorm, m.xsol, x);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    MrsState s;
    e = cudaMemcpyAsync(&s, W.st, sizeof(MrsState), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    *iters = s.j;
    *est = s.beta[0] > 0 ? std::fabs(s.t) / s.beta[0] : 0.0;
    return PARS3_OK;
}

// ||b - A x||^2 (fp64 product through the tile kernel), r left in W.r
static int true_residual(pars3_handle *h, MrsWork &W, double alpha, const double *b, const double *x,
                         cudaStream_t st, double *out) {
    int rc = launch_spmv(h, PARS3_F64, alpha, 1, x, W.y, st);
    if (rc != PARS3_OK) return rc;
    residual_kernel<<<red_blocks(h->n), kRedBlock, 0, st>>>(h->n, b, W.y, W.r, W.part, W.ticket, W.scal);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, W.scal, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return cuda_status(e);
}

}  // namespace pars3

using namespace pars3;

void pars3_release_graphs(pars3_handle *h) {
    if (!h || !h->graph_cache) return;
    MrsWork *W = static_cast<MrsWork *>(h->graph_cache);
    for (int d = 0; d < kNumDtypes; ++d) {
        if (W->g[d].exec) cudaGraphExecDestroy(W->g[d].exec);
        if (W->g[d].graph) cudaGraphDestroy(W->g[d].graph);
    }
    for (void *p : W->owned) cudaFree(p);
    if (W->capture) cudaStreamDestroy(W->capture);
    delete W;
    h->graph_cache = nullptr;
}

extern "C" int pars3_mrs(const pars3_handle *hc, double alpha, const double *b, double *x,
                         const pars3_mrs_opts *opts, pars3_mrs_result *res, void *stream) {
    pars3_handle *h = const_cast<pars3_handle *>(hc);
    if (!h || !opts) return PARS3_EINVAL;
    if (alpha == 0.0 || !std::isfinite(alpha)) return PARS3_EINVAL;
    const int inner = opts->inner;
    if (inner < 0 || inner >= kNumDtypes) return PARS3_EINVAL;
    if (!(h->dtypes & PARS3_DTYPE_BIT(PARS3_F64)) || !(h->dtypes & PARS3_DTYPE_BIT(inner))) return PARS3_EUNSUPPORTED;
    if (ready_on_device(h) != PARS3_OK) return PARS3_ESTATE;
    if (h->symmetric) return PARS3_EUNSUPPORTED;   // the recurrence needs a skew-symmetric S
    if (h->n > 0 && (!b || !x || (reinterpret_cast<uintptr_t>(b) & 15u) || (reinterpret_cast<uintptr_t>(x) & 15u)))
        return PARS3_EINVAL;
    pars3_mrs_result r{};
    r.status = PARS3_OK;
    if (h->n == 0) {
        if (res) *res = r;
        return PARS3_OK;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    MrsWork *W = nullptr;
    int rc = ensure_work(h, W);
    if (rc != PARS3_OK) return rc;
    rc = inner_graph(h, inner, *W);
    if (rc != PARS3_OK) return rc;
    const double rtol = opts->rtol > 0 ? opts->rtol : 1e-10;
    const int max_iter = opts->max_iter > 0 ? opts->max_iter : 100000;
    const int max_outer = opts->max_outer > 0 ? opts->max_outer : 50;
    const double inner_rtol = opts->inner_rtol > 0 ? opts->inner_rtol : 1e-5;
    // ||b||
    residual_kernel<<<red_blocks(h->n), kRedBlock, 0, st>>>(h->n, b, nullptr, nullptr, W->part, W->ticket, W->scal);
    double bb = 0.0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bb, W->scal, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    const double bnorm = std::sqrt(bb);
    if (bnorm == 0.0) {
        e = cudaMemsetAsync(x, 0, static_cast<size_t>(h->n) * 8, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (res) *res = r;
        return cuda_status(e);
    }
    int total = 0;
    double relres = 0.0;
    for (int outer = 0;; ++outer) {
        double rr = 0.0;
        if ((rc = true_residual(h, *W, alpha, b, x, st, &rr)) != PARS3_OK) return rc;
        relres = std::sqrt(rr) / bnorm;
        r.outer = outer;
        if (relres <= rtol) break;
        if (outer >= max_outer || total >= max_iter) {
            r.status = PARS3_ENOCONV;
            break;
        }
        // plain fp64: aim straight at the target; refinement: reduce by inner_rtol
        const double rnorm = std::sqrt(rr);
        const double rel = inner == PARS3_F64 ? std::max(0.5 * rtol * bnorm / rnorm, 1e-16) : inner_rtol;
        int it = 0;
        double est = 0.0;
        if ((rc = inner_solve(h, inner, *W, alpha, rnorm, rel, max_iter - total, x, st, &it, &est)) != PARS3_OK)
            return rc;
        total += it;
        r.est_relres = est * rnorm / bnorm;
        if (it == 0) {
            r.status = PARS3_ENOCONV;
            break;
        }
    }
    int32_t errw = 0;
    e = cudaMemcpyAsync(&errw, h->D.err, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    r.iters = total;
    r.true_relres = relres;
    if (res) *res = r;
    if (errw) return PARS3_ETIMEOUT;
    return r.status;
}
