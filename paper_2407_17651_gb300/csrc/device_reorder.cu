// device_reorder.cu -- pars3_reorder_device: the reverse Cuthill-McKee
// ordering of pars3_reorder (Sec. 1 and Sec. 3.1.2), computed on the GPU from
// a strict-lower pattern already in device memory.  The result is the same
// permutation, element for element, as the host ordering.
//
// Serial Cuthill-McKee dequeues vertices in order and appends each one's
// unvisited neighbours in (degree, index) order.  The same order is built
// one breadth-first level at a time:
//   * the vertices of level l+1 are the unvisited neighbours of level l;
//     each is appended by the FIRST vertex of level l (in queue order) that
//     is adjacent to it, so every such vertex is claimed by the smallest
//     queue position among its level-l neighbours (an atomic minimum);
//   * a parent's children keep its adjacency order, and adjacency lists are
//     sorted by the neighbours' (degree, index) rank once, up front, so no
//     sort runs per level;
//   * parents append in queue order, so a parent's first child slot is a
//     prefix sum of the children counts over the level.
// Connected components do not interact, so all of them are searched at once:
// components are placed in the order of their (degree, index)-smallest
// vertex (the serial start rule), each owns a contiguous queue segment, and
// a level step processes the current level of every unfinished component.
//
// Supporting pieces, all on the device: input validation, degrees, a stable
// LSD radix sort (32-bit keys with 32-bit values), connected components by
// union-find with hooking towards the smaller root, and single-block prefix
// sums for sizes that live in device memory.
#include "device_prims.cuh"

namespace pars3 {
namespace {

constexpr int kHookRounds = 1 << 22;                // bound on the union-find retries of one edge
constexpr int kLevelsPerCheck = 8;                  // level steps between two host checks
constexpr int kSmallComp = 1 << 19;                 // components up to this size are searched by one block each

// error bits of Ctl::err (bit kErrPattern is the pattern check's)
constexpr int kErrHook = 2;       // union-find retries ran out
constexpr int kErrPlaced = 4;     // a vertex was left without a position

struct Ctl {
    int err;
    int nact[2];                  // unfinished frontier entries, per buffer
    int level;                    // level steps taken
    int active;                   // components still moving their start (pseudo-peripheral search)
};

// One frontier entry: queue positions [fb, fe) are the current level of one
// component (comp is that component's index in start order).
struct Front {
    int fb, fe, comp, pad;
};

// deg[j] += number of rows holding column j (the upper part of each degree)
__global__ void degree_kernel(int nnz, const int32_t *__restrict__ ci, int32_t *deg) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += gridDim.x * blockDim.x)
        atomicAdd(&deg[ci[k]], 1);
}

// ------------------------------------------------------------ components

// Root of x.  Parents always point to a smaller index, so the walk ends
// after at most x steps; the path is halved on the way (every write stores
// an ancestor, so concurrent walks stay valid).
__device__ __forceinline__ int find_root(int *parent, int x) {
    volatile int *p = parent;
    int px = p[x];
    while (px != x) {
        const int g = p[px];
        if (g != px) p[x] = g;
        x = px;
        px = p[x];
    }
    return x;
}

// Union of the two ends of every stored entry: the larger root is hooked
// below the smaller one, so every component ends with its smallest vertex as
// root.  A failed compare-and-swap means the root was hooked meanwhile; the
// retries are bounded (each failure removes a root).
__global__ void hook_kernel(int nnz, const int32_t *__restrict__ rowof, const int32_t *__restrict__ ci,
                            int *parent, Ctl *ctl) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += gridDim.x * blockDim.x) {
        const int i = rowof[k], j = ci[k];
        bool done = false;
        for (int it = 0; it < kHookRounds && !done; ++it) {
            const int ri = find_root(parent, i), rj = find_root(parent, j);
            if (ri == rj) {
                done = true;
            } else {
                const int lo = min(ri, rj), hi = max(ri, rj);
                done = atomicCAS(&parent[hi], hi, lo) == hi;
            }
        }
        if (!done) atomicOr(&ctl->err, kErrHook);
    }
}

// comp[v] = root of v (the smallest vertex of its component); the smallest
// (degree, index) rank of each component and its size are gathered at the root.
__global__ void comp_kernel(int n, int *parent, const int32_t *__restrict__ rank, int32_t *__restrict__ comp,
                            int32_t *cmin, int32_t *csize) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int r = find_root(parent, v);
        comp[v] = r;
        atomicMin(&cmin[r], rank[v]);
        atomicAdd(&csize[r], 1);
    }
}

// rank[by_deg[i]] = i
__global__ void rank_kernel(int n, const int32_t *__restrict__ by_deg, int32_t *__restrict__ rank) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) rank[by_deg[i]] = i;
}

// flag[i] = 1 when the vertex of rank i is the (degree, index)-smallest of
// its component, i.e. the vertex serial Cuthill-McKee starts that component at
__global__ void start_flag_kernel(int n, const int32_t *__restrict__ by_deg, const int32_t *__restrict__ comp,
                                  const int32_t *__restrict__ cmin, int32_t *__restrict__ flag) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        flag[i] = cmin[comp[by_deg[i]]] == i ? 1 : 0;
}

// Components in start order: cstart[c] = the start candidate of the c-th
// component, csz[c] its size.
__global__ void start_list_kernel(int n, const int32_t *__restrict__ by_deg, const int32_t *__restrict__ comp,
                                  const int32_t *__restrict__ csize, const int32_t *__restrict__ flag,
                                  const int32_t *__restrict__ sidx, int32_t *__restrict__ cstart,
                                  int32_t *__restrict__ csz) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (!flag[i]) continue;
        const int v = by_deg[i];
        cstart[sidx[i]] = v;
        csz[sidx[i]] = csize[comp[v]];
    }
}

// ------------------------------------------------------------ adjacency

// Every directed edge (v -> u), listed source by source in (degree, index)
// order of the source: key = u, value = v.  One warp per source.  aun/cur
// is the unordered adjacency (filled with atomics, any order).
__global__ void edges_by_rank_kernel(int n, const int32_t *__restrict__ by_deg, const int32_t *__restrict__ arp,
                                     const int32_t *__restrict__ aun, const int32_t *__restrict__ epos,
                                     uint32_t *__restrict__ key, int32_t *__restrict__ val) {
    const int lane = threadIdx.x & 31;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += (gridDim.x * blockDim.x) >> 5) {
        const int v = by_deg[i];
        const int a = arp[v], d = arp[v + 1] - a, o = epos[i];
        for (int t = lane; t < d; t += 32) {
            key[o + t] = static_cast<uint32_t>(aun[a + t]);
            val[o + t] = v;
        }
    }
}

// unordered adjacency: both directions of every stored entry
__global__ void scatter_adj_kernel(int nnz, const int32_t *__restrict__ rowof, const int32_t *__restrict__ ci,
                                   const int32_t *__restrict__ arp, int32_t *cur, int32_t *__restrict__ aun) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += gridDim.x * blockDim.x) {
        const int i = rowof[k], j = ci[k];
        aun[arp[i] + atomicAdd(&cur[i], 1)] = j;
        aun[arp[j] + atomicAdd(&cur[j], 1)] = i;
    }
}

// out[pre[c]] = c for every c with flag[c] set
__global__ void compact_list_kernel(int count, const int32_t *__restrict__ flag, const int32_t *__restrict__ pre,
                                    int32_t *__restrict__ out) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < count; c += gridDim.x * blockDim.x)
        if (flag[c]) out[pre[c]] = c;
}

// ------------------------------------------------------------ level steps
//
// The current level is a list of frontier entries act[0 .. nact) (nact =
// ctl->nact[b]); fpre[s] is the number of frontier vertices before entry s,
// so flat index f in [0, fpre[nact]) names one frontier vertex.  One warp
// handles one frontier vertex and walks its adjacency list.

__device__ __forceinline__ int entry_of(const int32_t *__restrict__ fpre, int nact, int f) {
    int lo = 0, hi = nact;   // fpre[lo] <= f < fpre[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (fpre[mid] <= f) lo = mid;
        else hi = mid;
    }
    return lo;
}

// start positions: component c begins its queue segment at cbase[c] with
// root[c]; the large components (bigpos: their exclusive prefix count) form
// the first frontier of the grid-wide level steps
__global__ void bfs_init_kernel(int ncomp, const int32_t *__restrict__ root, const int32_t *__restrict__ cbase,
                                const int32_t *__restrict__ csz, const int32_t *__restrict__ bigpos,
                                int32_t *__restrict__ cm, int32_t *__restrict__ pos, Front *__restrict__ act,
                                int32_t *__restrict__ fpre, Ctl *ctl) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncomp; c += gridDim.x * blockDim.x) {
        const int v = root[c], q = cbase[c];
        cm[q] = v;
        pos[v] = q;
        if (csz[c] > kSmallComp) {
            const int k = bigpos[c];
            act[k] = Front{q, q + 1, c, 0};
            fpre[k] = k;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int nbig = bigpos[ncomp];
        fpre[nbig] = nbig;
        ctl->nact[0] = nbig;
        ctl->nact[1] = 0;
        ctl->level = 0;
    }
}

// size classes of the components: large ones take the grid-wide level
// steps, the others (more than one vertex) a block each
__global__ void comp_class_kernel(int ncomp, const int32_t *__restrict__ csz, int32_t *__restrict__ big,
                                  int32_t *__restrict__ small) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncomp; c += gridDim.x * blockDim.x) {
        big[c] = csz[c] > kSmallComp;
        small[c] = csz[c] > 1 && csz[c] <= kSmallComp;
    }
}

// single-vertex components: eccentricity 0, the last level is the vertex
__global__ void single_comp_kernel(int ncomp, const int32_t *__restrict__ csz, const int32_t *__restrict__ cbase,
                                   int32_t *__restrict__ ecc, int2 *__restrict__ last) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncomp; c += gridDim.x * blockDim.x)
        if (csz[c] == 1) {
            ecc[c] = 0;
            last[c] = make_int2(cbase[c], cbase[c] + 1);
        }
}

// One block searches one component of at most kSmallComp vertices through
// all its levels, with block barriers between the steps of a level (claim,
// count, prefix sum, write: the same steps as the grid-wide kernels), so a
// deep, narrow search costs no launch per level.  A frontier vertex of
// degree up to 32 is handled by one thread (its few neighbours in a loop),
// a larger one by a warp (lanes over its adjacency, ballots keeping the
// children in adjacency order).  Components go to blocks in turn; with ecc /
// last set, each one's eccentricity and last level are recorded.
__global__ void __launch_bounds__(kScanThreads) component_search_kernel(
    int nsmall, const int32_t *__restrict__ list, const int32_t *__restrict__ cbase, const int32_t *__restrict__ csz,
    const int32_t *__restrict__ arp, const int32_t *__restrict__ adj, int32_t *cm, int32_t *pos, int32_t *claim,
    int32_t *cnt, int32_t *coff, int32_t *__restrict__ ecc, int2 *__restrict__ last) {
    __shared__ int ws[32];
    const int tid = threadIdx.x, P = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = P >> 5;
    const unsigned lt = static_cast<unsigned>(lanemask_lt());
    for (int i = blockIdx.x; i < nsmall; i += gridDim.x) {
        const int c = list[i];
        const int end = cbase[c] + csz[c];
        int fb = cbase[c], fe = fb + 1, level = 0;
        for (;;) {
            // claim: every unvisited neighbour takes the smallest frontier position
            for (int q = fb + tid; q < fe; q += P) {
                const int v = cm[q], e1 = arp[v + 1];
                if (e1 - arp[v] > 32) continue;
                for (int e = arp[v]; e < e1; ++e) {
                    const int u = adj[e];
                    if (pos[u] < 0) atomicMin(&claim[u], q);
                }
            }
            for (int q = fb + warp; q < fe; q += nw) {
                const int v = cm[q], e1 = arp[v + 1];
                if (e1 - arp[v] <= 32) continue;
                for (int e = arp[v] + lane; e < e1; e += 32) {
                    const int u = adj[e];
                    if (pos[u] < 0) atomicMin(&claim[u], q);
                }
            }
            __syncthreads();
            // count: the children of every frontier vertex
            for (int q = fb + tid; q < fe; q += P) {
                const int v = cm[q], e1 = arp[v + 1];
                if (e1 - arp[v] > 32) continue;
                int k = 0;
                for (int e = arp[v]; e < e1; ++e) k += claim[adj[e]] == q;
                cnt[q] = k;
            }
            for (int q = fb + warp; q < fe; q += nw) {
                const int v = cm[q], e1 = arp[v + 1];
                if (e1 - arp[v] <= 32) continue;
                int k = 0;
                for (int e0 = arp[v]; e0 < e1; e0 += 32) {
                    const int e = e0 + lane;
                    k += __popc(__ballot_sync(0xffffffffu, e < e1 && claim[adj[e]] == q));
                }
                if (lane == 0) cnt[q] = k;
            }
            __syncthreads();
            block_scan_array(cnt + fb, coff + fb, fe - fb, ws);   // coff[fe] receives the level's total
            __syncthreads();
            const int total = coff[fe];
            // write: the children at their slots, in adjacency order
            for (int q = fb + tid; q < fe; q += P) {
                const int v = cm[q], e1 = arp[v + 1];
                if (e1 - arp[v] > 32) continue;
                int slot = fe + coff[q];
                for (int e = arp[v]; e < e1; ++e) {
                    const int u = adj[e];
                    if (claim[u] == q) {
                        cm[slot] = u;
                        pos[u] = slot;
                        ++slot;
                    }
                }
            }
            for (int q = fb + warp; q < fe; q += nw) {
                const int v = cm[q], e1 = arp[v + 1];
                if (e1 - arp[v] <= 32) continue;
                int slot = fe + coff[q];
                for (int e0 = arp[v]; e0 < e1; e0 += 32) {
                    const int e = e0 + lane;
                    const int u = e < e1 ? adj[e] : -1;
                    const bool hit = u >= 0 && claim[u] == q;
                    const unsigned m = __ballot_sync(0xffffffffu, hit);
                    if (hit) {
                        const int p = slot + __popc(m & lt);
                        cm[p] = u;
                        pos[u] = p;
                    }
                    slot += __popc(m);
                }
            }
            __syncthreads();
            if (total == 0 || fe + total > end) {   // done (the second test guards the segment)
                if (ecc && tid == 0) {
                    ecc[c] = level;
                    last[c] = make_int2(fb, fe);
                }
                break;
            }
            fb = fe;
            fe += total;
            ++level;
        }
    }
}

// Every unvisited neighbour u of frontier vertex q takes claim[u] = min(claim[u], q).
__global__ void __launch_bounds__(kThreads) claim_kernel(const Ctl *ctl, int b, const Front *__restrict__ act,
                                                         const int32_t *__restrict__ fpre,
                                                         const int32_t *__restrict__ cm,
                                                         const int32_t *__restrict__ arp,
                                                         const int32_t *__restrict__ adj,
                                                         const int32_t *__restrict__ pos, int32_t *claim) {
    const int nact = ctl->nact[b];
    const int F = fpre[nact];
    const int lane = threadIdx.x & 31;
    for (int f = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; f < F; f += (gridDim.x * blockDim.x) >> 5) {
        const int s = entry_of(fpre, nact, f);
        const int q = act[s].fb + f - fpre[s];
        const int v = cm[q];
        for (int e = arp[v] + lane; e < arp[v + 1]; e += 32) {
            const int u = adj[e];
            if (pos[u] < 0) atomicMin(&claim[u], q);
        }
    }
}

// cnt[f] = children of frontier vertex f (neighbours it claimed)
__global__ void __launch_bounds__(kThreads) count_kernel(const Ctl *ctl, int b, const Front *__restrict__ act,
                                                         const int32_t *__restrict__ fpre,
                                                         const int32_t *__restrict__ cm,
                                                         const int32_t *__restrict__ arp,
                                                         const int32_t *__restrict__ adj,
                                                         const int32_t *__restrict__ claim,
                                                         int32_t *__restrict__ cnt) {
    const int nact = ctl->nact[b];
    const int F = fpre[nact];
    const int lane = threadIdx.x & 31;
    for (int f = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; f < F; f += (gridDim.x * blockDim.x) >> 5) {
        const int s = entry_of(fpre, nact, f);
        const int q = act[s].fb + f - fpre[s];
        const int v = cm[q];
        int c = 0;
        for (int e0 = arp[v]; e0 < arp[v + 1]; e0 += 32) {
            const int e = e0 + lane;
            c += __popc(__ballot_sync(0xffffffffu, e < arp[v + 1] && claim[adj[e]] == q));
        }
        if (lane == 0) cnt[f] = c;
    }
}

// One block: coff = exclusive prefix of cnt over the level; the entries with
// children become the next level's entries (in order), each starting where
// its component's current level ends.  An entry without children closes its
// component's search: with track set, its level number (the eccentricity of
// the start) and its last level are recorded.
__global__ void __launch_bounds__(kScanThreads) plan_kernel(Ctl *ctl, int b, const Front *__restrict__ act,
                                                            const int32_t *__restrict__ fpre,
                                                            const int32_t *__restrict__ cnt,
                                                            int32_t *__restrict__ coff, Front *__restrict__ act2,
                                                            int32_t *__restrict__ fpre2, int32_t *__restrict__ ecc,
                                                            int2 *__restrict__ last) {
    __shared__ int ws[32];
    __shared__ long long wl[32];
    const int nact = ctl->nact[b];
    const int level = ctl->level;
    block_scan_array(cnt, coff, fpre[nact], ws);
    __syncthreads();
    long long carry = 0;   // (entries kept) << 32 | children so far
    for (int base = 0; base < nact; base += kScanThreads) {
        const int s = base + threadIdx.x;
        int ch = 0;
        Front e{};
        if (s < nact) {
            e = act[s];
            ch = coff[fpre[s + 1]] - coff[fpre[s]];
            if (ch == 0 && ecc) {
                ecc[e.comp] = level;
                last[e.comp] = make_int2(e.fb, e.fe);
            }
        }
        const long long mine = ch > 0 ? ((1LL << 32) | ch) : 0LL;
        long long total;
        const long long before = carry + block_excl_scan<long long>(mine, wl, &total);
        if (ch > 0) {
            const int k = static_cast<int>(before >> 32);
            act2[k] = Front{e.fe, e.fe + ch, e.comp, 0};
            fpre2[k] = static_cast<int>(before & 0xffffffffLL);
        }
        carry += total;
    }
    if (threadIdx.x == 0) {
        const int kept = static_cast<int>(carry >> 32);
        fpre2[kept] = static_cast<int>(carry & 0xffffffffLL);
        ctl->nact[b ^ 1] = kept;
        ctl->level = level + 1;
    }
}

// Frontier vertex q appends the neighbours it claimed, in adjacency order,
// from slot fe(entry) + coff[f] - coff[first f of the entry].
__global__ void __launch_bounds__(kThreads) write_kernel(const Ctl *ctl, int b, const Front *__restrict__ act,
                                                         const int32_t *__restrict__ fpre,
                                                         const int32_t *__restrict__ coff, int32_t *cm,
                                                         const int32_t *__restrict__ arp,
                                                         const int32_t *__restrict__ adj,
                                                         const int32_t *__restrict__ claim,
                                                         int32_t *__restrict__ pos) {
    const int nact = ctl->nact[b];
    const int F = fpre[nact];
    const int lane = threadIdx.x & 31;
    const unsigned lt = static_cast<unsigned>(lanemask_lt());
    for (int f = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; f < F; f += (gridDim.x * blockDim.x) >> 5) {
        const int s = entry_of(fpre, nact, f);
        const Front e = act[s];
        const int q = e.fb + f - fpre[s];
        const int v = cm[q];
        int slot = e.fe + coff[f] - coff[fpre[s]];
        const int end = arp[v + 1];
        for (int e0 = arp[v]; e0 < end; e0 += 32) {
            const int i = e0 + lane;
            const int u = i < end ? adj[i] : -1;
            const bool hit = u >= 0 && claim[u] == q;
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (hit) {
                const int p = slot + __popc(m & lt);
                cm[p] = u;
                pos[u] = p;
            }
            slot += __popc(m);
        }
    }
}

// x[c] = the vertex of smallest (degree, index) rank in the last level of c
__global__ void last_min_kernel(int ncomp, const int2 *__restrict__ last, const int32_t *__restrict__ cm,
                                const int32_t *__restrict__ rank, const int32_t *__restrict__ by_deg,
                                int32_t *__restrict__ x) {
    const int lane = threadIdx.x & 31;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < ncomp; c += (gridDim.x * blockDim.x) >> 5) {
        const int2 L = last[c];
        int best = INT_MAX;
        for (int q = L.x + lane; q < L.y; q += 32) best = min(best, rank[cm[q]]);
        best = __reduce_min_sync(0xffffffffu, best);
        if (lane == 0) x[c] = by_deg[best];
    }
}

// One George-Liu step per still-active component: the search from x[c]
// reached eccentricity ex[c]; when that exceeds e[c], r moves to x and x to
// y (the smallest vertex of the new last level), else the component is done.
__global__ void peripheral_step_kernel(int ncomp, int32_t *__restrict__ active, int32_t *__restrict__ r,
                                       int32_t *__restrict__ e, int32_t *__restrict__ x,
                                       const int32_t *__restrict__ ex, const int32_t *__restrict__ y, Ctl *ctl) {
    int still = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncomp; c += gridDim.x * blockDim.x) {
        if (!active[c]) continue;
        if (ex[c] > e[c]) {
            r[c] = x[c];
            e[c] = ex[c];
            x[c] = y[c];
            ++still;
        } else {
            active[c] = 0;
        }
    }
    still = __reduce_add_sync(0xffffffffu, still);
    if ((threadIdx.x & 31) == 0 && still) atomicAdd(&ctl->active, still);
}

// start of every component for the next search: x[c] while active, else r[c]
__global__ void select_kernel(int ncomp, const int32_t *__restrict__ active, const int32_t *__restrict__ r,
                              const int32_t *__restrict__ x, int32_t *__restrict__ out) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncomp; c += gridDim.x * blockDim.x)
        out[c] = active[c] ? x[c] : r[c];
}


// ------------------------------------------------------------ result

// Each matrix's vertices hold the queue positions [moff[m], moff[m+1]) (its
// components come first in rank order); its permutation is that segment
// reversed, in the matrix's own numbering.
__global__ void perm_kernel(int n, Blocks B, const int32_t *__restrict__ cm, const int32_t *__restrict__ pos,
                            int32_t *const *__restrict__ perms, Ctl *ctl) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
        const int m = B.mid ? B.mid[g] : 0;
        const int o = B.moff[m], nm = B.moff[m + 1] - o;
        const int k = g - o;
        perms[m][k] = cm[o + nm - 1 - k] - o;
        if (pos[g] < 0) atomicOr(&ctl->err, kErrPlaced);
    }
}

// Bandwidths of every matrix before (i - j over its stored (i, j)) and
// after (|pos i - pos j|, the same distance in the reversed order):
// bw[2m] and bw[2m+1].
__global__ void bandwidth_kernel(int nnz, const int32_t *mid, const int32_t *__restrict__ rowof,
                                 const int32_t *__restrict__ ci, const int32_t *__restrict__ pos,
                                 unsigned long long *bw) {
    const int lane = threadIdx.x & 31;
    for (int k0 = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; k0 < nnz; k0 += gridDim.x * blockDim.x) {
        const int k = k0 + lane;
        unsigned d0 = 0, d1 = 0;
        int m = -1;
        if (k < nnz) {
            const int i = rowof[k], j = ci[k];
            m = mid ? mid[i] : 0;
            d0 = static_cast<unsigned>(i - j);
            d1 = static_cast<unsigned>(abs(pos[i] - pos[j]));
        }
        const int m0 = __shfl_sync(0xffffffffu, m, 0);
        if (__all_sync(0xffffffffu, m == m0 || m < 0)) {   // one matrix in this warp
            d0 = __reduce_max_sync(0xffffffffu, d0);
            d1 = __reduce_max_sync(0xffffffffu, d1);
            if (lane == 0 && m0 >= 0) {
                atomicMax(&bw[2 * m0], static_cast<unsigned long long>(d0));
                atomicMax(&bw[2 * m0 + 1], static_cast<unsigned long long>(d1));
            }
        } else if (m >= 0) {
            atomicMax(&bw[2 * m], static_cast<unsigned long long>(d0));
            atomicMax(&bw[2 * m + 1], static_cast<unsigned long long>(d1));
        }
    }
}

// ------------------------------------------------------------ batches

// nnz of every matrix: nz[m] = rowptr_m[n_m]
__global__ void nnz_kernel(int count, const int32_t *const *__restrict__ rps, const int32_t *__restrict__ ns,
                           int32_t *__restrict__ nz) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < count; m += gridDim.x * blockDim.x)
        nz[m] = rps[m][ns[m]];
}

__device__ __forceinline__ int block_of(const int32_t *__restrict__ off, int count, int x) {
    int lo = 0, hi = count;   // off[lo] <= x < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

// the union's row pointers (each matrix's shifted by its first entry) and
// the matrix of every vertex (the search lands on the matrix whose range
// holds g, so matrices without vertices are passed over)
__global__ void union_rows_kernel(int n, int count, const int32_t *const *__restrict__ rps,
                                  const int32_t *__restrict__ moff, const int32_t *__restrict__ eoff,
                                  int32_t *__restrict__ rp, int32_t *__restrict__ mid) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
        const int m = block_of(moff, count, g);
        mid[g] = m;
        rp[g] = rps[m][g - moff[m]] + eoff[m];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) rp[n] = eoff[count];
}

// the union's columns: each matrix's shifted by its first vertex
__global__ void union_cols_kernel(int nnz, int count, const int32_t *const *__restrict__ cis,
                                  const int32_t *__restrict__ moff, const int32_t *__restrict__ eoff,
                                  int32_t *__restrict__ ci) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += gridDim.x * blockDim.x) {
        const int m = block_of(eoff, count, e);
        ci[e] = cis[m][e - eoff[m]] + moff[m];
    }
}

// ------------------------------------------------------------ local edges

constexpr int64_t kLocalDeg = 4096;   // edges between vertices whose degree product exceeds this stay untested

// 1 when v is in the sorted list adj[lo .. hi)
__device__ __forceinline__ bool in_sorted(const int32_t *__restrict__ adj, int lo, int hi, int v) {
    const int end = hi;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (adj[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo < end && adj[lo] == v;
}

// flag[k] = 1 when stored entry k = (u, v) is a local edge: deg u * deg v
// above kLocalDeg, or a neighbour a != v of u adjacent to v (a triangle), or
// a neighbour a != v of u adjacent to a neighbour b of v other than u and a
// (a 4-cycle).  sadj holds the adjacency lists sorted by index.
__global__ void local_edge_kernel(int nnz, const int32_t *__restrict__ rowof, const int32_t *__restrict__ ci,
                                  const int32_t *__restrict__ arp, const int32_t *__restrict__ sadj,
                                  int32_t *__restrict__ flag) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += gridDim.x * blockDim.x) {
        const int u = rowof[k], v = ci[k];
        const int u0 = arp[u], u1 = arp[u + 1], v0 = arp[v], v1 = arp[v + 1];
        bool local = static_cast<int64_t>(u1 - u0) * (v1 - v0) > kLocalDeg;
        for (int x = u0; !local && x < u1; ++x) {
            const int a = sadj[x];
            if (a == v) continue;
            if (in_sorted(sadj, v0, v1, a)) {
                local = true;
                break;
            }
            const int a0 = arp[a], a1 = arp[a + 1];
            for (int y = v0; y < v1; ++y) {
                const int b = sadj[y];
                if (b == u || b == a) continue;
                if (in_sorted(sadj, a0, a1, b)) {
                    local = true;
                    break;
                }
            }
        }
        flag[k] = local ? 1 : 0;
    }
}

// the filtered pattern: rp2[i] = fscan[rp[i]], the kept entries in order
__global__ void filter_kernel(int n, int nnz, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                              const int32_t *__restrict__ flag, const int32_t *__restrict__ fscan,
                              int32_t *__restrict__ rp2, int32_t *__restrict__ ci2) {
    const int span = max(n + 1, nnz);
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < span; x += gridDim.x * blockDim.x) {
        if (x <= n) rp2[x] = fscan[rp[x]];
        if (x < nnz && flag[x]) ci2[fscan[x]] = ci[x];
    }
}

// dst[i] = src[idx[i]]
__global__ void row_gather_kernel(int count, const int32_t *__restrict__ idx, const int32_t *__restrict__ src,
                                  int32_t *__restrict__ dst) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) dst[i] = src[idx[i]];
}

// ------------------------------------------------------------ host side


// One pattern (the union of `count` matrices when count > 1, see Blocks) in
// device memory; perms[m] (device array of device pointers) receive the
// orderings, bw0/bw1 (host, count each) the bandwidths.
struct Problem {
    int n, nnz, count;
    const int32_t *rp, *ci;
    Blocks B;
    int32_t *const *perms;
    std::vector<int32_t> moff_h;   // host copy of B.moff
    std::vector<int32_t *> perms_h;
};

// The RCM of P's pattern into P.perms, with its bandwidths and guard per
// matrix; pos_out (device, n, may be null) receives every vertex's position
// in the unreversed order (before the guard).
int rcm_core(const Problem &P, int32_t flags, int64_t *bw0, int64_t *bw1, cudaStream_t st,
             int32_t *pos_out = nullptr) {
    const int n = P.n, nnz = P.nnz, m2 = 2 * P.nnz;
    const int G = kThreads;
    Scratch S;
    Ctl *ctl = S.get<Ctl>(1);
    int32_t *rowof = S.get<int32_t>(nnz), *deg = S.get<int32_t>(n + 1);
    if (S.err() != cudaSuccess) return PARS3_ENOMEM;
    Ctl hc{};
    cudaError_t ce = cudaMemsetAsync(ctl, 0, sizeof(Ctl), st);
    if (ce != cudaSuccess) return cuda_status(ce);

    // validation, then degrees
    validate_kernel<<<grid_for(n, G), G, 0, st>>>(n, P.B, P.rp, P.ci, rowof, deg, &ctl->err);
    int rc = fetch(&hc, ctl, sizeof(Ctl), st);
    if (rc != PARS3_OK) return rc;
    if (hc.err) return PARS3_ENOTSKEW;
    degree_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, P.ci, deg);

    // vertices in (matrix, degree, index) order: stable sorts of 0 .. n-1 by
    // degree, then by matrix
    const int nbits = bits_for(n);
    const int sort_max = std::max(n, m2);
    const int ntiles = (sort_max + kSortTile - 1) / kSortTile;
    uint32_t *ka = S.get<uint32_t>(sort_max), *kb = S.get<uint32_t>(sort_max);
    int32_t *va = S.get<int32_t>(sort_max), *vb = S.get<int32_t>(sort_max);
    int32_t *hist = S.get<int32_t>(256 * static_cast<size_t>(ntiles) + 1);
    int32_t *hoff = S.get<int32_t>(256 * static_cast<size_t>(ntiles) + 1);
    int32_t *sws = S.get<int32_t>(scan_ws_size(std::max(sort_max, 256 * ntiles + 1)));
    int32_t *by_deg = S.get<int32_t>(n), *rank = S.get<int32_t>(n);
    int32_t *arp = S.get<int32_t>(n + 1), *cur = S.get<int32_t>(n), *aun = S.get<int32_t>(m2);
    int32_t *sdeg = S.get<int32_t>(n), *epos = S.get<int32_t>(n + 1), *adj = S.get<int32_t>(m2);
    if (S.err() != cudaSuccess) return PARS3_ENOMEM;
    uint32_t *ko;
    int32_t *vo;
    cudaMemcpyAsync(ka, deg, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st);
    iota_kernel<<<grid_for(n, G), G, 0, st>>>(n, va);
    radix_sort(ka, va, kb, vb, n, nbits, hist, hoff, sws, st, &ko, &vo);
    if (P.B.mid) {
        uint32_t *kx = ko == ka ? kb : ka;
        int32_t *vx = vo == va ? vb : va;
        gather_kernel<<<grid_for(n, G), G, 0, st>>>(n, vo, P.B.mid, reinterpret_cast<int32_t *>(kx));
        uint32_t *k2;
        int32_t *v2;
        radix_sort(kx, vo, ko, vx, n, bits_for(P.count), hist, hoff, sws, st, &k2, &v2);
        vo = v2;
    }
    cudaMemcpyAsync(by_deg, vo, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st);
    rank_kernel<<<grid_for(n, G), G, 0, st>>>(n, by_deg, rank);

    // adjacency lists sorted by the neighbours' rank: the directed edges are
    // listed source by source in rank order, then sorted stably by target
    scan_exclusive(deg, arp, n, sws, st);
    cudaMemsetAsync(cur, 0, sizeof(int32_t) * n, st);
    scatter_adj_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, rowof, P.ci, arp, cur, aun);
    gather_kernel<<<grid_for(n, G), G, 0, st>>>(n, by_deg, deg, sdeg);
    scan_exclusive(sdeg, epos, n, sws, st);
    edges_by_rank_kernel<<<grid_for(static_cast<int64_t>(n) * 32, G), G, 0, st>>>(n, by_deg, arp, aun, epos, ka, va);
    radix_sort(ka, va, kb, vb, m2, nbits, hist, hoff, sws, st, &ko, &vo);
    cudaMemcpyAsync(adj, vo, sizeof(int32_t) * m2, cudaMemcpyDeviceToDevice, st);

    // connected components, their start candidates (in start order) and sizes
    int32_t *parent = S.get<int32_t>(n), *comp = S.get<int32_t>(n), *cmin = S.get<int32_t>(n);
    int32_t *csize = S.get<int32_t>(n), *flag = S.get<int32_t>(n), *sidx = S.get<int32_t>(n + 1);
    if (S.err() != cudaSuccess) return PARS3_ENOMEM;
    iota_kernel<<<grid_for(n, G), G, 0, st>>>(n, parent);
    hook_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, rowof, P.ci, parent, ctl);
    fill_kernel<<<grid_for(n, G), G, 0, st>>>(n, INT_MAX, cmin);
    cudaMemsetAsync(csize, 0, sizeof(int32_t) * n, st);
    comp_kernel<<<grid_for(n, G), G, 0, st>>>(n, parent, rank, comp, cmin, csize);
    start_flag_kernel<<<grid_for(n, G), G, 0, st>>>(n, by_deg, comp, cmin, flag);
    scan_exclusive(flag, sidx, n, sws, st);
    int32_t ncomp = 0;
    cudaMemcpyAsync(&ncomp, sidx + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if ((rc = fetch(&hc, ctl, sizeof(Ctl), st)) != PARS3_OK) return rc;
    if (hc.err & kErrHook) return PARS3_ETIMEOUT;
    if (ncomp < 1 || ncomp > n) return PARS3_ECUDA;
    int32_t *cstart = S.get<int32_t>(ncomp), *csz = S.get<int32_t>(ncomp), *cbase = S.get<int32_t>(ncomp + 1);
    int32_t *cm = S.get<int32_t>(n), *pos = S.get<int32_t>(n), *claim = S.get<int32_t>(n);
    int32_t *cnt = S.get<int32_t>(n), *coff = S.get<int32_t>(n + 1);
    Front *act[2] = {S.get<Front>(ncomp), S.get<Front>(ncomp)};
    int32_t *fpre[2] = {S.get<int32_t>(ncomp + 1), S.get<int32_t>(ncomp + 1)};
    if (S.err() != cudaSuccess) return PARS3_ENOMEM;
    start_list_kernel<<<grid_for(n, G), G, 0, st>>>(n, by_deg, comp, csize, flag, sidx, cstart, csz);
    scan_exclusive(csz, cbase, ncomp, sws, st);
    // components by size: large ones take the grid-wide level steps, the
    // others one block each
    int32_t *bigf = S.get<int32_t>(ncomp), *bigpos = S.get<int32_t>(ncomp + 1);
    int32_t *smallf = S.get<int32_t>(ncomp), *smallpos = S.get<int32_t>(ncomp + 1);
    int32_t *smalllist = S.get<int32_t>(ncomp);
    if (S.err() != cudaSuccess) return PARS3_ENOMEM;
    comp_class_kernel<<<grid_for(ncomp, G), G, 0, st>>>(ncomp, csz, bigf, smallf);
    scan_exclusive(bigf, bigpos, ncomp, sws, st);
    scan_exclusive(smallf, smallpos, ncomp, sws, st);
    compact_list_kernel<<<grid_for(ncomp, G), G, 0, st>>>(ncomp, smallf, smallpos, smalllist);
    int32_t nbig = 0, nsmall = 0;
    cudaMemcpyAsync(&nbig, bigpos + ncomp, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if ((rc = fetch(&nsmall, smallpos + ncomp, sizeof(int32_t), st)) != PARS3_OK) return rc;

    // one breadth-first search of every component from root[c]; with ecc and
    // last set, each component's eccentricity and last level are recorded
    auto search = [&](const int32_t *root, int32_t *ecc, int2 *last) -> int {
        cudaMemsetAsync(pos, 0xff, sizeof(int32_t) * n, st);
        fill_kernel<<<grid_for(n, G), G, 0, st>>>(n, INT_MAX, claim);
        bfs_init_kernel<<<grid_for(ncomp, G), G, 0, st>>>(ncomp, root, cbase, csz, bigpos, cm, pos, act[0], fpre[0],
                                                          ctl);
        if (ecc) single_comp_kernel<<<grid_for(ncomp, G), G, 0, st>>>(ncomp, csz, cbase, ecc, last);
        if (nsmall > 0)
            component_search_kernel<<<std::min(nsmall, 2 * sm_count()), kScanThreads, 0, st>>>(
                nsmall, smalllist, cbase, csz, arp, adj, cm, pos, claim, cnt, coff, ecc, last);
        if (nbig == 0) return cuda_status(cudaGetLastError());
        const int wg = 4 * sm_count();   // warp-per-vertex kernels: grid-stride over the level
        int b = 0;
        for (int64_t steps = 0;; steps += kLevelsPerCheck) {
            for (int l = 0; l < kLevelsPerCheck; ++l) {
                claim_kernel<<<wg, G, 0, st>>>(ctl, b, act[b], fpre[b], cm, arp, adj, pos, claim);
                count_kernel<<<wg, G, 0, st>>>(ctl, b, act[b], fpre[b], cm, arp, adj, claim, cnt);
                plan_kernel<<<1, kScanThreads, 0, st>>>(ctl, b, act[b], fpre[b], cnt, coff, act[b ^ 1], fpre[b ^ 1],
                                                        ecc, last);
                write_kernel<<<wg, G, 0, st>>>(ctl, b, act[b], fpre[b], coff, cm, arp, adj, claim, pos);
                b ^= 1;
            }
            const int r2 = fetch(&hc, ctl, sizeof(Ctl), st);
            if (r2 != PARS3_OK) return r2;
            if (hc.nact[b] == 0) return PARS3_OK;
            if (steps > static_cast<int64_t>(n) + kLevelsPerCheck) return PARS3_ECUDA;   // more levels than vertices
        }
    };

    const int32_t *root = cstart;
    if (flags & PARS3_RCM_PERIPHERAL) {
        // George-Liu pseudo-peripheral starts for all components at once
        int32_t *r = S.get<int32_t>(ncomp), *e = S.get<int32_t>(ncomp), *x = S.get<int32_t>(ncomp);
        int32_t *ex = S.get<int32_t>(ncomp), *y = S.get<int32_t>(ncomp), *active = S.get<int32_t>(ncomp);
        int32_t *sel = S.get<int32_t>(ncomp);
        int2 *last = S.get<int2>(ncomp);
        if (S.err() != cudaSuccess) return PARS3_ENOMEM;
        const int cg = grid_for(static_cast<int64_t>(ncomp) * 32, G);
        cudaMemcpyAsync(r, cstart, sizeof(int32_t) * ncomp, cudaMemcpyDeviceToDevice, st);
        if ((rc = search(r, e, last)) != PARS3_OK) return rc;
        last_min_kernel<<<cg, G, 0, st>>>(ncomp, last, cm, rank, by_deg, x);
        fill_kernel<<<grid_for(ncomp, G), G, 0, st>>>(ncomp, 1, active);
        for (int round = 0;; ++round) {
            select_kernel<<<grid_for(ncomp, G), G, 0, st>>>(ncomp, active, r, x, sel);
            if ((rc = search(sel, ex, last)) != PARS3_OK) return rc;
            last_min_kernel<<<cg, G, 0, st>>>(ncomp, last, cm, rank, by_deg, y);
            cudaMemsetAsync(&ctl->active, 0, sizeof(int), st);
            peripheral_step_kernel<<<grid_for(ncomp, G), G, 0, st>>>(ncomp, active, r, e, x, ex, y, ctl);
            if ((rc = fetch(&hc, ctl, sizeof(Ctl), st)) != PARS3_OK) return rc;
            if (hc.active == 0) break;
            if (round > n) return PARS3_ECUDA;   // each round raises an eccentricity, which is below n
        }
        root = r;
    }
    if ((rc = search(root, nullptr, nullptr)) != PARS3_OK) return rc;

    // reverse per matrix, bandwidths, guard
    unsigned long long *bw = S.get<unsigned long long>(2 * static_cast<size_t>(P.count));
    if (S.err() != cudaSuccess) return PARS3_ENOMEM;
    cudaMemsetAsync(bw, 0, sizeof(unsigned long long) * 2 * P.count, st);
    perm_kernel<<<grid_for(n, G), G, 0, st>>>(n, P.B, cm, pos, P.perms, ctl);
    bandwidth_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, P.B.mid, rowof, P.ci, pos, bw);
    if (pos_out) cudaMemcpyAsync(pos_out, pos, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st);
    std::vector<unsigned long long> bw_h(2 * static_cast<size_t>(P.count));
    cudaMemcpyAsync(bw_h.data(), bw, sizeof(unsigned long long) * bw_h.size(), cudaMemcpyDeviceToHost, st);
    if ((rc = fetch(&hc, ctl, sizeof(Ctl), st)) != PARS3_OK) return rc;
    if (hc.err & kErrPlaced) return PARS3_ECUDA;
    bool reset = false;
    for (int m = 0; m < P.count; ++m) {
        int64_t b0 = static_cast<int64_t>(bw_h[2 * m]), b1 = static_cast<int64_t>(bw_h[2 * m + 1]);
        const int nm = P.moff_h[m + 1] - P.moff_h[m];
        if ((flags & PARS3_RCM_GUARD) && b1 > b0) {
            if (nm > 0) iota_kernel<<<grid_for(nm, G), G, 0, st>>>(nm, P.perms_h[m]);
            b1 = b0;
            reset = true;
        }
        if (bw0) bw0[m] = b0;
        if (bw1) bw1[m] = b1;
    }
    if (reset && (ce = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_status(ce);
    return cuda_status(cudaGetLastError());
}

int check_flags(int32_t flags) {
    if (flags & ~(PARS3_RCM_GUARD | PARS3_RCM_PERIPHERAL | PARS3_RCM_LOCAL)) return PARS3_EINVAL;
    return PARS3_OK;
}

// The local-edge RCM (PARS3_RCM_LOCAL): the RCM, with the caller's start
// rule, of the pattern restricted to its local edges -- those on a triangle
// or a 4-cycle, or between two vertices whose degree product exceeds
// kLocalDeg (kept untested) -- so that random long-range edges do not steer
// the order; they stay in the matrix, and the bandwidths and the guard
// count every stored entry.
int rcm_local(const Problem &P, int32_t flags, int64_t *bw0, int64_t *bw1, cudaStream_t st) {
    const int n = P.n, nnz = P.nnz, m2 = 2 * P.nnz;
    const int G = kThreads;
    Scratch S;
    int *err = S.get<int>(1);
    int32_t *rowof = S.get<int32_t>(nnz), *deg = S.get<int32_t>(n + 1), *arp = S.get<int32_t>(n + 1);
    int32_t *cur = S.get<int32_t>(n), *aun = S.get<int32_t>(m2), *iota = S.get<int32_t>(n);
    uint32_t *ka = S.get<uint32_t>(m2), *kb = S.get<uint32_t>(m2);
    int32_t *va = S.get<int32_t>(m2), *vb = S.get<int32_t>(m2);
    const int ntiles = (m2 + kSortTile - 1) / kSortTile;
    int32_t *hist = S.get<int32_t>(256 * static_cast<size_t>(ntiles) + 1);
    int32_t *hoff = S.get<int32_t>(256 * static_cast<size_t>(ntiles) + 1);
    int32_t *sws = S.get<int32_t>(scan_ws_size(std::max(std::max(n, m2), 256 * ntiles + 1)));
    int32_t *flag = S.get<int32_t>(nnz), *fscan = S.get<int32_t>(static_cast<size_t>(nnz) + 1);
    int32_t *rp2 = S.get<int32_t>(n + 1), *ci2 = S.get<int32_t>(nnz), *pos = S.get<int32_t>(n);
    int32_t *eoff2 = S.get<int32_t>(static_cast<size_t>(P.count) + 1);
    unsigned long long *bw = S.get<unsigned long long>(2 * static_cast<size_t>(P.count));
    if (S.err() != cudaSuccess) return PARS3_ENOMEM;
    cudaMemsetAsync(err, 0, sizeof(int), st);
    validate_kernel<<<grid_for(n, G), G, 0, st>>>(n, P.B, P.rp, P.ci, rowof, deg, err);
    int herr = 0;
    int rc = fetch(&herr, err, sizeof(int), st);
    if (rc != PARS3_OK) return rc;
    if (herr) return PARS3_ENOTSKEW;
    degree_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, P.ci, deg);
    // adjacency lists sorted by index: the directed edges listed source by
    // source in index order, then sorted stably by target
    scan_exclusive(deg, arp, n, sws, st);
    cudaMemsetAsync(cur, 0, sizeof(int32_t) * n, st);
    scatter_adj_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, rowof, P.ci, arp, cur, aun);
    iota_kernel<<<grid_for(n, G), G, 0, st>>>(n, iota);
    edges_by_rank_kernel<<<grid_for(static_cast<int64_t>(n) * 32, G), G, 0, st>>>(n, iota, arp, aun, arp, ka, va);
    uint32_t *ko;
    int32_t *sadj;
    radix_sort(ka, va, kb, vb, m2, bits_for(n), hist, hoff, sws, st, &ko, &sadj);
    // the local entries, kept in their order: the filtered pattern
    local_edge_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, rowof, P.ci, arp, sadj, flag);
    scan_exclusive(flag, fscan, nnz, sws, st);
    filter_kernel<<<grid_for(std::max(n + 1, nnz), G), G, 0, st>>>(n, nnz, P.rp, P.ci, flag, fscan, rp2, ci2);
    row_gather_kernel<<<grid_for(P.count + 1, G), G, 0, st>>>(P.count + 1, P.B.moff, rp2, eoff2);
    int32_t nnz2 = 0;
    if ((rc = fetch(&nnz2, fscan + nnz, sizeof(int32_t), st)) != PARS3_OK) return rc;
    Problem P2{n, nnz2, P.count, rp2, ci2, Blocks{P.B.mid, P.B.moff, eoff2}, P.perms, P.moff_h, P.perms_h};
    if ((rc = rcm_core(P2, flags & PARS3_RCM_PERIPHERAL, nullptr, nullptr, st, pos)) != PARS3_OK) return rc;
    // bandwidths over every stored entry, and the guard
    cudaMemsetAsync(bw, 0, sizeof(unsigned long long) * 2 * P.count, st);
    bandwidth_kernel<<<grid_for(nnz, G), G, 0, st>>>(nnz, P.B.mid, rowof, P.ci, pos, bw);
    std::vector<unsigned long long> bw_h(2 * static_cast<size_t>(P.count));
    if ((rc = fetch(bw_h.data(), bw, sizeof(unsigned long long) * bw_h.size(), st)) != PARS3_OK) return rc;
    bool reset = false;
    for (int m = 0; m < P.count; ++m) {
        int64_t b0 = static_cast<int64_t>(bw_h[2 * m]), b1 = static_cast<int64_t>(bw_h[2 * m + 1]);
        const int nm = P.moff_h[m + 1] - P.moff_h[m];
        if ((flags & PARS3_RCM_GUARD) && b1 > b0) {
            if (nm > 0) iota_kernel<<<grid_for(nm, G), G, 0, st>>>(nm, P.perms_h[m]);
            b1 = b0;
            reset = true;
        }
        if (bw0) bw0[m] = b0;
        if (bw1) bw1[m] = b1;
    }
    if (reset) {
        const cudaError_t ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) return cuda_status(ce);
    }
    return cuda_status(cudaGetLastError());
}

int rcm_entry(const Problem &P, int32_t flags, int64_t *bw0, int64_t *bw1, cudaStream_t st) {
    return (flags & PARS3_RCM_LOCAL) ? rcm_local(P, flags, bw0, bw1, st) : rcm_core(P, flags, bw0, bw1, st);
}

int reorder_device(int32_t n, const int32_t *rp, const int32_t *ci, int32_t flags, int32_t *perm,
                   int64_t *bw_before, int64_t *bw_after, cudaStream_t st) {
    if (n < 0) return PARS3_EINVAL;
    int rc = check_flags(flags);
    if (rc != PARS3_OK) return rc;
    if (bw_before) *bw_before = 0;
    if (bw_after) *bw_after = 0;
    if (n == 0) return PARS3_OK;
    if (!rp || !perm) return PARS3_EINVAL;
    int32_t nnz = 0;
    if ((rc = fetch(&nnz, rp + n, sizeof(int32_t), st)) != PARS3_OK) return rc;
    if (nnz < 0) return PARS3_ENOTSKEW;
    if (nnz > 0 && !ci) return PARS3_EINVAL;
    if (nnz >= (1 << 30)) return PARS3_EUNSUPPORTED;   // 2 nnz directed edges are indexed by int32
    Scratch S;
    int32_t *off = S.get<int32_t>(4);
    int32_t **perms = S.get<int32_t *>(1);
    if (S.err() != cudaSuccess) return PARS3_ENOMEM;
    const int32_t off_h[4] = {0, n, 0, nnz};   // moff = {0, n}, eoff = {0, nnz}
    cudaError_t ce = cudaMemcpyAsync(off, off_h, sizeof(off_h), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(perms, &perm, sizeof(int32_t *), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);   // the host sources above are stack memory
    if (ce != cudaSuccess) return cuda_status(ce);
    Problem P{n, nnz, 1, rp, ci, Blocks{nullptr, off, off + 2}, perms, {0, n}, {perm}};
    return rcm_entry(P, flags, bw_before, bw_after, st);
}

int reorder_device_batched(int32_t count, const int32_t *ns, const int32_t *const *rps,
                           const int32_t *const *cis, int32_t flags, int32_t *const *perms, int64_t *bw_before,
                           int64_t *bw_after, cudaStream_t st) {
    if (count < 0 || (count > 0 && (!ns || !rps || !cis || !perms))) return PARS3_EINVAL;
    int rc = check_flags(flags);
    if (rc != PARS3_OK) return rc;
    if (count == 0) return PARS3_OK;
    std::vector<int32_t> moff(count + 1, 0), eoff(count + 1, 0);
    for (int m = 0; m < count; ++m) {
        if (ns[m] < 0 || !rps[m] || (ns[m] > 0 && !perms[m])) return PARS3_EINVAL;
        if (bw_before) bw_before[m] = 0;
        if (bw_after) bw_after[m] = 0;
        if (static_cast<int64_t>(moff[m]) + ns[m] > INT32_MAX) return PARS3_EUNSUPPORTED;
        moff[m + 1] = moff[m] + ns[m];
    }
    Scratch S;
    int32_t *ns_d = S.get<int32_t>(count), *nz_d = S.get<int32_t>(count);
    const int32_t **rps_d = S.get<const int32_t *>(count), **cis_d = S.get<const int32_t *>(count);
    int32_t **perms_d = S.get<int32_t *>(count);
    int32_t *off_d = S.get<int32_t>(2 * (static_cast<size_t>(count) + 1));
    if (S.err() != cudaSuccess) return PARS3_ENOMEM;
    cudaError_t ce = cudaMemcpyAsync(ns_d, ns, sizeof(int32_t) * count, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(rps_d, rps, sizeof(int32_t *) * count, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(cis_d, cis, sizeof(int32_t *) * count, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(perms_d, perms, sizeof(int32_t *) * count, cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) return cuda_status(ce);
    nnz_kernel<<<grid_for(count, kThreads), kThreads, 0, st>>>(count, rps_d, ns_d, nz_d);
    std::vector<int32_t> nz(count);
    if ((rc = fetch(nz.data(), nz_d, sizeof(int32_t) * count, st)) != PARS3_OK) return rc;
    for (int m = 0; m < count; ++m) {
        if (nz[m] < 0) return PARS3_ENOTSKEW;
        if (nz[m] > 0 && !cis[m]) return PARS3_EINVAL;
        if (static_cast<int64_t>(eoff[m]) + nz[m] >= (1 << 30)) return PARS3_EUNSUPPORTED;
        eoff[m + 1] = eoff[m] + nz[m];
    }
    const int n = moff[count], nnz = eoff[count];
    if (n == 0) return PARS3_OK;
    int32_t *rp = S.get<int32_t>(n + 1), *ci = S.get<int32_t>(nnz), *mid = S.get<int32_t>(n);
    if (S.err() != cudaSuccess) return PARS3_ENOMEM;
    int32_t *moff_d = off_d, *eoff_d = off_d + count + 1;
    ce = cudaMemcpyAsync(moff_d, moff.data(), sizeof(int32_t) * (count + 1), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(eoff_d, eoff.data(), sizeof(int32_t) * (count + 1), cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) return cuda_status(ce);
    union_rows_kernel<<<grid_for(n, kThreads), kThreads, 0, st>>>(n, count, rps_d, moff_d, eoff_d, rp, mid);
    union_cols_kernel<<<grid_for(nnz, kThreads), kThreads, 0, st>>>(nnz, count, cis_d, moff_d, eoff_d, ci);
    Problem P{n, nnz, count, rp, ci, Blocks{mid, moff_d, eoff_d}, perms_d, moff,
              std::vector<int32_t *>(perms, perms + count)};
    rc = rcm_entry(P, flags, bw_before, bw_after, st);
    // the host vectors copied from above must outlive the copies
    const cudaError_t se = cudaStreamSynchronize(st);
    return rc != PARS3_OK ? rc : cuda_status(se);
}

}  // namespace
}  // namespace pars3

extern "C" int pars3_reorder_device(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t flags,
                                    int32_t *perm_out, int64_t *bw_before, int64_t *bw_after, void *stream) {
    return pars3::reorder_device(n, rowptr, col, flags, perm_out, bw_before, bw_after,
                                 static_cast<cudaStream_t>(stream));
}

extern "C" int pars3_reorder_device_batched(int32_t count, const int32_t *n, const int32_t *const *rowptr,
                                            const int32_t *const *col, int32_t flags, int32_t *const *perm_out,
                                            int64_t *bw_before, int64_t *bw_after, void *stream) {
    return pars3::reorder_device_batched(count, n, rowptr, col, flags, perm_out, bw_before, bw_after,
                                         static_cast<cudaStream_t>(stream));
}
