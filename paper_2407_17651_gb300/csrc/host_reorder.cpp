// host_reorder.cpp -- input validation and the deterministic reverse
// Cuthill-McKee ordering (Sec. 1 and Sec. 3.1.2 of the paper: RCM squeezes
// the skew matrix into a band before the split; its cost is linear in the
// number of nonzeros).  Host code, linear time:
//   * adjacency lists are produced directly in (degree, index) order by
//     visiting the vertices in that order and appending each one to the
//     lists of its neighbours, so the breadth-first search only filters
//     out visited vertices and never sorts;
//   * start vertices are the unvisited vertex of least (degree, index),
//     found with a pointer into the same (degree, index) order.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

namespace pars3 {

int validate_lower(int32_t n, const int32_t *rowptr, const int32_t *col) {
    if (n < 0) return PARS3_EINVAL;
    if (!rowptr || (n > 0 && rowptr[n] > 0 && !col)) return PARS3_EINVAL;
    if (rowptr[0] != 0) return PARS3_ENOTSKEW;
    for (int32_t i = 0; i < n; ++i) {
        int32_t a = rowptr[i], b = rowptr[i + 1];
        if (b < a) return PARS3_ENOTSKEW;
        int32_t prev = -1;
        for (int32_t k = a; k < b; ++k) {
            int32_t j = col[k];
            if (j <= prev || j >= i || j < 0) return PARS3_ENOTSKEW;
            prev = j;
        }
    }
    return PARS3_OK;
}

// max |pinv[i] - pinv[j]| over stored (i, j); pinv == nullptr is the identity
int64_t bandwidth(int32_t n, const int32_t *rowptr, const int32_t *col, const int32_t *pinv) {
    int64_t bw = 0;
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            int64_t a = pinv ? pinv[i] : i;
            int64_t b = pinv ? pinv[col[k]] : col[k];
            int64_t d = a > b ? a - b : b - a;
            if (d > bw) bw = d;
        }
    }
    return bw;
}

// Level structure rooted at r: eccentricity of r, and in *last_min the vertex
// of the last level with the smallest (degree, index).  dist is -1 on entry
// and on exit; queue holds the component in breadth-first order.
static int32_t last_level(const std::vector<int64_t> &aptr, const std::vector<int32_t> &adj,
                          const std::vector<int32_t> &deg, int32_t r, std::vector<int32_t> &dist,
                          std::vector<int32_t> &queue, int32_t *last_min) {
    int32_t head = 0, tail = 0;
    dist[r] = 0;
    queue[tail++] = r;
    while (head < tail) {
        const int32_t v = queue[head++];
        for (int64_t k = aptr[v]; k < aptr[v + 1]; ++k) {
            const int32_t u = adj[k];
            if (dist[u] < 0) {
                dist[u] = dist[v] + 1;
                queue[tail++] = u;
            }
        }
    }
    const int32_t ecc = dist[queue[tail - 1]];
    int32_t best = -1;
    for (int32_t q = tail - 1; q >= 0 && dist[queue[q]] == ecc; --q) {
        const int32_t v = queue[q];
        if (best < 0 || deg[v] < deg[best] || (deg[v] == deg[best] && v < best)) best = v;
    }
    for (int32_t q = 0; q < tail; ++q) dist[queue[q]] = -1;
    *last_min = best;
    return ecc;
}

// George-Liu: from r, move to the last level's smallest (degree, index)
// vertex while that is strictly more eccentric.
static int32_t pseudo_peripheral(const std::vector<int64_t> &aptr, const std::vector<int32_t> &adj,
                                 const std::vector<int32_t> &deg, int32_t r, std::vector<int32_t> &dist,
                                 std::vector<int32_t> &queue) {
    int32_t x;
    int32_t e = last_level(aptr, adj, deg, r, dist, queue, &x);
    for (;;) {
        int32_t y;
        const int32_t ex = last_level(aptr, adj, deg, x, dist, queue, &y);
        if (ex <= e) return r;
        r = x;
        e = ex;
        x = y;
    }
}

static int rcm_core(int32_t n, const int32_t *rowptr, const int32_t *col, bool peripheral, int32_t *perm) {
    const int64_t nnz = rowptr[n];
    std::vector<int32_t> deg(n, 0);
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            ++deg[i];
            ++deg[col[k]];
        }
    }
    // vertices in (degree, index) order: counting sort by degree, stable in index
    int32_t maxdeg = 0;
    for (int32_t i = 0; i < n; ++i) maxdeg = std::max(maxdeg, deg[i]);
    std::vector<int64_t> bucket(static_cast<size_t>(maxdeg) + 2, 0);
    for (int32_t i = 0; i < n; ++i) ++bucket[deg[i] + 1];
    for (int32_t d = 0; d <= maxdeg; ++d) bucket[d + 1] += bucket[d];
    std::vector<int32_t> order(n);
    for (int32_t i = 0; i < n; ++i) order[bucket[deg[i]]++] = i;

    // adjacency with every list in (degree, index) order
    std::vector<int64_t> aptr(static_cast<size_t>(n) + 1, 0);
    for (int32_t i = 0; i < n; ++i) aptr[i + 1] = aptr[i] + deg[i];
    // lower neighbours of u are col[rowptr[u]..]; upper neighbours are the rows
    // that store u: build the transpose pattern once
    std::vector<int64_t> tptr(static_cast<size_t>(n) + 1, 0);
    for (int64_t k = 0; k < nnz; ++k) ++tptr[col[k] + 1];
    for (int32_t i = 0; i < n; ++i) tptr[i + 1] += tptr[i];
    std::vector<int32_t> trow(static_cast<size_t>(nnz));
    {
        std::vector<int64_t> fill(tptr.begin(), tptr.end() - 1);
        for (int32_t i = 0; i < n; ++i)
            for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) trow[fill[col[k]]++] = i;
    }
    std::vector<int32_t> adj(static_cast<size_t>(2 * nnz));
    {
        std::vector<int64_t> fill(aptr.begin(), aptr.end() - 1);
        for (int32_t q = 0; q < n; ++q) {
            int32_t u = order[q];
            for (int32_t k = rowptr[u]; k < rowptr[u + 1]; ++k) adj[fill[col[k]]++] = u;
            for (int64_t k = tptr[u]; k < tptr[u + 1]; ++k) adj[fill[trow[k]]++] = u;
        }
    }
    std::vector<uint8_t> seen(n, 0);
    std::vector<int32_t> cm(n);
    std::vector<int32_t> dist, queue;
    if (peripheral) {
        dist.assign(n, -1);
        queue.resize(n);
    }
    int32_t count = 0, head = 0, next_start = 0;
    while (count < n) {
        while (seen[order[next_start]]) ++next_start;
        int32_t s = order[next_start];
        if (peripheral && deg[s] > 0) s = pseudo_peripheral(aptr, adj, deg, s, dist, queue);
        seen[s] = 1;
        cm[count++] = s;
        while (head < count) {
            int32_t v = cm[head++];
            for (int64_t k = aptr[v]; k < aptr[v + 1]; ++k) {
                int32_t u = adj[k];
                if (!seen[u]) {
                    seen[u] = 1;
                    cm[count++] = u;
                }
            }
        }
    }
    for (int32_t k = 0; k < n; ++k) perm[k] = cm[n - 1 - k];
    return PARS3_OK;
}

}  // namespace pars3

// The local edges of the pattern (PARS3_RCM_LOCAL): a stored {u, v} is local
// when it lies on a triangle or a 4-cycle, or when deg(u) deg(v) exceeds
// kLocalDeg (then it is kept untested).  Output: strict-lower CSR of the local
// edges, in the input's order.  Neighbour lists are index-sorted for free:
// the lower neighbours of u (its stored columns) precede its upper ones (the
// rows that store u, in increasing order).
constexpr int64_t kLocalDeg = 4096;
static void local_edges(int32_t n, const int32_t *rowptr, const int32_t *col, std::vector<int32_t> &rp2,
                        std::vector<int32_t> &ci2) {
    const int64_t nnz = rowptr[n];
    std::vector<int64_t> tptr(static_cast<size_t>(n) + 1, 0);
    for (int64_t k = 0; k < nnz; ++k) ++tptr[col[k] + 1];
    for (int32_t i = 0; i < n; ++i) tptr[i + 1] += tptr[i];
    std::vector<int32_t> trow(static_cast<size_t>(nnz));
    {
        std::vector<int64_t> fill(tptr.begin(), tptr.end() - 1);
        for (int32_t i = 0; i < n; ++i)
            for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) trow[fill[col[k]]++] = i;
    }
    std::vector<int64_t> aptr(static_cast<size_t>(n) + 1, 0);
    for (int32_t i = 0; i < n; ++i)
        aptr[i + 1] = aptr[i] + (rowptr[i + 1] - rowptr[i]) + (tptr[i + 1] - tptr[i]);
    std::vector<int32_t> adj(static_cast<size_t>(2 * nnz));
    for (int32_t i = 0; i < n; ++i) {
        int64_t q = aptr[i];
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) adj[q++] = col[k];
        for (int64_t k = tptr[i]; k < tptr[i + 1]; ++k) adj[q++] = trow[k];
    }
    auto has = [&](int32_t a, int32_t b) {
        return std::binary_search(adj.begin() + aptr[a], adj.begin() + aptr[a + 1], b);
    };
    rp2.assign(static_cast<size_t>(n) + 1, 0);
    ci2.clear();
    for (int32_t u = 0; u < n; ++u) {
        for (int32_t k = rowptr[u]; k < rowptr[u + 1]; ++k) {
            const int32_t v = col[k];
            bool local = (aptr[u + 1] - aptr[u]) * (aptr[v + 1] - aptr[v]) > kLocalDeg;
            for (int64_t x = aptr[u]; !local && x < aptr[u + 1]; ++x) {   // triangles
                const int32_t a = adj[x];
                local = a != v && has(v, a);
            }
            for (int64_t x = aptr[u]; !local && x < aptr[u + 1]; ++x) {   // 4-cycles u-a-b-v
                const int32_t a = adj[x];
                if (a == v) continue;
                for (int64_t y = aptr[v]; y < aptr[v + 1]; ++y) {
                    const int32_t b = adj[y];
                    if (b != u && b != a && has(a, b)) {
                        local = true;
                        break;
                    }
                }
            }
            if (local) ci2.push_back(v);
        }
        rp2[u + 1] = static_cast<int32_t>(ci2.size());
    }
}

extern "C" int pars3_reorder(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t flags,
                             int32_t *perm_out, int64_t *bw_before, int64_t *bw_after) {
    using namespace pars3;
    if (n < 0 || !rowptr || !perm_out) return PARS3_EINVAL;
    int rc = validate_lower(n, rowptr, col);
    if (rc != PARS3_OK) return rc;
    try {
        if (flags & ~(PARS3_RCM_GUARD | PARS3_RCM_PERIPHERAL | PARS3_RCM_LOCAL)) return PARS3_EINVAL;
        if (flags & PARS3_RCM_LOCAL) {
            std::vector<int32_t> rp2, ci2;
            local_edges(n, rowptr, col, rp2, ci2);
            rc = rcm_core(n, rp2.data(), ci2.data(), (flags & PARS3_RCM_PERIPHERAL) != 0, perm_out);
        } else {
            rc = rcm_core(n, rowptr, col, (flags & PARS3_RCM_PERIPHERAL) != 0, perm_out);
        }
        if (rc != PARS3_OK) return rc;
        std::vector<int32_t> pinv(n);
        for (int32_t k = 0; k < n; ++k) pinv[perm_out[k]] = k;
        int64_t b0 = bandwidth(n, rowptr, col, nullptr);
        int64_t b1 = bandwidth(n, rowptr, col, pinv.data());
        if ((flags & PARS3_RCM_GUARD) && b1 > b0) {
            for (int32_t k = 0; k < n; ++k) perm_out[k] = k;
            b1 = b0;
        }
        if (bw_before) *bw_before = b0;
        if (bw_after) *bw_after = b1;
    } catch (const std::bad_alloc &) {
        return PARS3_ENOMEM;
    }
    return PARS3_OK;
}
