/*
 * oracle.c -- plain, slow, obviously correct FP64 CPU oracle for the PARS3
 * hot path (Yildirim & Manguoglu, "PARS3: Parallel Sparse Skew-Symmetric
 * Matrix-Vector Multiplication with Reverse Cuthill-McKee Reordering").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file.  It shares no code,
 * header, table or helper with the CUDA library; the product path never
 * calls it.
 *
 * Everything here is single-threaded and written for clarity, not speed.
 * Inputs are the strict lower triangle L of S = L - L^T in CSR form (the
 * half storage of Sec. 3): row pointers rp[n+1], sorted unique column
 * indices ci[nnz] with ci < row, values v[nnz].  All arithmetic is FP64.
 *
 * The mirror sign m is -1 for the skew-symmetric S = L - L^T of the paper
 * and +1 for the symmetric S = L + L^T, to which the paper says the same
 * method applies (abstract; Sec. 5): the stored l_ij acts as s_ij = l_ij
 * and s_ji = m l_ij.
 *
 * Functions:
 *   orc_validate     input checks (strict lower, sorted, unique, in range)
 *   orc_full_csr     full storage of S = L + m L^T         (Sec. 1, Eq. 1)
 *   orc_spmv_full    y = (alpha I + S) x by plain row sums   (Sec. 1)
 *   orc_spmv_sss     the serial SSS skew SpMV baseline       (Sec. 3.1.1)
 *   orc_rcm          reverse Cuthill-McKee ordering          (Sec. 1, 3.1.2),
 *                    optionally from George-Liu pseudo-peripheral starts
 *   orc_bandwidth    max |p^-1(i) - p^-1(j)| over stored pairs (Table 1)
 *   orc_split        3-way band split, canonical form        (Sec. 3.1.2)
 *   orc_auto_cut     default cut point W (and tile T)        (Sec. 3.1.2, Fig. 8)
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOTSKEW -2
#define ORC_ENOMEM -3

/* ------------------------------------------------------------------------ */
/* input validation                                                           */
/* ------------------------------------------------------------------------ */

/* Returns ORC_OK when rp/ci describe a strict lower triangle with sorted,
 * unique, in-range column indices (the SSS half storage of Sec. 3). */
int orc_validate(int32_t n, const int32_t *rp, const int32_t *ci)
{
    if (n < 0) return ORC_EINVAL;
    if (rp[0] != 0) return ORC_EINVAL;
    for (int32_t i = 0; i < n; i++) {
        if (rp[i + 1] < rp[i]) return ORC_EINVAL;
        for (int32_t k = rp[i]; k < rp[i + 1]; k++) {
            if (ci[k] < 0 || ci[k] >= i) return ORC_ENOTSKEW;
            if (k > rp[i] && ci[k] <= ci[k - 1]) return ORC_ENOTSKEW;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* O1: the operator y = (alpha I + S) x                                       */
/* ------------------------------------------------------------------------ */

/* Full-storage CSR of S = L - L^T (Eq. 1: A = -A^T; Sec. 1: CRS stores every
 * nonzero).  Row i holds s_ij = l_ij for j < i and s_ij = -l_ji for j > i,
 * columns ascending.  frp has n+1 entries, fci/fv have 2*nnz entries. */
int orc_full_csr(int32_t n, const int32_t *rp, const int32_t *ci, const double *v, double mirror,
                 int64_t *frp, int32_t *fci, double *fv)
{
    int64_t *fill = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!fill) return ORC_ENOMEM;
    /* count: each stored (i, j) appears in row i and in row j */
    for (int64_t i = 0; i <= n; i++) frp[i] = 0;
    for (int32_t i = 0; i < n; i++)
        for (int32_t k = rp[i]; k < rp[i + 1]; k++) {
            frp[i + 1]++;
            frp[ci[k] + 1]++;
        }
    for (int32_t i = 0; i < n; i++) frp[i + 1] += frp[i];
    /* lower part of row i first (columns < i, ascending) */
    for (int32_t i = 0; i < n; i++) {
        fill[i] = frp[i];
        for (int32_t k = rp[i]; k < rp[i + 1]; k++) {
            fci[fill[i]] = ci[k];
            fv[fill[i]] = v[k];
            fill[i]++;
        }
    }
    /* then the mirrored upper part: row j receives (j, i, m l_ij); visiting i
     * in increasing order keeps the columns of row j ascending */
    for (int32_t i = 0; i < n; i++)
        for (int32_t k = rp[i]; k < rp[i + 1]; k++) {
            int32_t j = ci[k];
            fci[fill[j]] = i;
            fv[fill[j]] = mirror * v[k];
            fill[j]++;
        }
    free(fill);
    return ORC_OK;
}

/* y_i = alpha x_i + sum_j s_ij x_j, one row at a time (the plain definition
 * of the shifted skew-symmetric operator A = alpha I + S, Sec. 1). */
void orc_spmv_full(int32_t n, double alpha, const int64_t *frp, const int32_t *fci,
                   const double *fv, const double *x, double *y)
{
    for (int32_t i = 0; i < n; i++) {
        double s = alpha * x[i];
        for (int64_t k = frp[i]; k < frp[i + 1]; k++) s += fv[k] * x[fci[k]];
        y[i] = s;
    }
}

/* Same operator applied to k right-hand sides stored row-major (X[i*k + c]). */
void orc_spmm_full(int32_t n, int32_t k, double alpha, const int64_t *frp, const int32_t *fci,
                   const double *fv, const double *X, double *Y)
{
    for (int32_t i = 0; i < n; i++)
        for (int32_t c = 0; c < k; c++) {
            double s = alpha * X[(int64_t)i * k + c];
            for (int64_t q = frp[i]; q < frp[i + 1]; q++)
                s += fv[q] * X[(int64_t)fci[q] * k + c];
            Y[(int64_t)i * k + c] = s;
        }
}

/* The paper's serial baseline (Sec. 3.1.1, adapted to skew symmetry, with the
 * pair update of Eqs. 2-6): every stored l_ij is read once and used twice,
 * y_i += l_ij x_j and y_j += (-l_ij) x_i. */
void orc_spmv_sss(int32_t n, double alpha, double mirror, const int32_t *rp, const int32_t *ci,
                  const double *v, const double *x, double *y)
{
    for (int32_t i = 0; i < n; i++) y[i] = alpha * x[i];
    for (int32_t i = 0; i < n; i++)
        for (int32_t k = rp[i]; k < rp[i + 1]; k++) {
            int32_t j = ci[k];
            double a = v[k];
            y[i] += a * x[j];          /* Eq. 3 and Eq. 5 */
            y[j] += (mirror * a) * x[i];   /* Eq. 2, Eq. 4 and Eq. 6 (m = -1) */
        }
}

/* ------------------------------------------------------------------------ */
/* O2: reverse Cuthill-McKee (Sec. 1 and Sec. 3.1.2; tie rule: degree, then   */
/* index; start vertex: unvisited vertex of minimum degree, then index)       */
/* ------------------------------------------------------------------------ */

static const int32_t *g_deg; /* comparator context (the oracle is single-threaded) */

static int cmp_deg_idx(const void *pa, const void *pb)
{
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    if (g_deg[a] != g_deg[b]) return g_deg[a] < g_deg[b] ? -1 : 1;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* Bandwidth of the ordering perm (new -> old): the largest |p^-1(i) - p^-1(j)|
 * over stored pairs; 0 without nonzeros.  perm == NULL means identity. */
int64_t orc_bandwidth(int32_t n, const int32_t *rp, const int32_t *ci, const int32_t *perm)
{
    int32_t *pinv = NULL;
    if (perm) {
        pinv = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        for (int32_t k = 0; k < n; k++) pinv[perm[k]] = k;
    }
    int64_t bw = 0;
    for (int32_t i = 0; i < n; i++)
        for (int32_t k = rp[i]; k < rp[i + 1]; k++) {
            int64_t a = pinv ? pinv[i] : i, b = pinv ? pinv[ci[k]] : ci[k];
            int64_t d = a > b ? a - b : b - a;
            if (d > bw) bw = d;
        }
    free(pinv);
    return bw;
}

/* perm[k] = old index of the vertex placed at new position k.
 * Steps: (1) graph with an edge {i, j} per stored (i, j); (2) while vertices
 * remain unvisited, start a breadth-first search at the unvisited vertex of
 * least degree (lowest index on ties); (3) on dequeuing a vertex, append its
 * unvisited neighbours in (degree, index) order, marking them visited when
 * they are enqueued; (4) the concatenated visit order is the Cuthill-McKee
 * order, reversed as a whole it is RCM; (5) with guard != 0, when the RCM
 * bandwidth exceeds the original one, the identity is returned instead. */
/* Level structure rooted at r (breadth-first search over the whole graph,
 * which reaches exactly r's component): returns the eccentricity of r (the
 * index of the last level) and, in *last_min, the vertex of the last level
 * with the smallest (degree, index).  dist[] is -1 on entry and on exit. */
static int32_t orc_last_level(const int64_t *arp, const int32_t *adj, const int32_t *deg, int32_t r,
                              int32_t *dist, int32_t *queue, int32_t *last_min)
{
    int32_t head = 0, tail = 0;
    dist[r] = 0;
    queue[tail++] = r;
    while (head < tail) {
        int32_t v = queue[head++];
        for (int64_t k = arp[v]; k < arp[v + 1]; k++)
            if (dist[adj[k]] < 0) {
                dist[adj[k]] = dist[v] + 1;
                queue[tail++] = adj[k];
            }
    }
    int32_t ecc = dist[queue[tail - 1]];
    int32_t best = -1;
    for (int32_t q = 0; q < tail; q++) {
        int32_t v = queue[q];
        if (dist[v] == ecc && (best < 0 || deg[v] < deg[best] || (deg[v] == deg[best] && v < best))) best = v;
    }
    for (int32_t q = 0; q < tail; q++) dist[queue[q]] = -1;
    *last_min = best;
    return ecc;
}

/* George-Liu pseudo-peripheral vertex of r's component: from r, take the
 * last level's smallest (degree, index) vertex x; while x is strictly more
 * eccentric than r, move r to x and repeat. */
static int32_t orc_pseudo_peripheral(const int64_t *arp, const int32_t *adj, const int32_t *deg, int32_t r,
                                     int32_t *dist, int32_t *queue)
{
    int32_t x;
    int32_t e = orc_last_level(arp, adj, deg, r, dist, queue, &x);
    for (;;) {
        int32_t y;
        int32_t ex = orc_last_level(arp, adj, deg, x, dist, queue, &y);
        if (ex <= e) return r;
        r = x;
        e = ex;
        x = y;
    }
}

static int cmp_i32(const void *pa, const void *pb)
{
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    return a < b ? -1 : (a > b ? 1 : 0);
}

int orc_rcm(int32_t n, const int32_t *rp, const int32_t *ci, int32_t flags,
            int32_t *perm, int64_t *bw_before, int64_t *bw_after);

/* 1 when v is in the sorted list adj[lo .. hi) */
static int orc_in_sorted(const int32_t *adj, int64_t lo, int64_t hi, int32_t v)
{
    const int64_t end = hi;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (adj[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo < end && adj[lo] == v ? 1 : 0;
}

/* Local-edge RCM (flags bit 2), a reordering for small-world patterns, where
 * a few long-range "shortcut" edges make every breadth-first level huge (the
 * paper notes that RCM's benefit depends on the pattern, Sec. 4.1, Fig. 5):
 * RCM, with the caller's start rule, of the pattern restricted to its local
 * edges.  An edge {u, v} is local when it lies on a triangle or a 4-cycle
 * (u and v have a common neighbour, or a neighbour a of u other than v is
 * adjacent to a neighbour b of v other than u and a), or when deg(u) deg(v) >
 * ORC_LOCAL_DEG (then it is kept untested).  The other edges stay in the
 * matrix; only the ordering ignores them.  The guard is applied by the
 * caller to the final order over all edges. */
#define ORC_LOCAL_DEG 4096
static int orc_rcm_local(int32_t n, const int32_t *rp, const int32_t *ci, int32_t flags, int32_t *perm)
{
    size_t nn = (size_t)(n > 0 ? n : 1);
    int64_t m = rp[n];
    int64_t *arp = (int64_t *)calloc(nn + 1, sizeof(int64_t));
    int32_t *adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    int64_t *fill = (int64_t *)calloc(nn, sizeof(int64_t));
    int32_t *rp2 = (int32_t *)malloc(sizeof(int32_t) * (nn + 1));
    int32_t *ci2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
    if (!arp || !adj || !fill || !rp2 || !ci2) {
        free(arp); free(adj); free(fill); free(rp2); free(ci2);
        return ORC_ENOMEM;
    }
    /* sorted adjacency lists of the symmetric pattern */
    for (int32_t i = 0; i < n; i++)
        for (int32_t k = rp[i]; k < rp[i + 1]; k++) { arp[i + 1]++; arp[ci[k] + 1]++; }
    for (int32_t i = 0; i < n; i++) arp[i + 1] += arp[i];
    for (int32_t i = 0; i < n; i++) fill[i] = arp[i];
    for (int32_t i = 0; i < n; i++)
        for (int32_t k = rp[i]; k < rp[i + 1]; k++) {
            adj[fill[i]++] = ci[k];
            adj[fill[ci[k]]++] = i;
        }
    for (int32_t i = 0; i < n; i++) qsort(adj + arp[i], (size_t)(arp[i + 1] - arp[i]), sizeof(int32_t), cmp_i32);
    /* the local edges, in the order of the input */
    int32_t q = 0;
    rp2[0] = 0;
    for (int32_t u = 0; u < n; u++) {
        for (int32_t k = rp[u]; k < rp[u + 1]; k++) {
            int32_t v = ci[k];
            int64_t du = arp[u + 1] - arp[u], dv = arp[v + 1] - arp[v];
            int local = du * dv > ORC_LOCAL_DEG;
            for (int64_t x = arp[u]; !local && x < arp[u + 1]; x++) {
                int32_t a = adj[x];
                if (a == v) continue;
                if (orc_in_sorted(adj, arp[v], arp[v + 1], a)) { local = 1; break; }      /* triangle */
                for (int64_t y = arp[v]; y < arp[v + 1]; y++) {
                    int32_t b = adj[y];
                    if (b == u || b == a) continue;
                    if (orc_in_sorted(adj, arp[a], arp[a + 1], b)) { local = 1; break; } /* 4-cycle */
                }
            }
            if (local) ci2[q++] = v;
        }
        rp2[u + 1] = q;
    }
    int rc = orc_rcm(n, rp2, ci2, flags & 2, perm, NULL, NULL);
    free(arp); free(adj); free(fill); free(rp2); free(ci2);
    return rc;
}

/* flags: bit 0 (1) the identity guard, bit 1 (2) start each component at a
 * pseudo-peripheral vertex found from the (degree, index) candidate, bit 2
 * (4) RCM of the local edges only (orc_rcm_local). */
int orc_rcm(int32_t n, const int32_t *rp, const int32_t *ci, int32_t flags,
            int32_t *perm, int64_t *bw_before, int64_t *bw_after)
{
    const int32_t guard = flags & 1, peripheral = flags & 2;
    if (n < 0) return ORC_EINVAL;
    if (flags & 4) {
        int rc = orc_rcm_local(n, rp, ci, flags, perm);
        if (rc != ORC_OK) return rc;
        int64_t b0 = orc_bandwidth(n, rp, ci, NULL);
        int64_t b1 = orc_bandwidth(n, rp, ci, perm);
        if (guard && b1 > b0) {
            for (int32_t k = 0; k < n; k++) perm[k] = k;
            b1 = b0;
        }
        if (bw_before) *bw_before = b0;
        if (bw_after) *bw_after = b1;
        return ORC_OK;
    }
    size_t nn = (size_t)(n > 0 ? n : 1);
    int64_t nnz = rp[n];
    int64_t *arp = (int64_t *)calloc(nn + 1, sizeof(int64_t));
    int32_t *adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * nnz + 1));
    int32_t *deg = (int32_t *)calloc(nn, sizeof(int32_t));
    int32_t *by_deg = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *cm = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * nn);
    char *seen = (char *)calloc(nn, 1);
    int64_t *fill = (int64_t *)calloc(nn, sizeof(int64_t));
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * nn);
    if (!arp || !adj || !deg || !by_deg || !cm || !tmp || !seen || !fill || !dist || !queue) {
        free(arp); free(adj); free(deg); free(by_deg); free(cm); free(tmp); free(seen); free(fill);
        free(dist); free(queue);
        return ORC_ENOMEM;
    }
    for (int32_t i = 0; i < n; i++) dist[i] = -1;
    /* (1) adjacency lists of the symmetric pattern */
    for (int32_t i = 0; i < n; i++)
        for (int32_t k = rp[i]; k < rp[i + 1]; k++) { deg[i]++; deg[ci[k]]++; }
    for (int32_t i = 0; i < n; i++) arp[i + 1] = arp[i] + deg[i];
    for (int32_t i = 0; i < n; i++) fill[i] = arp[i];
    for (int32_t i = 0; i < n; i++)
        for (int32_t k = rp[i]; k < rp[i + 1]; k++) {
            adj[fill[i]++] = ci[k];
            adj[fill[ci[k]]++] = i;
        }
    /* (2) all vertices in (degree, index) order: the first unvisited one in
     * this list is the next start vertex */
    for (int32_t i = 0; i < n; i++) by_deg[i] = i;
    g_deg = deg;
    qsort(by_deg, (size_t)n, sizeof(int32_t), cmp_deg_idx);

    int32_t count = 0, head = 0, next_start = 0;
    while (count < n) {
        while (seen[by_deg[next_start]]) next_start++;
        int32_t s = by_deg[next_start];
        if (peripheral && deg[s] > 0) s = orc_pseudo_peripheral(arp, adj, deg, s, dist, queue);
        seen[s] = 1;
        cm[count++] = s;
        /* (3) breadth-first search, the cm array doubles as the FIFO queue */
        while (head < count) {
            int32_t v = cm[head++];
            int32_t m = 0;
            for (int64_t k = arp[v]; k < arp[v + 1]; k++)
                if (!seen[adj[k]]) tmp[m++] = adj[k];
            g_deg = deg;
            qsort(tmp, (size_t)m, sizeof(int32_t), cmp_deg_idx);
            for (int32_t q = 0; q < m; q++) {
                seen[tmp[q]] = 1;
                cm[count++] = tmp[q];
            }
        }
    }
    /* (4) reverse */
    for (int32_t k = 0; k < n; k++) perm[k] = cm[n - 1 - k];

    int64_t b0 = orc_bandwidth(n, rp, ci, NULL);
    int64_t b1 = orc_bandwidth(n, rp, ci, perm);
    /* (5) guard: a matrix that is already banded gains nothing (Sec. 4.1) */
    if (guard && b1 > b0) {
        for (int32_t k = 0; k < n; k++) perm[k] = k;
        b1 = b0;
    }
    if (bw_before) *bw_before = b0;
    if (bw_after) *bw_after = b1;
    free(arp); free(adj); free(deg); free(by_deg); free(cm); free(tmp); free(seen); free(fill);
    free(dist); free(queue);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* O3: the 3-way band split in canonical form (Sec. 3.1.2, Figs. 7-8)        */
/* ------------------------------------------------------------------------ */

/* class codes of a stored entry of the reordered lower triangle */
#define ORC_MID_LOCAL 0  /* 1 <= i-j <= W and j in the same row tile as i */
#define ORC_MID_HALO 1   /* 1 <= i-j <= W and j in an earlier tile (the one before) */
#define ORC_OUTER 2      /* i-j > W */

typedef struct { int32_t r, c; double v; } orc_trip;

static int cmp_trip_rc(const void *pa, const void *pb)
{
    const orc_trip *a = (const orc_trip *)pa, *b = (const orc_trip *)pb;
    if (a->r != b->r) return a->r < b->r ? -1 : 1;
    if (a->c != b->c) return a->c < b->c ? -1 : 1;
    return 0;
}

static const int32_t *g_row_of, *g_col_of; /* comparator context */

static int cmp_entry_cr(const void *pa, const void *pb)
{
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    if (g_col_of[a] != g_col_of[b]) return g_col_of[a] < g_col_of[b] ? -1 : 1;
    if (g_row_of[a] != g_row_of[b]) return g_row_of[a] < g_row_of[b] ? -1 : 1;
    return 0;
}

/* Canonical split of P S P^T for the ordering perm (new -> old), row tile T
 * and middle bandwidth W (1 <= W <= T):
 *  - brp/bci/bv: strict lower CSR of P S P^T.  An entry (i, j, a) moves to
 *    (p^-1(i), p^-1(j)); when that lands above the diagonal it is stored
 *    transposed with its sign flipped (a_ji = -a_ij, Eq. 2).
 *  - cls[e]: ORC_MID_LOCAL / ORC_MID_HALO / ORC_OUTER for entry e (rows are
 *    split in tiles of T rows: tile t holds rows [tT, tT+T)).
 *  - tile_ptr[ntiles+1] / tile_list: for each tile, the indices e of its
 *    middle entries (local and halo) sorted by (column, row): the order in
 *    which the mirrored products y_j -= a_ij x_i are summed.
 *  - outer_csr: indices of the outer entries in (row, column) order;
 *    outer_csc: the same indices in (column, row) order.
 *  - counts[0..2]: number of entries of each class.
 * Arrays are caller-allocated: brp[n+1], bci/bv/cls[nnz], tile_ptr[ntiles+1],
 * tile_list[nnz], outer_csr/outer_csc[nnz]. */
int orc_split(int32_t n, const int32_t *rp, const int32_t *ci, const double *v, double mirror,
              const int32_t *perm, int32_t T, int32_t W,
              int32_t *brp, int32_t *bci, double *bv, uint8_t *cls,
              int32_t *tile_ptr, int32_t *tile_list, int32_t *outer_csr, int32_t *outer_csc,
              int64_t *counts)
{
    if (n < 0 || T < 1 || W < 1 || W > T) return ORC_EINVAL;
    int64_t nnz = rp[n];
    size_t nn = (size_t)(n > 0 ? n : 1);
    int32_t ntiles = (n + T - 1) / T;
    int32_t *pinv = (int32_t *)malloc(sizeof(int32_t) * nn);
    orc_trip *tr = (orc_trip *)malloc(sizeof(orc_trip) * (size_t)(nnz > 0 ? nnz : 1));
    int32_t *row_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    if (!pinv || !tr || !row_of) { free(pinv); free(tr); free(row_of); return ORC_ENOMEM; }
    for (int32_t k = 0; k < n; k++) pinv[perm[k]] = k;

    /* re-triangularize */
    int64_t m = 0;
    for (int32_t i = 0; i < n; i++)
        for (int32_t k = rp[i]; k < rp[i + 1]; k++) {
            int32_t a = pinv[i], b = pinv[ci[k]];
            if (a > b) { tr[m].r = a; tr[m].c = b; tr[m].v = v[k]; }
            else       { tr[m].r = b; tr[m].c = a; tr[m].v = mirror * v[k]; }
            m++;
        }
    qsort(tr, (size_t)nnz, sizeof(orc_trip), cmp_trip_rc);
    for (int32_t i = 0; i <= n; i++) brp[i] = 0;
    for (int64_t e = 0; e < nnz; e++) {
        brp[tr[e].r + 1]++;
        bci[e] = tr[e].c;
        bv[e] = tr[e].v;
        row_of[e] = tr[e].r;
    }
    for (int32_t i = 0; i < n; i++) brp[i + 1] += brp[i];

    /* classify */
    counts[0] = counts[1] = counts[2] = 0;
    for (int64_t e = 0; e < nnz; e++) {
        int32_t i = row_of[e], j = bci[e];
        int32_t r0 = (i / T) * T;
        if (i - j <= W) cls[e] = (j >= r0) ? ORC_MID_LOCAL : ORC_MID_HALO;
        else cls[e] = ORC_OUTER;
        counts[cls[e]]++;
    }

    /* per-tile middle lists in (column, row) order */
    g_row_of = row_of;
    g_col_of = bci;
    int32_t q = 0;
    for (int32_t t = 0; t < ntiles; t++) {
        tile_ptr[t] = q;
        int32_t r0 = t * T, r1 = (t + 1) * T < n ? (t + 1) * T : n;
        int32_t start = q;
        for (int32_t i = r0; i < r1; i++)
            for (int32_t e = brp[i]; e < brp[i + 1]; e++)
                if (cls[e] != ORC_OUTER) tile_list[q++] = e;
        qsort(tile_list + start, (size_t)(q - start), sizeof(int32_t), cmp_entry_cr);
    }
    tile_ptr[ntiles] = q;

    /* outer entries in row order and in column order */
    int32_t o = 0;
    for (int64_t e = 0; e < nnz; e++)
        if (cls[e] == ORC_OUTER) { outer_csr[o] = (int32_t)e; outer_csc[o] = (int32_t)e; o++; }
    qsort(outer_csc, (size_t)o, sizeof(int32_t), cmp_entry_cr);

    free(pinv); free(tr); free(row_of);
    return ORC_OK;
}

/* Default cut point (Fig. 8: the distance from the diagonal to the outer
 * split is a bandwidth parameter).  Rule of this implementation: W is the
 * smallest power of two >= the reordered bandwidth, clamped to
 * [w_min, w_cap]; the row tile is T = max(W, t_min).  w_min, w_cap and t_min
 * are powers of two supplied by the caller. */
void orc_auto_cut(int64_t bw, int32_t w_min, int32_t w_cap, int32_t t_min,
                  int32_t *T_out, int32_t *W_out)
{
    int64_t W = w_min;
    while (W < bw && W < w_cap) W *= 2;
    if (W > w_cap) W = w_cap;
    *W_out = (int32_t)W;
    *T_out = (int32_t)(W > t_min ? W : t_min);
}
