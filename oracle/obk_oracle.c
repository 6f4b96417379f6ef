/*
 * obk_oracle.c -- plain, slow, single-threaded FP64 CPU oracle for OBK-RCM.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header or table with the CUDA
 * path.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no FMA contraction,
 * IEEE sqrt and division, round to nearest everywhere).
 *
 * What it computes, step by step, in the paper's order (Liang & Li, "OBK-RCM",
 * arXiv 2401.00672):
 *   extend      Section 4.1 Algorithm 5 (m > n: A^ = [A, O], f^ = f) and
 *               Section 4.2 Algorithm 6 (m < n: A^ = [A; O], f^ = [f; 0]).
 *   rcm         Section 3.2 / Algorithm 4 step 1: Reverse Cuthill-McKee.  The
 *               paper names the method only; the reading used here (graph of
 *               pattern(A^ + A^T) without self loops, George-Liu pseudo-peripheral
 *               start from the minimum-(degree, index) vertex, children in
 *               (degree, index) order, components in order of their
 *               minimum-(degree, index) vertex, one reversal of the whole list).
 *   permute     Eq. 3.1-3.2: A~ = P A^ P^T, f~ = P f^.
 *   norms       ||A_i||^2 of Eq. 1.2 (left fold over ascending columns).
 *   groups      Section 3.3 cosine table and threshold rule, taken at k = m
 *               (one block per row): cos_ij = (A_i, A_j) / (||A_i|| ||A_j||),
 *               conflict when |cos_ij| >= thr, greedy first-fit groups in index
 *               order (each row joins the first group holding no conflicting
 *               earlier row).
 *   sweep       Eq. 1.2 / Eq. 1.3 / Eq. 3.3 / Algorithm 4 iteration: for each
 *               group, y_i = (f_i - A_i x) / ||A_i||^2 for every row of the group
 *               from the group-start x, then x += sum_i y_i A_i^T (rows ascending).
 *               For a group of mutually orthogonal rows this is exactly
 *               x + A_tau^+ (f_tau - A_tau x).
 *   residual    ||f - A x||_2 / ||f||_2 after each sweep (stop rule).
 *   unpermute   x = P^T x~ (Algorithm 4 last step), then x = x^(1:n) for m > n.
 *   refine      FP32 inner sweeps inside FP64 iterative refinement (not in the
 *               paper; the FP32 arithmetic is done in C float, no contraction).
 *   stats       Definitions 1-2 at the row level: the nonzero entries of the
 *               N x N row-cosine table and the sum of their |cos|, each rounded
 *               to a multiple of 2^-32 (zn and nn follow from the two).
 *   pinv step   Eq. 1.3 for a near-orthogonal group: y solves the group's Gram
 *               system (A_tau A_tau^T) y = f_tau - A_tau x by K Jacobi steps from
 *               the simultaneous step y = r / ||A_i||^2, then x += A_tau^T y.
 *   blocks      Algorithm 4 as printed: k blocks of consecutive rows, centroid
 *               cosines, Oclass pairs and Nclass blocks, each block's
 *               correction A_b^+ r as the CGLS least-squares solution from zero.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_NOT_CONVERGED 1
#define ORC_INVALID (-1)
#define ORC_NOMEM (-2)

/* ------------------------------------------------------------------ */
/* validation                                                          */
/* ------------------------------------------------------------------ */

/* Returns ORC_OK if (row_ptr, col_idx, val) is a valid m x n CSR: row_ptr
 * monotone from 0 to nnz, columns in [0, n) strictly increasing in each row,
 * finite values. */
int orc_validate(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci,
                 const double* v, int64_t nnz)
{
    if (m <= 0 || n <= 0 || nnz < 0) return ORC_INVALID;
    if (rp[0] != 0 || rp[m] != nnz) return ORC_INVALID;
    for (int64_t i = 0; i < m; ++i) {
        if (rp[i + 1] < rp[i]) return ORC_INVALID;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            if (ci[e] < 0 || (int64_t)ci[e] >= n) return ORC_INVALID;
            if (e > rp[i] && ci[e] <= ci[e - 1]) return ORC_INVALID;
            if (!isfinite(v[e])) return ORC_INVALID;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* extension to a square system (Algorithms 5 and 6)                   */
/* ------------------------------------------------------------------ */

/* N = max(m, n).  Writes the N+1 row pointers of A^ (columns and values are
 * those of A: [A, O] adds only columns that hold no entry, [A; O] adds empty
 * rows), f^ (N) and x^0 (N). x0 may be NULL (zero start). */
void orc_extend(int64_t m, int64_t n, const int64_t* rp, const double* f,
                const double* x0, int64_t* rp_hat, double* f_hat, double* x_hat)
{
    int64_t N = m > n ? m : n;
    for (int64_t i = 0; i <= m; ++i) rp_hat[i] = rp[i];
    for (int64_t i = m + 1; i <= N; ++i) rp_hat[i] = rp[m];
    for (int64_t i = 0; i < N; ++i) f_hat[i] = i < m ? f[i] : 0.0;
    for (int64_t i = 0; i < N; ++i) x_hat[i] = (i < n && x0) ? x0[i] : 0.0;
}

/* ------------------------------------------------------------------ */
/* Reverse Cuthill-McKee                                               */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t N;
    int64_t* ptr; /* N+1 */
    int32_t* adj; /* sorted, unique neighbour lists, no self loops */
} graph_t;

static int cmp_i32(const void* a, const void* b)
{
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* Graph of pattern(A + A^T) minus self loops. */
static int build_sym_graph(int64_t N, const int64_t* rp, const int32_t* ci, graph_t* g)
{
    int64_t nnz = rp[N];
    int64_t* cnt = calloc((size_t)N + 1, sizeof(int64_t));
    if (!cnt) return ORC_NOMEM;
    for (int64_t i = 0; i < N; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
            if (ci[e] != i) { cnt[i]++; cnt[ci[e]]++; }
    int64_t* ptr = malloc(((size_t)N + 1) * sizeof(int64_t));
    int32_t* tmp = malloc((size_t)(2 * nnz + 1) * sizeof(int32_t));
    if (!ptr || !tmp) { free(cnt); free(ptr); free(tmp); return ORC_NOMEM; }
    ptr[0] = 0;
    for (int64_t i = 0; i < N; ++i) ptr[i + 1] = ptr[i] + cnt[i];
    for (int64_t i = 0; i < N; ++i) cnt[i] = ptr[i];
    for (int64_t i = 0; i < N; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
            if (ci[e] != i) { tmp[cnt[i]++] = ci[e]; tmp[cnt[ci[e]]++] = (int32_t)i; }
    /* sort and drop duplicates, compacting in place */
    int64_t w = 0;
    int64_t* nptr = malloc(((size_t)N + 1) * sizeof(int64_t));
    if (!nptr) { free(cnt); free(ptr); free(tmp); return ORC_NOMEM; }
    nptr[0] = 0;
    for (int64_t i = 0; i < N; ++i) {
        int64_t s = ptr[i], e = ptr[i + 1];
        qsort(tmp + s, (size_t)(e - s), sizeof(int32_t), cmp_i32);
        for (int64_t k = s; k < e; ++k)
            if (k == s || tmp[k] != tmp[k - 1]) tmp[w++] = tmp[k];
        nptr[i + 1] = w;
    }
    free(cnt);
    free(ptr);
    g->N = N;
    g->ptr = nptr;
    g->adj = tmp;
    return ORC_OK;
}

static const int64_t* g_deg_for_sort; /* qsort has no context argument */

/* (degree, index) order */
static int cmp_deg_idx(const void* a, const void* b)
{
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    int64_t dx = g_deg_for_sort[x], dy = g_deg_for_sort[y];
    if (dx != dy) return (dx > dy) - (dx < dy);
    return (x > y) - (x < y);
}

static int deg_idx_less(const int64_t* deg, int32_t a, int32_t b)
{
    return deg[a] < deg[b] || (deg[a] == deg[b] && a < b);
}

/* Breadth-first level structure rooted at r.  Uses stamp[] == tag to mark
 * vertices reached in this search.  Returns the eccentricity of r (index of the
 * last level) and the vertex of the last level with minimum (degree, index). */
static int64_t bfs_last_level(const graph_t* g, const int64_t* deg, int32_t r,
                              int32_t* queue, int64_t* stamp, int64_t tag, int32_t* best)
{
    int64_t head = 0, tail = 0, level = 0;
    queue[tail++] = r;
    stamp[r] = tag;
    int64_t level_start = 0, level_end = 1;
    for (;;) {
        while (head < level_end) {
            int32_t u = queue[head++];
            for (int64_t e = g->ptr[u]; e < g->ptr[u + 1]; ++e) {
                int32_t w = g->adj[e];
                if (stamp[w] != tag) { stamp[w] = tag; queue[tail++] = w; }
            }
        }
        if (tail == level_end) break; /* no next level */
        level++;
        level_start = level_end;
        level_end = tail;
    }
    int32_t b = queue[level_start];
    for (int64_t k = level_start + 1; k < level_end; ++k)
        if (deg_idx_less(deg, queue[k], b)) b = queue[k];
    *best = b;
    return level;
}

/* perm[k] = old index of the vertex placed at new position k. */
int orc_rcm(int64_t N, const int64_t* rp, const int32_t* ci, int32_t* perm)
{
    graph_t g;
    int rc = build_sym_graph(N, rp, ci, &g);
    if (rc) return rc;
    int64_t* deg = malloc((size_t)N * sizeof(int64_t));
    int32_t* by_deg = malloc((size_t)N * sizeof(int32_t));
    int32_t* order = malloc((size_t)N * sizeof(int32_t));
    int32_t* queue = malloc((size_t)N * sizeof(int32_t));
    int64_t* stamp = malloc((size_t)N * sizeof(int64_t));
    char* visited = calloc((size_t)N, 1);
    int32_t* kids = malloc((size_t)N * sizeof(int32_t));
    if (!deg || !by_deg || !order || !queue || !stamp || !visited || !kids) {
        rc = ORC_NOMEM;
        goto done;
    }
    for (int64_t v = 0; v < N; ++v) {
        deg[v] = g.ptr[v + 1] - g.ptr[v];
        by_deg[v] = (int32_t)v;
        stamp[v] = -1;
    }
    g_deg_for_sort = deg;
    qsort(by_deg, (size_t)N, sizeof(int32_t), cmp_deg_idx);

    int64_t placed = 0, scan = 0, tag = 0;
    while (placed < N) {
        /* s0: unvisited vertex with minimum (degree, index) */
        while (visited[by_deg[scan]]) scan++;
        int32_t v = by_deg[scan];
        /* pseudo-peripheral node (George-Liu) */
        int32_t u;
        int64_t ecc_v = bfs_last_level(&g, deg, v, queue, stamp, tag++, &u);
        for (;;) {
            int32_t u2;
            int64_t ecc_u = bfs_last_level(&g, deg, u, queue, stamp, tag++, &u2);
            if (ecc_u > ecc_v) { v = u; ecc_v = ecc_u; u = u2; }
            else break;
        }
        /* Cuthill-McKee from v */
        int64_t head = placed;
        order[placed++] = v;
        visited[v] = 1;
        while (head < placed) {
            int32_t p = order[head++];
            int64_t nk = 0;
            for (int64_t e = g.ptr[p]; e < g.ptr[p + 1]; ++e) {
                int32_t w = g.adj[e];
                if (!visited[w]) { visited[w] = 1; kids[nk++] = w; }
            }
            qsort(kids, (size_t)nk, sizeof(int32_t), cmp_deg_idx);
            for (int64_t k = 0; k < nk; ++k) order[placed++] = kids[k];
        }
    }
    for (int64_t k = 0; k < N; ++k) perm[k] = order[N - 1 - k];
done:
    free(deg); free(by_deg); free(order); free(queue); free(stamp); free(visited); free(kids);
    free(g.ptr); free(g.adj);
    return rc;
}

/* Half bandwidth max |i - j| over stored entries. */
int64_t orc_bandwidth(int64_t N, const int64_t* rp, const int32_t* ci)
{
    int64_t bw = 0;
    for (int64_t i = 0; i < N; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            int64_t d = i - ci[e];
            if (d < 0) d = -d;
            if (d > bw) bw = d;
        }
    return bw;
}

/* ------------------------------------------------------------------ */
/* symmetric permutation A~ = P A P^T (Eq. 3.1)                        */
/* ------------------------------------------------------------------ */

typedef struct { int32_t c; double v; } entry_t;
static int cmp_entry(const void* a, const void* b)
{
    int32_t x = ((const entry_t*)a)->c, y = ((const entry_t*)b)->c;
    return (x > y) - (x < y);
}

int orc_permute(int64_t N, const int64_t* rp, const int32_t* ci, const double* v,
                const int32_t* perm, int64_t* rp_out, int32_t* ci_out, double* v_out)
{
    int32_t* iperm = malloc((size_t)N * sizeof(int32_t));
    int64_t maxlen = 0;
    for (int64_t i = 0; i < N; ++i)
        if (rp[i + 1] - rp[i] > maxlen) maxlen = rp[i + 1] - rp[i];
    entry_t* buf = malloc((size_t)(maxlen + 1) * sizeof(entry_t));
    if (!iperm || !buf) { free(iperm); free(buf); return ORC_NOMEM; }
    for (int64_t k = 0; k < N; ++k) iperm[perm[k]] = (int32_t)k;
    rp_out[0] = 0;
    for (int64_t k = 0; k < N; ++k) {
        int64_t old = perm[k], len = rp[old + 1] - rp[old];
        for (int64_t t = 0; t < len; ++t) {
            buf[t].c = iperm[ci[rp[old] + t]];
            buf[t].v = v[rp[old] + t];
        }
        qsort(buf, (size_t)len, sizeof(entry_t), cmp_entry);
        for (int64_t t = 0; t < len; ++t) {
            ci_out[rp_out[k] + t] = buf[t].c;
            v_out[rp_out[k] + t] = buf[t].v;
        }
        rp_out[k + 1] = rp_out[k] + len;
    }
    free(iperm);
    free(buf);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* row norms ||A_i||^2 (Eq. 1.2 denominator)                           */
/* ------------------------------------------------------------------ */

void orc_row_norms(int64_t N, const int64_t* rp, const double* v, double* nsq)
{
    for (int64_t i = 0; i < N; ++i) {
        double s = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) s = s + v[e] * v[e];
        nsq[i] = s;
    }
}

/* ------------------------------------------------------------------ */
/* cosine-threshold grouping (Section 3.3 at k = m)                    */
/* ------------------------------------------------------------------ */

/* group_of[i] = group of row i (-1 for an all-zero row, which takes no part
 * in the iteration).  Returns the number of groups in *G.  Optionally writes the
 * number of conflicting pairs (i > j, |cos| >= thr) in *n_conflicts. */
int orc_group_build(int64_t N, const int64_t* rp, const int32_t* ci, const double* v,
                    const double* nsq, double thr, int32_t* group_of, int64_t* G,
                    int64_t* n_conflicts)
{
    int64_t nnz = rp[N];
    /* column lists: rows ascending, with values */
    int64_t* cptr = calloc((size_t)N + 1, sizeof(int64_t));
    int32_t* crow = malloc((size_t)(nnz + 1) * sizeof(int32_t));
    double* cval = malloc((size_t)(nnz + 1) * sizeof(double));
    double* acc = calloc((size_t)N, sizeof(double));
    char* touched = calloc((size_t)N, 1);
    int32_t* tlist = malloc((size_t)N * sizeof(int32_t));
    double* s = malloc((size_t)N * sizeof(double));
    int32_t* conf = malloc((size_t)N * sizeof(int32_t));
    int64_t* fill = malloc((size_t)N * sizeof(int64_t));
    if (!cptr || !crow || !cval || !acc || !touched || !tlist || !s || !conf || !fill) {
        free(cptr); free(crow); free(cval); free(acc); free(touched); free(tlist);
        free(s); free(conf); free(fill);
        return ORC_NOMEM;
    }
    for (int64_t e = 0; e < nnz; ++e) cptr[ci[e] + 1]++;
    for (int64_t c = 0; c < N; ++c) cptr[c + 1] += cptr[c];
    for (int64_t c = 0; c < N; ++c) fill[c] = cptr[c];
    for (int64_t i = 0; i < N; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            int64_t p = fill[ci[e]]++;
            crow[p] = (int32_t)i;
            cval[p] = v[e];
        }
    for (int64_t i = 0; i < N; ++i) s[i] = sqrt(nsq[i]);

    int64_t ng = 0, nconf_total = 0;
    for (int64_t i = 0; i < N; ++i) {
        if (nsq[i] == 0.0) { group_of[i] = -1; continue; }
        /* dot products with every earlier row sharing a column; for each such
         * row the products are added in ascending column order (left fold) */
        int64_t nt = 0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            int32_t c = ci[e];
            for (int64_t p = cptr[c]; p < cptr[c + 1]; ++p) {
                int32_t j = crow[p];
                if (j >= i) break; /* rows ascending in the column */
                if (nsq[j] == 0.0) continue;
                if (!touched[j]) { touched[j] = 1; acc[j] = 0.0; tlist[nt++] = j; }
                acc[j] = acc[j] + v[e] * cval[p];
            }
        }
        int64_t nc = 0;
        for (int64_t t = 0; t < nt; ++t) {
            int32_t j = tlist[t];
            double cosv = acc[j] / (s[j] * s[i]);
            if (fabs(cosv) >= thr) conf[nc++] = group_of[j];
            touched[j] = 0;
        }
        nconf_total += nc;
        /* first-fit: smallest group index not used by a conflicting earlier row */
        int32_t g = 0;
        for (;;) {
            int used = 0;
            for (int64_t t = 0; t < nc; ++t)
                if (conf[t] == g) { used = 1; break; }
            if (!used) break;
            g++;
        }
        group_of[i] = g;
        if (g + 1 > ng) ng = g + 1;
    }
    *G = ng;
    if (n_conflicts) *n_conflicts = nconf_total;
    free(cptr); free(crow); free(cval); free(acc); free(touched); free(tlist);
    free(s); free(conf); free(fill);
    return ORC_OK;
}

/* Cosine table statistics (Section 3.6, Definitions 1 and 2, read at the row
 * level k = N): C is the N x N table of row cosines C_ij = dot_ij /
 * (||A_i|| ||A_j||) with dot_ij the left fold of the products over the common
 * columns in ascending order (the grouping's arithmetic), C_ii = 1 for a
 * nonzero row, and every entry of a zero row 0.  *nz = number of nonzero
 * entries of C; *sum = sum over the nonzero entries of |C_ij| rounded to the
 * nearest multiple of 2^-32, in units of 2^-32 (an integer, so the total does
 * not depend on the order of summation).  Then zn = (N^2 - nz) / N^2 and
 * nn = sum 2^-32 / N^2. */
int orc_cosine_stats(int64_t N, const int64_t* rp, const int32_t* ci, const double* v, const double* nsq,
                     int64_t* nz, uint64_t* sum)
{
    int64_t nnz = rp[N];
    int64_t* cptr = calloc((size_t)N + 1, sizeof(int64_t));
    int32_t* crow = malloc((size_t)(nnz + 1) * sizeof(int32_t));
    double* cval = malloc((size_t)(nnz + 1) * sizeof(double));
    double* acc = calloc((size_t)N, sizeof(double));
    char* touched = calloc((size_t)N, 1);
    int32_t* tlist = malloc((size_t)N * sizeof(int32_t));
    double* s = malloc((size_t)N * sizeof(double));
    int64_t* fill = malloc((size_t)N * sizeof(int64_t));
    if (!cptr || !crow || !cval || !acc || !touched || !tlist || !s || !fill) {
        free(cptr); free(crow); free(cval); free(acc); free(touched); free(tlist); free(s); free(fill);
        return ORC_NOMEM;
    }
    for (int64_t e = 0; e < nnz; ++e) cptr[ci[e] + 1]++;
    for (int64_t c = 0; c < N; ++c) cptr[c + 1] += cptr[c];
    for (int64_t c = 0; c < N; ++c) fill[c] = cptr[c];
    for (int64_t i = 0; i < N; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            int64_t p = fill[ci[e]]++;
            crow[p] = (int32_t)i;
            cval[p] = v[e];
        }
    for (int64_t i = 0; i < N; ++i) s[i] = sqrt(nsq[i]);
    int64_t cnt = 0;
    uint64_t tot = 0;
    for (int64_t i = 0; i < N; ++i) {
        if (nsq[i] == 0.0) continue;
        cnt += 1;                     /* C_ii = 1 */
        tot += (uint64_t)1 << 32;
        int64_t nt = 0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            int32_t c = ci[e];
            for (int64_t p = cptr[c]; p < cptr[c + 1]; ++p) {
                int32_t j = crow[p];
                if (j >= i) break;
                if (nsq[j] == 0.0) continue;
                if (!touched[j]) { touched[j] = 1; acc[j] = 0.0; tlist[nt++] = j; }
                acc[j] = acc[j] + v[e] * cval[p];
            }
        }
        for (int64_t t = 0; t < nt; ++t) {
            int32_t j = tlist[t];
            double cosv = acc[j] / (s[j] * s[i]);
            if (cosv != 0.0) {        /* C_ij and C_ji */
                cnt += 2;
                tot += 2 * (uint64_t)llrint(fabs(cosv) * 0x1p32);
            }
            touched[j] = 0;
        }
    }
    *nz = cnt;
    *sum = tot;
    free(cptr); free(crow); free(cval); free(acc); free(touched); free(tlist); free(s); free(fill);
    return ORC_OK;
}

/* group_ptr[G+1], group_rows[count of grouped rows]: rows ascending per group. */
void orc_group_lists(int64_t N, const int32_t* group_of, int64_t G, int64_t* gptr, int32_t* grows)
{
    for (int64_t g = 0; g <= G; ++g) gptr[g] = 0;
    for (int64_t i = 0; i < N; ++i)
        if (group_of[i] >= 0) gptr[group_of[i] + 1]++;
    for (int64_t g = 0; g < G; ++g) gptr[g + 1] += gptr[g];
    int64_t* fill = malloc((size_t)(G + 1) * sizeof(int64_t));
    for (int64_t g = 0; g < G; ++g) fill[g] = gptr[g];
    for (int64_t i = 0; i < N; ++i)
        if (group_of[i] >= 0) grows[fill[group_of[i]]++] = (int32_t)i;
    free(fill);
}

/* ------------------------------------------------------------------ */
/* the orthogonal-group sweep (Eq. 1.3 / 3.3, Algorithm 4 iteration)   */
/* ------------------------------------------------------------------ */

static double row_dot(const int64_t* rp, const int32_t* ci, const double* v, int64_t i,
                      const double* x)
{
    double d = 0.0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) d = d + v[e] * x[ci[e]];
    return d;
}

/* One group step: y for every row of the group from the group-start x, then
 * x += sum_i y_i A_i^T with rows ascending.  y (scratch) has room for the group. */
static void group_step(const int64_t* rp, const int32_t* ci, const double* v,
                       const double* nsq, const double* f, const int32_t* rows,
                       int64_t cnt, double* x, double* y)
{
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t i = rows[t];
        y[t] = (f[i] - row_dot(rp, ci, v, i, x)) / nsq[i];
    }
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t i = rows[t];
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) x[ci[e]] = x[ci[e]] + v[e] * y[t];
    }
}

/* Group step with the projection of Eq. 1.3, x += A_tau^+ (f_tau - A_tau x),
 * for a group whose rows are not exactly orthogonal: y solves
 * (A_tau A_tau^T) y = r_tau, r_tau = f_tau - A_tau x from the group-start x,
 * by K Jacobi steps from y0 = r / ||A_i||^2,
 *   y_t <- (r_t - sum_{u != t} (A_i . A_j) y_u) / ||A_i||^2   (i = rows[t], j = rows[u]),
 * the off-diagonal Gram entries being the dot products of the group's rows
 * that share a column; then x += sum_t y_t A_i^T.  K = 0 is the simultaneous
 * step.  With every row's sum of |cos| to the others below one the Jacobi
 * steps converge to the exact solution (Gershgorin), so a large K gives the
 * pseudo-inverse projection of Eq. 1.3.  cptr/crow/cval: the column lists of
 * A; pos: N entries, all -1 (restored on return). */
static int group_step_pinv(int64_t N, const int64_t* rp, const int32_t* ci, const double* v, const double* nsq,
                           const double* f, const int32_t* rows, int64_t cnt, double* x, int32_t K,
                           const int64_t* cptr, const int32_t* crow, const double* cval, int64_t* pos)
{
    double* r = malloc((size_t)(cnt + 1) * sizeof(double));
    double* y = malloc((size_t)(cnt + 1) * sizeof(double));
    double* yn = malloc((size_t)(cnt + 1) * sizeof(double));
    int64_t* gp = calloc((size_t)cnt + 1, sizeof(int64_t));
    double* acc = calloc((size_t)cnt + 1, sizeof(double));
    char* touched = calloc((size_t)cnt + 1, 1);
    int64_t* tl = malloc((size_t)(cnt + 1) * sizeof(int64_t));
    int64_t gcap = 16 * (cnt + 1), gn = 0;
    int64_t* gu = malloc((size_t)gcap * sizeof(int64_t));
    double* gv = malloc((size_t)gcap * sizeof(double));
    int rc = ORC_OK;
    if (!r || !y || !yn || !gp || !acc || !touched || !tl || !gu || !gv) { rc = ORC_NOMEM; goto out; }
    for (int64_t t = 0; t < cnt; ++t) pos[rows[t]] = t;
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t i = rows[t];
        r[t] = f[i] - row_dot(rp, ci, v, i, x);
        y[t] = r[t] / nsq[i];
    }
    /* off-diagonal Gram entries of the group, row by row (partners ascending) */
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t i = rows[t], nt = 0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
            for (int64_t q = cptr[ci[e]]; q < cptr[ci[e] + 1]; ++q) {
                int64_t u = pos[crow[q]];
                if (u < 0 || u == t) continue;
                if (!touched[u]) { touched[u] = 1; acc[u] = 0.0; tl[nt++] = u; }
                acc[u] = acc[u] + v[e] * cval[q];
            }
        /* ascending partner order */
        for (int64_t a = 1; a < nt; ++a) {
            int64_t key = tl[a], b = a - 1;
            while (b >= 0 && tl[b] > key) { tl[b + 1] = tl[b]; --b; }
            tl[b + 1] = key;
        }
        for (int64_t a = 0; a < nt; ++a) {
            int64_t u = tl[a];
            touched[u] = 0;
            if (acc[u] == 0.0) continue;
            if (gn == gcap) {
                gcap *= 2;
                int64_t* nu = realloc(gu, (size_t)gcap * sizeof(int64_t));
                double* nv = realloc(gv, (size_t)gcap * sizeof(double));
                if (!nu || !nv) { free(nu ? nu : gu); free(nv ? nv : gv); gu = NULL; gv = NULL; rc = ORC_NOMEM; goto out; }
                gu = nu; gv = nv;
            }
            gu[gn] = u; gv[gn] = acc[u]; ++gn;
        }
        gp[t + 1] = gn;
    }
    for (int32_t k = 0; k < K; ++k) {
        for (int64_t t = 0; t < cnt; ++t) {
            double sacc = r[t];
            for (int64_t a = gp[t]; a < gp[t + 1]; ++a) sacc = sacc - gv[a] * y[gu[a]];
            yn[t] = sacc / nsq[rows[t]];
        }
        double* tmp = y; y = yn; yn = tmp;
    }
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t i = rows[t];
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) x[ci[e]] = x[ci[e]] + v[e] * y[t];
    }
out:
    for (int64_t t = 0; t < cnt; ++t) pos[rows[t]] = -1;
    (void)N;
    free(r); free(y); free(yn); free(gp); free(acc); free(touched); free(tl); free(gu); free(gv);
    return rc;
}

/* column lists of A (rows ascending) with values */
static int build_columns(int64_t N, const int64_t* rp, const int32_t* ci, const double* v, int64_t** cptr,
                         int32_t** crow, double** cval)
{
    int64_t nnz = rp[N];
    *cptr = calloc((size_t)N + 1, sizeof(int64_t));
    *crow = malloc((size_t)(nnz + 1) * sizeof(int32_t));
    *cval = malloc((size_t)(nnz + 1) * sizeof(double));
    int64_t* fill = malloc((size_t)(N + 1) * sizeof(int64_t));
    if (!*cptr || !*crow || !*cval || !fill) { free(fill); return ORC_NOMEM; }
    for (int64_t e = 0; e < nnz; ++e) (*cptr)[ci[e] + 1]++;
    for (int64_t c = 0; c < N; ++c) (*cptr)[c + 1] += (*cptr)[c];
    for (int64_t c = 0; c < N; ++c) fill[c] = (*cptr)[c];
    for (int64_t i = 0; i < N; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            int64_t q = fill[ci[e]]++;
            (*crow)[q] = (int32_t)i;
            (*cval)[q] = v[e];
        }
    free(fill);
    return ORC_OK;
}

/* Single group step of Eq. 1.3 with K Jacobi steps, exposed for tests. */
int orc_group_step_pinv(int64_t N, const int64_t* rp, const int32_t* ci, const double* v, const double* nsq,
                        const double* f, const int32_t* rows, int64_t cnt, double* x, int32_t K)
{
    int64_t* cptr = NULL; int32_t* crow = NULL; double* cval = NULL;
    int64_t* pos = malloc((size_t)(N + 1) * sizeof(int64_t));
    int rc = build_columns(N, rp, ci, v, &cptr, &crow, &cval);
    if (rc == ORC_OK && !pos) rc = ORC_NOMEM;
    if (rc == ORC_OK) {
        for (int64_t i = 0; i < N; ++i) pos[i] = -1;
        rc = group_step_pinv(N, rp, ci, v, nsq, f, rows, cnt, x, K, cptr, crow, cval, pos);
    }
    free(cptr); free(crow); free(cval); free(pos);
    return rc;
}

/* nsweeps full sweeps over groups 0..G-1 in order. */
int orc_sweep(int64_t N, const int64_t* rp, const int32_t* ci, const double* v,
              const double* nsq, const double* f, int64_t G, const int64_t* gptr,
              const int32_t* grows, double* x, int64_t nsweeps)
{
    (void)N;
    int64_t maxc = 1;
    for (int64_t g = 0; g < G; ++g)
        if (gptr[g + 1] - gptr[g] > maxc) maxc = gptr[g + 1] - gptr[g];
    double* y = malloc((size_t)maxc * sizeof(double));
    if (!y) return ORC_NOMEM;
    for (int64_t s = 0; s < nsweeps; ++s)
        for (int64_t g = 0; g < G; ++g)
            group_step(rp, ci, v, nsq, f, grows + gptr[g], gptr[g + 1] - gptr[g], x, y);
    free(y);
    return ORC_OK;
}

/* Single group step exposed for tests (group given as a row list). */
int orc_group_step(const int64_t* rp, const int32_t* ci, const double* v, const double* nsq,
                   const double* f, const int32_t* rows, int64_t cnt, double* x)
{
    double* y = malloc((size_t)(cnt + 1) * sizeof(double));
    if (!y) return ORC_NOMEM;
    group_step(rp, ci, v, nsq, f, rows, cnt, x, y);
    free(y);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* residual ||f - A x|| / ||f||                                        */
/* ------------------------------------------------------------------ */

double orc_residual(int64_t N, const int64_t* rp, const int32_t* ci, const double* v,
                    const double* f, const double* x)
{
    double rr = 0.0, ff = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double r = f[i] - row_dot(rp, ci, v, i, x);
        rr = rr + r * r;
        ff = ff + f[i] * f[i];
    }
    if (ff == 0.0) return sqrt(rr);
    return sqrt(rr) / sqrt(ff);
}

/* ------------------------------------------------------------------ */
/* whole solve                                                         */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t sweeps;
    double rel_res;
    int64_t groups;
    int64_t bandwidth_before;
    int64_t bandwidth_after;
    int64_t n_conflicts;
    int64_t outer_iters;
    int64_t status;
} orc_info;

typedef struct {
    int32_t check_every;   /* residual checked after every check_every-th sweep */
    int32_t precision;     /* 0 = FP64 sweeps, 1 = FP32 inner sweeps + FP64 refinement */
    int32_t inner_sweeps;  /* FP32 sweeps per refinement step */
    int32_t max_outer;     /* refinement steps at most */
    double stagnation;     /* stop (not converged) when rr moved less than this over 10 checks */
    int32_t pinv_iters;    /* > 0: group steps of Eq. 1.3 with this many Jacobi steps (FP64 form) */
    int32_t reserved;
} orc_opts;

/* Adaptive residual-check schedule (a stopping-test cadence, not part of the
 * paper's method): from the last two checks (sweeps s_prev < s, residuals
 * rr_prev > rr) the linear rate predicts k more sweeps to reach tol; the next
 * check comes after min(k, s) sweeps, or after one sweep without a rate. */
static int64_t next_check(int64_t s, double rr, int64_t s_prev, double rr_prev, double tol)
{
    int64_t step = 1;
    if (s_prev > 0 && rr < rr_prev && rr > tol && rr > 0.0) {
        double rate = pow(rr / rr_prev, 1.0 / (double)(s - s_prev));
        if (rate > 0.0 && rate < 1.0) {
            double k = ceil(log(tol / rr) / log(rate));
            if (k > (double)s) k = (double)s;
            if (k > 1.0) step = (int64_t)k;
        }
    }
    return s + step;
}

/* Setup shared by both precisions: extend, RCM, permute, norms, groups. */
typedef struct {
    int64_t N;
    int64_t* rp; int32_t* ci; double* v; /* A~ */
    double* f; double* x;                /* f~, x~ */
    int32_t* perm;
    double* nsq;
    int32_t* group_of;
    int64_t G; int64_t* gptr; int32_t* grows;
} orc_sys;

static void sys_free(orc_sys* s)
{
    free(s->rp); free(s->ci); free(s->v); free(s->f); free(s->x); free(s->perm);
    free(s->nsq); free(s->group_of); free(s->gptr); free(s->grows);
}

static int sys_setup(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci,
                     const double* v, const double* f, const double* x0, double thr,
                     orc_sys* s, orc_info* info)
{
    memset(s, 0, sizeof(*s));
    int64_t nnz = rp[m];
    int64_t N = m > n ? m : n;
    s->N = N;
    int64_t* rph = malloc(((size_t)N + 1) * sizeof(int64_t));
    double* fh = malloc((size_t)N * sizeof(double));
    double* xh = malloc((size_t)N * sizeof(double));
    s->rp = malloc(((size_t)N + 1) * sizeof(int64_t));
    s->ci = malloc((size_t)(nnz + 1) * sizeof(int32_t));
    s->v = malloc((size_t)(nnz + 1) * sizeof(double));
    s->f = malloc((size_t)N * sizeof(double));
    s->x = malloc((size_t)N * sizeof(double));
    s->perm = malloc((size_t)N * sizeof(int32_t));
    s->nsq = malloc((size_t)N * sizeof(double));
    s->group_of = malloc((size_t)N * sizeof(int32_t));
    if (!rph || !fh || !xh || !s->rp || !s->ci || !s->v || !s->f || !s->x || !s->perm ||
        !s->nsq || !s->group_of) {
        free(rph); free(fh); free(xh); sys_free(s);
        return ORC_NOMEM;
    }
    orc_extend(m, n, rp, f, x0, rph, fh, xh);
    info->bandwidth_before = orc_bandwidth(N, rph, ci);
    int rc = orc_rcm(N, rph, ci, s->perm);
    if (!rc) rc = orc_permute(N, rph, ci, v, s->perm, s->rp, s->ci, s->v);
    if (!rc) {
        for (int64_t k = 0; k < N; ++k) { s->f[k] = fh[s->perm[k]]; s->x[k] = xh[s->perm[k]]; }
        info->bandwidth_after = orc_bandwidth(N, s->rp, s->ci);
        orc_row_norms(N, s->rp, s->v, s->nsq);
        rc = orc_group_build(N, s->rp, s->ci, s->v, s->nsq, thr, s->group_of, &s->G,
                             &info->n_conflicts);
    }
    if (!rc) {
        s->gptr = malloc(((size_t)s->G + 1) * sizeof(int64_t));
        s->grows = malloc(((size_t)N + 1) * sizeof(int32_t));
        if (!s->gptr || !s->grows) rc = ORC_NOMEM;
        else orc_group_lists(N, s->group_of, s->G, s->gptr, s->grows);
        info->groups = s->G;
    }
    free(rph); free(fh); free(xh);
    if (rc) sys_free(s);
    return rc;
}

static void sys_unpermute(const orc_sys* s, int64_t n, double* x_out)
{
    double* xh = malloc((size_t)s->N * sizeof(double));
    for (int64_t k = 0; k < s->N; ++k) xh[s->perm[k]] = s->x[k];
    for (int64_t i = 0; i < n; ++i) x_out[i] = xh[i];
    free(xh);
}

/* One FP32 inner sweep on A32 d = b32: y_i = (b_i - A32_i d) * inv32_i (float
 * arithmetic), then d += sum y_i A32_i^T. */
static void sweep_fp32(const orc_sys* s, const float* v32, const float* inv32, const float* b,
                       float* d, float* y)
{
    for (int64_t g = 0; g < s->G; ++g) {
        const int32_t* rows = s->grows + s->gptr[g];
        int64_t cnt = s->gptr[g + 1] - s->gptr[g];
        for (int64_t t = 0; t < cnt; ++t) {
            int64_t i = rows[t];
            float dot = 0.0f;
            for (int64_t e = s->rp[i]; e < s->rp[i + 1]; ++e) dot = dot + v32[e] * d[s->ci[e]];
            y[t] = (b[i] - dot) * inv32[i];
        }
        for (int64_t t = 0; t < cnt; ++t) {
            int64_t i = rows[t];
            for (int64_t e = s->rp[i]; e < s->rp[i + 1]; ++e)
                d[s->ci[e]] = d[s->ci[e]] + v32[e] * y[t];
        }
    }
}

int orc_solve(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
              const double* f, const double* x0, double thr, double tol, int64_t maxit,
              const orc_opts* opts, double* x_out, orc_info* info, int32_t* perm_out,
              int32_t* group_of_out)
{
    memset(info, 0, sizeof(*info));
    int64_t nnz = rp[m];
    if (orc_validate(m, n, rp, ci, v, nnz) != ORC_OK) return ORC_INVALID;
    if (!(thr > 0.0 && thr <= 1.0) || !(tol > 0.0) || maxit < 1) return ORC_INVALID;
    for (int64_t i = 0; i < m; ++i)
        if (!isfinite(f[i])) return ORC_INVALID;
    /* check_every > 0: fixed cadence; < 0: adaptive schedule (next_check) */
    int32_t check_every = opts && opts->check_every != 0 ? opts->check_every : 1;
    double stag = opts ? opts->stagnation : 0.0;

    orc_sys s;
    int rc = sys_setup(m, n, rp, ci, v, f, x0, thr, &s, info);
    if (rc) return rc;
    if (perm_out) memcpy(perm_out, s.perm, (size_t)s.N * sizeof(int32_t));
    if (group_of_out) memcpy(group_of_out, s.group_of, (size_t)s.N * sizeof(int32_t));

    int status = ORC_NOT_CONVERGED;
    double rr = orc_residual(s.N, s.rp, s.ci, s.v, s.f, s.x);
    double hist[10];
    int64_t nchk = 0;
    if (rr <= tol) status = ORC_OK;

    if (status != ORC_OK && (!opts || opts->precision == 0)) {
        int64_t maxc = 1;
        for (int64_t g = 0; g < s.G; ++g)
            if (s.gptr[g + 1] - s.gptr[g] > maxc) maxc = s.gptr[g + 1] - s.gptr[g];
        double* y = malloc((size_t)maxc * sizeof(double));
        int32_t K = opts ? opts->pinv_iters : 0;
        int64_t* cptr = NULL; int32_t* crow = NULL; double* cval = NULL; int64_t* pos = NULL;
        if (K > 0) {
            pos = malloc((size_t)(s.N + 1) * sizeof(int64_t));
            if (!pos || build_columns(s.N, s.rp, s.ci, s.v, &cptr, &crow, &cval) != ORC_OK) {
                free(y); free(pos); free(cptr); free(crow); free(cval);
                sys_free(&s);
                return ORC_NOMEM;
            }
            for (int64_t i = 0; i < s.N; ++i) pos[i] = -1;
        }
        int64_t next = 1, s_prev = 0;
        double rr_prev = rr;
        for (int64_t sw = 1; sw <= maxit; ++sw) {
            for (int64_t g = 0; g < s.G; ++g) {
                if (K > 0)
                    group_step_pinv(s.N, s.rp, s.ci, s.v, s.nsq, s.f, s.grows + s.gptr[g], s.gptr[g + 1] - s.gptr[g],
                                    s.x, K, cptr, crow, cval, pos);
                else
                    group_step(s.rp, s.ci, s.v, s.nsq, s.f, s.grows + s.gptr[g], s.gptr[g + 1] - s.gptr[g], s.x, y);
            }
            info->sweeps = sw;
            int check = check_every > 0 ? (sw % check_every == 0 || sw == maxit) : (sw >= next || sw == maxit);
            if (check) {
                rr = orc_residual(s.N, s.rp, s.ci, s.v, s.f, s.x);
                if (rr <= tol) { status = ORC_OK; break; }
                if (stag > 0.0) {
                    if (nchk >= 10 && fabs(rr - hist[nchk % 10]) < stag) break;
                    hist[nchk % 10] = rr;
                    nchk++;
                }
                next = next_check(sw, rr, s_prev, rr_prev, tol);
                s_prev = sw;
                rr_prev = rr;
            }
        }
        free(y); free(pos); free(cptr); free(crow); free(cval);
    } else if (status != ORC_OK) {
        /* precision form: FP64 residual and correction, FP32 inner sweeps */
        int64_t N = s.N;
        int32_t s_in = opts->inner_sweeps > 0 ? opts->inner_sweeps : 4;
        int32_t max_outer = opts->max_outer > 0 ? opts->max_outer : 100;
        float* v32 = malloc((size_t)(nnz + 1) * sizeof(float));
        float* inv32 = malloc((size_t)N * sizeof(float));
        float* b = malloc((size_t)N * sizeof(float));
        float* d = malloc((size_t)N * sizeof(float));
        float* y = malloc((size_t)N * sizeof(float));
        double* r = malloc((size_t)N * sizeof(double));
        for (int64_t e = 0; e < nnz; ++e) v32[e] = (float)s.v[e];
        for (int64_t i = 0; i < N; ++i) inv32[i] = s.nsq[i] > 0.0 ? (float)(1.0 / s.nsq[i]) : 0.0f;
        for (int64_t it = 1; it <= max_outer && info->sweeps < maxit; ++it) {
            /* FP64 residual of the current x (rr was checked against tol already) */
            double rsq = 0.0;
            for (int64_t i = 0; i < N; ++i) {
                r[i] = s.f[i] - row_dot(s.rp, s.ci, s.v, i, s.x);
                rsq = rsq + r[i] * r[i];
            }
            double beta = sqrt(rsq);
            for (int64_t i = 0; i < N; ++i) { b[i] = (float)(r[i] / beta); d[i] = 0.0f; }
            for (int32_t k = 0; k < s_in && info->sweeps < maxit; ++k) {
                sweep_fp32(&s, v32, inv32, b, d, y);
                info->sweeps++;
            }
            for (int64_t i = 0; i < N; ++i) s.x[i] = s.x[i] + beta * (double)d[i];
            info->outer_iters = it;
            rr = orc_residual(N, s.rp, s.ci, s.v, s.f, s.x);
            if (rr <= tol) { status = ORC_OK; break; }
        }
        free(v32); free(inv32); free(b); free(d); free(y); free(r);
    }
    info->rel_res = rr;
    info->status = status;
    sys_unpermute(&s, n, x_out);
    sys_free(&s);
    return status;
}

/* Setup only (extend, RCM, permute, norms, groups), exported for comparisons of
 * each intermediate.  Caller-allocated outputs: perm[N], rp_t[N+1], ci_t[nnz],
 * v_t[nnz], f_t[N], x_t[N], nsq[N], group_of[N]; *G receives the group count. */
int orc_setup_export(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci,
                     const double* v, const double* f, const double* x0, double thr,
                     int32_t* perm, int64_t* rp_t, int32_t* ci_t, double* v_t, double* f_t,
                     double* x_t, double* nsq, int32_t* group_of, int64_t* G, orc_info* info)
{
    memset(info, 0, sizeof(*info));
    int64_t nnz = rp[m];
    if (orc_validate(m, n, rp, ci, v, nnz) != ORC_OK) return ORC_INVALID;
    orc_sys s;
    int rc = sys_setup(m, n, rp, ci, v, f, x0, thr, &s, info);
    if (rc) return rc;
    int64_t N = s.N;
    memcpy(perm, s.perm, (size_t)N * sizeof(int32_t));
    memcpy(rp_t, s.rp, ((size_t)N + 1) * sizeof(int64_t));
    memcpy(ci_t, s.ci, (size_t)nnz * sizeof(int32_t));
    memcpy(v_t, s.v, (size_t)nnz * sizeof(double));
    memcpy(f_t, s.f, (size_t)N * sizeof(double));
    memcpy(x_t, s.x, (size_t)N * sizeof(double));
    memcpy(nsq, s.nsq, (size_t)N * sizeof(double));
    memcpy(group_of, s.group_of, (size_t)N * sizeof(int32_t));
    *G = s.G;
    sys_free(&s);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* The paper-literal block form (Section 3.3, Algorithm 4)             */
/* ------------------------------------------------------------------ */

/* rows of block b of k uniform chunks of N rows: the first k - 1 take
 * floor(N / k) rows each in order, the last the rest */
static void block_range(int64_t N, int32_t k, int32_t b, int64_t* b0, int64_t* b1)
{
    int64_t w = N / k;
    *b0 = (int64_t)b * w;
    *b1 = b == k - 1 ? N : *b0 + w;
}

/* Classes of Algorithm 4: centroid of block i = mean of its rows; blocks i
 * and j are orthogonal when |cos(centroid_i, centroid_j)| < thr (a zero
 * centroid is orthogonal to everything); for i = 0..k-1 in order, a block not
 * yet in a class is paired with the first later block, not yet in a class,
 * orthogonal to it.  pairs[2p], pairs[2p+1] for p < *np; the blocks left over
 * form Nclass, nclass[q] for q < *nq (ascending). */
int orc_block_classes(int64_t N, const int64_t* rp, const int32_t* ci, const double* v, int32_t k, double thr,
                      int32_t* pairs, int32_t* np, int32_t* nclass, int32_t* nq)
{
    double* cen = calloc((size_t)k * (size_t)N + 1, sizeof(double));
    double* nrm = calloc((size_t)k + 1, sizeof(double));
    char* used = calloc((size_t)k + 1, 1);
    if (!cen || !nrm || !used) { free(cen); free(nrm); free(used); return ORC_NOMEM; }
    for (int32_t b = 0; b < k; ++b) {
        int64_t b0, b1;
        block_range(N, k, b, &b0, &b1);
        double* cb = cen + (size_t)b * (size_t)N;
        for (int64_t i = b0; i < b1; ++i)
            for (int64_t e = rp[i]; e < rp[i + 1]; ++e) cb[ci[e]] = cb[ci[e]] + v[e];
        double cnt = (double)(b1 - b0);
        for (int64_t c = 0; c < N; ++c) cb[c] = cb[c] / cnt;
        double q = 0.0;
        for (int64_t c = 0; c < N; ++c) q = q + cb[c] * cb[c];
        nrm[b] = sqrt(q);
    }
    *np = 0;
    for (int32_t i = 0; i < k; ++i) {
        if (used[i]) continue;
        for (int32_t j = i + 1; j < k; ++j) {
            if (used[j]) continue;
            double g = 0.0;
            const double* a = cen + (size_t)i * (size_t)N;
            const double* b = cen + (size_t)j * (size_t)N;
            for (int64_t c = 0; c < N; ++c) g = g + a[c] * b[c];
            double den = nrm[i] * nrm[j];
            double cosv = den > 0.0 ? g / den : 0.0;
            if (fabs(cosv) < thr) {
                pairs[2 * *np] = i;
                pairs[2 * *np + 1] = j;
                (*np)++;
                used[i] = used[j] = 1;
                break;
            }
        }
    }
    *nq = 0;
    for (int32_t i = 0; i < k; ++i)
        if (!used[i]) nclass[(*nq)++] = i;
    free(cen); free(nrm); free(used);
    return ORC_OK;
}

/* x += A_b^+ (f_b - A_b x) for the rows [b0, b1) of A, the minimum-norm
 * correction computed by CGLS on min ||A_b d - r|| from d = 0 (which converges
 * to A_b^+ r): stops when ||A_b^T (r - A_b d)|| <= inner_tol ||A_b^T r|| or after
 * inner_max steps.  w: 3 N + 2 (b1 - b0) doubles of scratch.  Returns the
 * number of CGLS steps. */
static int64_t block_project(int64_t N, const int64_t* rp, const int32_t* ci, const double* v, const double* f,
                             int64_t b0, int64_t b1, double* x, int32_t inner_max, double inner_tol, double* w)
{
    int64_t B = b1 - b0;
    double* d = w;
    double* p = w + N;
    double* sv = w + 2 * N;
    double* r = w + 3 * N;
    double* q = r + B;
    for (int64_t c = 0; c < N; ++c) { d[c] = 0.0; sv[c] = 0.0; }
    for (int64_t t = 0; t < B; ++t) {
        int64_t i = b0 + t;
        double a = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) a = a + v[e] * x[ci[e]];
        r[t] = f[i] - a;
    }
    for (int64_t t = 0; t < B; ++t)
        for (int64_t e = rp[b0 + t]; e < rp[b0 + t + 1]; ++e) sv[ci[e]] = sv[ci[e]] + v[e] * r[t];
    double gamma = 0.0;
    for (int64_t c = 0; c < N; ++c) { p[c] = sv[c]; gamma = gamma + sv[c] * sv[c]; }
    double gamma0 = gamma;
    int64_t it = 0;
    while (it < inner_max && gamma > inner_tol * inner_tol * gamma0 && gamma > 0.0) {
        double qq = 0.0;
        for (int64_t t = 0; t < B; ++t) {
            int64_t i = b0 + t;
            double a = 0.0;
            for (int64_t e = rp[i]; e < rp[i + 1]; ++e) a = a + v[e] * p[ci[e]];
            q[t] = a;
            qq = qq + a * a;
        }
        if (qq == 0.0) break;
        double alpha = gamma / qq;
        for (int64_t c = 0; c < N; ++c) d[c] = d[c] + alpha * p[c];
        for (int64_t t = 0; t < B; ++t) r[t] = r[t] - alpha * q[t];
        for (int64_t c = 0; c < N; ++c) sv[c] = 0.0;
        for (int64_t t = 0; t < B; ++t)
            for (int64_t e = rp[b0 + t]; e < rp[b0 + t + 1]; ++e) sv[ci[e]] = sv[ci[e]] + v[e] * r[t];
        double gn = 0.0;
        for (int64_t c = 0; c < N; ++c) gn = gn + sv[c] * sv[c];
        double beta = gn / gamma;
        for (int64_t c = 0; c < N; ++c) p[c] = sv[c] + beta * p[c];
        gamma = gn;
        ++it;
    }
    for (int64_t c = 0; c < N; ++c) x[c] = x[c] + d[c];
    return it;
}

/* Single block projection exposed for tests. */
int orc_block_project(int64_t N, const int64_t* rp, const int32_t* ci, const double* v, const double* f, int64_t b0,
                      int64_t b1, double* x, int32_t inner_max, double inner_tol)
{
    double* w = malloc((size_t)(3 * N + 2 * (b1 - b0) + 1) * sizeof(double));
    if (!w) return ORC_NOMEM;
    block_project(N, rp, ci, v, f, b0, b1, x, inner_max, inner_tol, w);
    free(w);
    return ORC_OK;
}

/* Algorithm 4 as printed: extend, RCM, permute; k uniform blocks, their
 * classes (orc_block_classes); iteration j projects onto the blocks of the
 * pair j mod P one after the other, then onto the Nclass block j mod Q (either
 * step is skipped when its class list is empty); the relative residual is
 * checked after every iteration (info->sweeps counts iterations).  x = P^T x~
 * then x^(1:n). */
int orc_solve_blocks(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                     const double* f, const double* x0, int32_t k, double thr, double tol, int64_t maxit,
                     int32_t inner_max, double inner_tol, double* x_out, orc_info* info, int32_t* np_out,
                     int32_t* nq_out)
{
    memset(info, 0, sizeof(*info));
    int64_t nnz = rp[m];
    if (orc_validate(m, n, rp, ci, v, nnz) != ORC_OK) return ORC_INVALID;
    int64_t N0 = m > n ? m : n;
    if (k < 1 || k > N0 || !(thr > 0.0 && thr <= 1.0) || !(tol > 0.0) || maxit < 1 || inner_max < 1)
        return ORC_INVALID;
    orc_sys s;
    int rc = sys_setup(m, n, rp, ci, v, f, x0, thr, &s, info);
    if (rc) return rc;
    int64_t N = s.N;
    int32_t* pairs = malloc((size_t)(2 * k + 2) * sizeof(int32_t));
    int32_t* nclass = malloc((size_t)(k + 1) * sizeof(int32_t));
    double* w = malloc((size_t)(5 * N + 2) * sizeof(double));
    int32_t np = 0, nq = 0;
    if (!pairs || !nclass || !w) rc = ORC_NOMEM;
    if (!rc) rc = orc_block_classes(N, s.rp, s.ci, s.v, k, thr, pairs, &np, nclass, &nq);
    int status = ORC_NOT_CONVERGED;
    if (!rc) {
        double rr = orc_residual(N, s.rp, s.ci, s.v, s.f, s.x);
        if (rr <= tol) status = ORC_OK;
        for (int64_t j = 0; status != ORC_OK && j < maxit; ++j) {
            int64_t b0, b1;
            if (np > 0) {
                int32_t pp = (int32_t)(j % np);
                for (int h = 0; h < 2; ++h) {
                    block_range(N, k, pairs[2 * pp + h], &b0, &b1);
                    block_project(N, s.rp, s.ci, s.v, s.f, b0, b1, s.x, inner_max, inner_tol, w);
                }
            }
            if (nq > 0) {
                block_range(N, k, nclass[j % nq], &b0, &b1);
                block_project(N, s.rp, s.ci, s.v, s.f, b0, b1, s.x, inner_max, inner_tol, w);
            }
            info->sweeps = j + 1;
            rr = orc_residual(N, s.rp, s.ci, s.v, s.f, s.x);
            if (rr <= tol) status = ORC_OK;
        }
        info->rel_res = rr;
        sys_unpermute(&s, n, x_out);
    }
    info->status = status;
    if (np_out) *np_out = np;
    if (nq_out) *nq_out = nq;
    free(pairs); free(nclass); free(w);
    sys_free(&s);
    return rc ? rc : status;
}
