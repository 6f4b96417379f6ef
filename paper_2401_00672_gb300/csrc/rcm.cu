// rcm.cu -- Reverse Cuthill-McKee reordering on the GPU (paper Section 3.2,
// Eq. 3.1-3.2; the paper names RCM without its steps).
//
// Reading implemented (and matched bit for bit by the tests):
//   graph      pattern(A + A^T) without self loops; deg(v) = distinct neighbours
//   start      per connected component, George-Liu pseudo-peripheral search grown
//              from the component's minimum-(deg, index) vertex: root v, last BFS
//              level's minimum-(deg, index) vertex u; move to u while its
//              eccentricity is larger
//   order      Cuthill-McKee from the root, children appended in (deg, index)
//              order; components in order of their minimum-(deg, index) vertex;
//              the whole list is reversed once.
//
// GPU formulation:
//   * every vertex gets its rank r(v) in (deg, index) order, and every
//     adjacency list is sorted by r, so "children in (deg, index) order" is a
//     linear scan;
//   * components are labelled by min-hooking (label = smallest vertex index);
//   * all components run their breadth-first searches at the same time
//     (level-synchronous, cooperative kernels with bounded grid barriers);
//   * Cuthill-McKee levels: the frontier F_L is kept sorted by (component,
//     CM position).  A newly reached vertex w takes as parent the frontier
//     vertex of smallest frontier index (atomicMin), which is the earliest
//     placed neighbour of sequential Cuthill-McKee; children are then written
//     contiguously after an exclusive scan of per-parent child counts, in the
//     r order of the parent's adjacency list.  This reproduces the sequential
//     queue order exactly;
//   * the Cuthill-McKee pass overlaps the root search: it runs on a second
//     stream, beside the search's BFS, from the roots a search round would end
//     with, and is kept when the search ends with exactly those roots.
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace obk {
namespace {

constexpr int kBlock = 256;
constexpr int kCoopBlock = 512;      // cooperative kernels: 512 threads,
constexpr int kCoopBlocksPerSm = 2;  // two blocks per SM
constexpr int32_t kUnvisited = -1;
// level count of the first search from which the overlapped Cuthill-McKee pass
// starts from the first candidates
constexpr int32_t kEarlyPassLevels = 32;

// ---- symmetric graph: pattern(A + A^T) minus self loops -----------------------

// Merge row i of A (sorted columns) with row i of A^T (sorted rows of column i):
// the union without i.  Pass 0 counts, pass 1 writes.
template <bool kWrite>
__global__ void merge_sym(int64_t N, const int64_t* rp, const int32_t* ci, const int64_t* tp,
                          const uint32_t* tr, const int64_t* gp, int64_t* deg, int32_t* adj)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t a = rp[i], ae = rp[i + 1], b = tp[i], be = tp[i + 1];
        int64_t out = kWrite ? gp[i] : 0, cnt = 0;
        int64_t last = -1;
        while (a < ae || b < be) {
            int64_t va = a < ae ? (int64_t)ci[a] : INT64_MAX;
            int64_t vb = b < be ? (int64_t)tr[b] : INT64_MAX;
            int64_t v;
            if (va <= vb) { v = va; ++a; if (va == vb) ++b; }
            else { v = vb; ++b; }
            if (v == i || v == last) continue;
            last = v;
            if (kWrite) adj[out + cnt] = (int32_t)v;
            ++cnt;
        }
        if (!kWrite) deg[i] = cnt;
    }
}

// A structurally symmetric pattern is its own transpose, so the graph is each
// row without its diagonal entry.  Count: the row length less one when the
// (sorted) row holds i.
__global__ void drop_self_count(int64_t N, const int64_t* rp, const int32_t* ci, int64_t* deg)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = rp[i], hi = rp[i + 1];
        const int64_t len = hi - lo;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if ((int64_t)ci[mid] < i) lo = mid + 1;
            else hi = mid;
        }
        deg[i] = len - (lo < rp[i + 1] && (int64_t)ci[lo] == i ? 1 : 0);
    }
}

// Copy: one warp per row, the lanes over its entries in order; an entry after
// the diagonal moves back by one.
__global__ void drop_self_copy(int64_t N, const int64_t* rp, const int32_t* ci, const int64_t* gp, int32_t* adj)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < N; i += nw) {
        const int64_t b = rp[i], e1 = rp[i + 1], out = gp[i];
        int64_t shift = 0;
        for (int64_t e0 = b; e0 < e1; e0 += 32) {
            const int64_t e = e0 + lane;
            const int32_t c = e < e1 ? ci[e] : -1;
            const unsigned self = __ballot_sync(0xffffffffu, e < e1 && (int64_t)c == i);
            const int64_t before = shift + __popc(self & ((1u << lane) - 1u));
            if (e < e1 && (int64_t)c != i) adj[out + (e - b) - before] = c;
            shift += __popc(self);
        }
    }
}

// ---- ranks in (deg, index) order ---------------------------------------------

__global__ void deg_keys(int64_t N, const int64_t* gp, uint64_t* keys, uint32_t* vals, unsigned long long* dmax)
{
    unsigned long long mx = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
         v += (int64_t)gridDim.x * blockDim.x) {
        uint64_t d = (uint64_t)(gp[v + 1] - gp[v]);
        keys[v] = d;
        vals[v] = (uint32_t)v;
        mx = d > mx ? d : mx;
    }
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = t > mx ? t : mx;
    }
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(dmax, mx);
}

__global__ void rank_of(int64_t N, const uint32_t* by_rank, int32_t* r)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x)
        r[by_rank[k]] = (int32_t)k;
}

__global__ void adj_rank_keys(int64_t M, const int32_t* adj, const int32_t* r, uint32_t* keys,
                              uint32_t* vals)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < M;
         e += (int64_t)gridDim.x * blockDim.x) {
        keys[e] = (uint32_t)r[adj[e]];
        vals[e] = (uint32_t)adj[e];
    }
}

// Warp-aggregated per-component max / min / add: when every lane of the warp
// holds the same component label one lane issues the atomic.
__device__ __forceinline__ void agg_max(int32_t* arr, int32_t lab, int32_t val, bool act)
{
    unsigned am = __ballot_sync(0xffffffffu, act);
    if (!am) return;
    int32_t l0 = __shfl_sync(0xffffffffu, lab, __ffs(am) - 1);
    bool same = __all_sync(0xffffffffu, !act || lab == l0);
    if (same) {
        int32_t m = __reduce_max_sync(0xffffffffu, act ? val : INT32_MIN);
        if ((threadIdx.x & 31) == __ffs(am) - 1) atomicMax(arr + l0, m);
    } else if (act) {
        atomicMax(arr + lab, val);
    }
}
__device__ __forceinline__ void agg_min(int32_t* arr, int32_t lab, int32_t val, bool act)
{
    unsigned am = __ballot_sync(0xffffffffu, act);
    if (!am) return;
    int32_t l0 = __shfl_sync(0xffffffffu, lab, __ffs(am) - 1);
    bool same = __all_sync(0xffffffffu, !act || lab == l0);
    if (same) {
        int32_t m = __reduce_min_sync(0xffffffffu, act ? val : INT32_MAX);
        if ((threadIdx.x & 31) == __ffs(am) - 1) atomicMin(arr + l0, m);
    } else if (act) {
        atomicMin(arr + lab, val);
    }
}
__device__ __forceinline__ void agg_add(int32_t* arr, int32_t lab, int32_t val, bool act)
{
    unsigned am = __ballot_sync(0xffffffffu, act);
    if (!am) return;
    int32_t l0 = __shfl_sync(0xffffffffu, lab, __ffs(am) - 1);
    bool same = __all_sync(0xffffffffu, !act || lab == l0);
    if (same) {
        int32_t m = __reduce_add_sync(0xffffffffu, act ? val : 0);
        if ((threadIdx.x & 31) == __ffs(am) - 1) atomicAdd(arr + l0, m);
    } else if (act) {
        atomicAdd(arr + lab, val);
    }
}

// ---- connected components by min-hooking ---------------------------------------

__device__ __forceinline__ int32_t find_root(const int32_t* parent, int32_t v)
{
    int32_t p = ld_volatile_i32(parent + v);
    while (p != v) {
        v = p;
        p = ld_volatile_i32(parent + v);
    }
    return v;
}

__global__ void cc_init(int64_t N, int32_t* parent)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
         v += (int64_t)gridDim.x * blockDim.x)
        parent[v] = (int32_t)v;
}

__global__ void cc_hook(int64_t N, const int64_t* gp, const int32_t* adj, int32_t* parent, int* changed)
{
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < N;
         u += (int64_t)gridDim.x * blockDim.x) {
        for (int64_t e = gp[u]; e < gp[u + 1]; ++e) {
            int32_t w = adj[e];
            if (w <= u) continue;
            int32_t ru = find_root(parent, (int32_t)u), rw = find_root(parent, w);
            if (ru != rw) {
                int32_t hi = ru > rw ? ru : rw, lo = ru > rw ? rw : ru;
                atomicMin(parent + hi, lo);
                *changed = 1;
            }
        }
    }
}

__global__ void cc_compress(int64_t N, int32_t* parent)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
         v += (int64_t)gridDim.x * blockDim.x)
        parent[v] = find_root(parent, (int32_t)v);
}

// per component (indexed by its label): minimum rank, size
__global__ void comp_stats(int64_t N, const int32_t* label, const int32_t* r, int32_t* cmin_r,
                           int32_t* csize)
{
    for (int64_t v0 = (int64_t)blockIdx.x * blockDim.x; v0 < N; v0 += (int64_t)gridDim.x * blockDim.x) {
        int64_t v = v0 + threadIdx.x;
        bool act = v < N;
        int32_t lab = act ? label[v] : 0;
        agg_min(cmin_r, lab, act ? r[v] : 0, act);
        agg_add(csize, lab, 1, act);
    }
}

// starts[k] = 1 if the vertex of rank k is the minimum-rank vertex of its component
__global__ void comp_start_flags(int64_t N, const uint32_t* by_rank, const int32_t* label,
                                 const int32_t* cmin_r, int32_t* flag)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        int32_t v = (int32_t)by_rank[k];
        flag[k] = cmin_r[label[v]] == (int32_t)k ? 1 : 0;
    }
}

// component order: index = number of component starts of smaller rank
__global__ void comp_order(int64_t N, const uint32_t* by_rank, const int32_t* label, const int32_t* flag,
                           const int64_t* flag_scan, int32_t* cidx, int32_t* roots, int64_t* size_by_idx,
                           const int32_t* csize)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[k]) continue;
        int32_t v = (int32_t)by_rank[k];
        int32_t c = (int32_t)flag_scan[k];
        cidx[label[v]] = c;
        roots[c] = v;
        size_by_idx[c] = csize[label[v]];
    }
}

// ---- level-synchronous multi-source BFS (distances only) ------------------------

struct BfsParams {
    int64_t N;
    const int64_t* gp;
    const int32_t* adj;
    const int32_t* sources;
    int64_t nsrc;
    int32_t* dist;      // N, pre-set to kUnvisited
    int32_t* qa;        // N
    int32_t* qb;        // N
    int64_t* cnt;       // [0..2] rotating frontier counters (zeroed), [3] vertices reached
    int32_t* nlevels;   // out
    GridBarrier gb;
};

// Frontier vertices are split into contiguous chunks, one per block, so the
// scattered loads of a small frontier still spread over every SM.  Inside a
// block a group of G lanes takes one vertex, G the largest power of two up to
// 32 with chunk * G <= block size, and every lane loads kNbRound neighbours
// per round (independent loads): a level then costs a few dependent L2 round
// trips.  Vertices with more than kHeavyDeg neighbours that a small group
// would need several rounds for go to a per-block list that whole warps
// process afterwards.  Nothing inside the group loops is warp-collective.
// Newly reached vertices are collected per block in shared memory and
// appended to the next frontier with one global atomic per block and level
// (direct appends when the block buffer is full).
constexpr int kBfsBuf = 2048;
constexpr int kHeavyDeg = 32;
constexpr int kHeavyBuf = 512;
constexpr int kNbRound = 4;

__device__ __forceinline__ int group_lanes(int64_t items)
{
    int G = 32;
    while (G > 1 && (int64_t)G * items > (int64_t)blockDim.x) G >>= 1;
    return G;
}

// deferred to a warp: many neighbours for a group of G lanes
__device__ __forceinline__ bool heavy_for(int64_t deg, int G)
{
    return deg > kHeavyDeg && deg > 2 * kNbRound * G;
}

__device__ __forceinline__ void bfs_reach(const BfsParams& p, int32_t w, int L, int32_t* sbuf, int* s_cnt,
                                          int64_t* cnext, int32_t* nxt)
{
    if (atomicCAS(p.dist + w, kUnvisited, L + 1) != kUnvisited) return;
    int slot = atomicAdd(s_cnt, 1);
    if (slot < kBfsBuf) {
        sbuf[slot] = w;
    } else {
        unsigned long long pos = atomicAdd((unsigned long long*)cnext, 1ull);
        if ((int64_t)pos < p.N) nxt[pos] = w;
        else atomicCAS(p.gb.err, 0, (int)kDevOverflow);
    }
}

// lanes lg, lg + G, ... of a group of G over the neighbours [b, e) of a vertex
// (direct: narrow levels claim every neighbour with a compare-and-swap, one
// round trip to discovery; wide levels first read dist and skip the visited
// ones, sparing the atomics)
__device__ __forceinline__ void bfs_expand(const BfsParams& p, int64_t b, int64_t e, int G, int lg, int L,
                                           int32_t* sbuf, int* s_cnt, int64_t* cnext, int32_t* nxt, bool direct)
{
    for (int64_t q0 = b + lg; q0 < e; q0 += (int64_t)kNbRound * G) {
        int32_t w[kNbRound];
        int32_t d[kNbRound];
#pragma unroll
        for (int t = 0; t < kNbRound; ++t) w[t] = q0 + (int64_t)t * G < e ? p.adj[q0 + (int64_t)t * G] : -1;
#pragma unroll
        for (int t = 0; t < kNbRound; ++t)
            d[t] = (w[t] >= 0 && !direct) ? ld_volatile_i32(p.dist + w[t]) : kUnvisited;
#pragma unroll
        for (int t = 0; t < kNbRound; ++t)
            if (w[t] >= 0 && d[t] == kUnvisited) bfs_reach(p, w[t], L, sbuf, s_cnt, cnext, nxt);
    }
}

__global__ void __launch_bounds__(kCoopBlock) bfs_levels(BfsParams p)
{
    __shared__ int32_t sbuf[kBfsBuf];
    __shared__ int32_t heavy[kHeavyBuf];
    __shared__ int s_cnt, s_nheavy;
    __shared__ long long s_base;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int wpb = kCoopBlock / kWarp;
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t nth = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = tid; k < p.nsrc; k += nth) {
        p.dist[p.sources[k]] = 0;
        p.qa[k] = p.sources[k];
    }
    if (tid == 0) { p.cnt[0] = p.nsrc; p.cnt[3] = p.nsrc; }
    if (!grid_sync(p.gb)) return;
    int32_t* cur = p.qa;
    int32_t* nxt = p.qb;
    int L = 0;
    for (;;) {
        int64_t ncur = *(volatile int64_t*)(p.cnt + (L % 3));
        if (ncur == 0) break;
        if (tid == 0) {
            p.cnt[(L + 2) % 3] = 0;
            if (L > 0) p.cnt[3] += ncur;
        }
        int64_t* cnext = p.cnt + ((L + 1) % 3);
        if (threadIdx.x == 0) { s_cnt = 0; s_nheavy = 0; }
        __syncthreads();
        int64_t chunk = ceil_div(ncur, (int64_t)gridDim.x);
        int64_t c0 = (int64_t)blockIdx.x * chunk;
        int64_t c1 = c0 + chunk < ncur ? c0 + chunk : ncur;
        const int G = group_lanes(c1 - c0);
        const int lg = threadIdx.x & (G - 1);
        const int ipp = blockDim.x / G;
        // a frontier of at most a quarter of the threads counts as narrow
        const bool direct = ncur * 4 <= nth;
        for (int64_t k = c0 + threadIdx.x / G; k < c1; k += ipp) {
            int32_t u = cur[k];
            int64_t b = p.gp[u], e = p.gp[u + 1];
            if (heavy_for(e - b, G) && k - c0 < kHeavyBuf) {  // at most kHeavyBuf such vertices
                if (lg == 0) heavy[atomicAdd(&s_nheavy, 1)] = u;
                continue;
            }
            bfs_expand(p, b, e, G, lg, L, sbuf, &s_cnt, cnext, nxt, direct);
        }
        __syncthreads();
        for (int h = wid; h < s_nheavy; h += wpb) {
            int32_t u = heavy[h];
            bfs_expand(p, p.gp[u], p.gp[u + 1], 32, lane, L, sbuf, &s_cnt, cnext, nxt, direct);
        }
        __syncthreads();
        int nb = s_cnt < kBfsBuf ? s_cnt : kBfsBuf;
        if (threadIdx.x == 0) s_base = nb ? (long long)atomicAdd((unsigned long long*)cnext, (unsigned long long)nb) : 0;
        __syncthreads();
        for (int t = threadIdx.x; t < nb; t += blockDim.x) {
            int64_t pos = s_base + t;
            if (pos < p.N) nxt[pos] = sbuf[t];
            else atomicCAS(p.gb.err, 0, (int)kDevOverflow);
        }
        if (!grid_sync(p.gb)) return;
        int32_t* t = cur;
        cur = nxt;
        nxt = t;
        ++L;
    }
    if (tid == 0) *p.nlevels = L;
}

__global__ void ecc_per_comp(int64_t N, const int32_t* dist, const int32_t* label, int32_t* ecc)
{
    for (int64_t v0 = (int64_t)blockIdx.x * blockDim.x; v0 < N; v0 += (int64_t)gridDim.x * blockDim.x) {
        int64_t v = v0 + threadIdx.x;
        bool act = v < N && dist[v] >= 0;
        agg_max(ecc, act ? label[v] : 0, act ? dist[v] : 0, act);
    }
}

__global__ void last_level_min(int64_t N, const int32_t* dist, const int32_t* label, const int32_t* ecc,
                               const int32_t* r, int32_t* cand_r)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
         v += (int64_t)gridDim.x * blockDim.x)
        if (dist[v] >= 0 && dist[v] == ecc[label[v]]) atomicMin(cand_r + label[v], r[v]);
}

// George-Liu step per component (indexed by component order c).  active[c]:
// 1 while the root may still move.  Phase A (after the BFS from the roots):
// remember ecc(root) and the candidate u.  Phase B (after the BFS from the
// candidates): move when ecc(u) > ecc(root).
__global__ void gl_record_root(int64_t C, const int32_t* roots, const int32_t* label, const int32_t* ecc,
                               const int32_t* cand_r, const uint32_t* by_rank, int32_t* ecc_root,
                               int32_t* cand, const int32_t* active)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C;
         c += (int64_t)gridDim.x * blockDim.x) {
        if (!active[c]) continue;
        int32_t lab = label[roots[c]];
        ecc_root[c] = ecc[lab];
        cand[c] = (int32_t)by_rank[cand_r[lab]];
    }
}

__global__ void gl_compare(int64_t C, int32_t* roots, const int32_t* label, const int32_t* ecc,
                           const int32_t* cand_r, const uint32_t* by_rank, int32_t* ecc_root,
                           int32_t* cand, int32_t* active, int* any_active)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C;
         c += (int64_t)gridDim.x * blockDim.x) {
        if (!active[c]) continue;
        int32_t lab = label[roots[c]];
        int32_t e_u = ecc[lab];
        if (e_u > ecc_root[c]) {
            roots[c] = cand[c];
            ecc_root[c] = e_u;
            cand[c] = (int32_t)by_rank[cand_r[lab]];
            *any_active = 1;
        } else {
            active[c] = 0;
        }
    }
}

// roots_cm[c] = the root of component c if its candidate replaces it
__global__ void spec_roots(int64_t C, const int32_t* roots, const int32_t* cand, const int32_t* active,
                           int32_t* roots_cm)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C;
         c += (int64_t)gridDim.x * blockDim.x)
        roots_cm[c] = active[c] ? cand[c] : roots[c];
}

__global__ void roots_differ(int64_t C, const int32_t* a, const int32_t* b, int* differ)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C;
         c += (int64_t)gridDim.x * blockDim.x)
        if (a[c] != b[c]) *differ = 1;
}

__global__ void gather_active_sources(int64_t C, const int32_t* which, const int32_t* active, int32_t* src,
                                      int64_t* nsrc)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C;
         c += (int64_t)gridDim.x * blockDim.x)
        if (active[c]) src[atomicAdd((unsigned long long*)nsrc, 1ull)] = which[c];
}

// ---- Cuthill-McKee levels (all components at once) ----------------------------
//
// All levels live back to back in one queue Q: level L is Q[lo, hi).  Level 0
// holds the component roots in component order; inside every level the
// vertices are ordered by (component, CM position).  So Q lists, level by
// level, every component's Cuthill-McKee order interleaved; a stable partition
// of Q by component gives the concatenated order (nothing to do when
// connected).
//
// Priorities.  Every placed vertex v carries a 64-bit priority P(v) that
// orders vertices exactly as their queue positions do: a root gets its
// component index c (< 2^32) and the idx-th child (in rank order) of the
// vertex at queue position k gets ((k + 1) << 32) | idx.  Within a level this
// is (parent position, rank) order, the CM rule; every priority of level L+1
// exceeds every priority of level L because parents of level L+1 sit after
// those of level L.  claim[w] = min P over the vertices that have reached w,
// so after the vertices of level L have claimed, claim[w] = P(parent of w)
// for every w of level L+1 (later claims are larger and change nothing).
//
// Per level: (A) each frontier vertex u counts its children {w : claim[w] ==
// P(u)} -- all its neighbours lie in levels L-1..L+1, whose claims no longer
// change; (B) a look-back over the per-block child totals of this level
// (tagged with the level) gives the block's offset, and the children are
// written to Q in order with their priorities beside them; (C) every child
// records its adjacency range at its queue position and claims its
// neighbours; then one grid barrier.  A frontier vertex is read as (priority,
// adjacency range) at its queue position, one round of loads.

struct CmParams {
    int64_t N;
    const int64_t* gp;
    const int32_t* adj_r;            // adjacency sorted by rank
    const int32_t* roots;            // C roots in component order
    int64_t C;
    unsigned long long* claim;       // N, all ones
    unsigned long long* qp;          // N: priority of the vertex at each queue position
    int64_t* qb;                     // N: its first adjacency position
    int32_t* qd;                     // N: its degree
    int32_t* Q;                      // N
    int64_t* cnt;                    // N: per frontier vertex, block-local offset of its children
    unsigned long long* agg;         // gridDim: ((level + 1) << 40) | block total, zeroed
    int64_t* ntot;                   // 2: size of the next level (alternating slots)
    int64_t* nlevels;                // out: [0] levels, [1] vertices placed
    GridBarrier gb;
};

constexpr int kAggShift = 40;  // a block total is below 2^31; the tag is (level + 1) mod 2^24
constexpr unsigned long long kAggTagMask = (1ull << (64 - kAggShift)) - 1ull;

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Vertex w with priority pw claims its neighbours: lanes lg, lg + G, ... of
// a group of G, kNbRound independent loads per lane and round; neighbours
// already claimed lower are skipped without an atomic.
__device__ __forceinline__ void claim_group(const CmParams& p, int64_t b, int64_t e, int G, int lg,
                                            unsigned long long pw)
{
    for (int64_t q0 = b + lg; q0 < e; q0 += (int64_t)kNbRound * G) {
        int32_t x[kNbRound];
#pragma unroll
        for (int t = 0; t < kNbRound; ++t) x[t] = q0 + (int64_t)t * G < e ? p.adj_r[q0 + (int64_t)t * G] : -1;
        // reductions without a result: nothing waits for them before the barrier
#pragma unroll
        for (int t = 0; t < kNbRound; ++t)
            if (x[t] >= 0) atomicMin(p.claim + x[t], pw);
    }
}

constexpr int kStage = 8;  // children of one frontier vertex kept in shared memory

constexpr int kChildStage = 512;  // children of a block per level kept in shared memory

struct CmShared {
    int32_t sj[kStage][kCoopBlock];  // adjacency offset of a staged child
    int32_t sw[kStage][kCoopBlock];  // the child
    int32_t cw[kChildStage];         // the block's first children of this level
    unsigned long long cp[kChildStage];  // and their priorities
    int32_t scnt[kCoopBlock];        // children per frontier vertex of the chunk
    int64_t soff[kCoopBlock];        // their block-local offsets
    int32_t heavy[kHeavyBuf];
    int64_t wsum[kCoopBlock / kWarp];
    int64_t s_tot, s_before;
    int s_fail, s_nheavy;
};

// Children of frontier vertex k (priority pu, neighbours [b, e)) counted by a
// group of G lanes; staged mode records (offset, child) pairs per vertex in
// shared memory, otherwise counts go to p.cnt[k].
__device__ __forceinline__ void cm_count(const CmParams& p, CmShared& sh, int64_t b, int64_t e, int G, int lg,
                                         unsigned long long pu, int64_t k, int kl, bool staged)
{
    for (int64_t q0 = b + lg; q0 < e; q0 += (int64_t)kNbRound * G) {
        int32_t w[kNbRound];
        unsigned long long c[kNbRound];
#pragma unroll
        for (int t = 0; t < kNbRound; ++t) w[t] = q0 + (int64_t)t * G < e ? p.adj_r[q0 + (int64_t)t * G] : -1;
#pragma unroll
        for (int t = 0; t < kNbRound; ++t) c[t] = w[t] >= 0 ? ld_relaxed_u64(p.claim + w[t]) : ~0ull;
#pragma unroll
        for (int t = 0; t < kNbRound; ++t) {
            if (w[t] < 0 || c[t] != pu) continue;
            if (staged) {
                int slot = atomicAdd(&sh.scnt[kl], 1);
                if (slot < kStage) {
                    sh.sj[slot][kl] = (int32_t)(q0 + (int64_t)t * G - b);
                    sh.sw[slot][kl] = w[t];
                }
            } else {
                atomicAdd((unsigned long long*)(p.cnt + k), 1ull);
            }
        }
    }
}

// the idx-th child w of the vertex at queue position k goes to position pos;
// the block's first kChildStage children are also kept in shared memory
__device__ __forceinline__ void cm_place(const CmParams& p, CmShared& sh, int64_t base_pos, int64_t pos, int32_t w,
                                         int64_t k, int64_t idx)
{
    unsigned long long pw = ((unsigned long long)(k + 1) << 32) | (unsigned long long)idx;
    if (pos < p.N) {
        p.Q[pos] = w;
        p.qp[pos] = pw;
    } else {
        atomicCAS(p.gb.err, 0, (int)kDevOverflow);
    }
    int64_t l = pos - base_pos;
    if (l >= 0 && l < kChildStage) {
        sh.cw[l] = w;
        sh.cp[l] = pw;
    }
}

// Children of frontier vertex k in rank (adjacency) order, found again from
// the claims by one thread.
__device__ void cm_rescan_thread(const CmParams& p, CmShared& sh, int64_t base_pos, int64_t k, int64_t o)
{
    unsigned long long pu = p.qp[k];
    int64_t b = p.qb[k], e = b + p.qd[k];
    int64_t i = 0;
    for (int64_t q0 = b; q0 < e; q0 += 2 * kNbRound) {
        int32_t w[2 * kNbRound];
        unsigned long long c[2 * kNbRound];
#pragma unroll
        for (int t = 0; t < 2 * kNbRound; ++t) w[t] = q0 + t < e ? p.adj_r[q0 + t] : -1;
#pragma unroll
        for (int t = 0; t < 2 * kNbRound; ++t) c[t] = w[t] >= 0 ? ld_relaxed_u64(p.claim + w[t]) : ~0ull;
#pragma unroll
        for (int t = 0; t < 2 * kNbRound; ++t)
            if (w[t] >= 0 && c[t] == pu) {
                cm_place(p, sh, base_pos, o + i, w[t], k, i);
                ++i;
            }
    }
}

// The same by a whole warp (ballots keep the order).
__device__ void cm_rescan_warp(const CmParams& p, CmShared& sh, int64_t base_pos, int64_t k, int64_t o, int lane)
{
    unsigned lt = (1u << lane) - 1u;
    unsigned long long pu = p.qp[k];
    int64_t b = p.qb[k], e = b + p.qd[k];
    int64_t i = 0;
    for (int64_t base = b; base < e; base += 32) {
        int64_t q = base + lane;
        int32_t w = 0;
        bool child = false;
        if (q < e) {
            w = p.adj_r[q];
            child = ld_relaxed_u64(p.claim + w) == pu;
        }
        unsigned m = __ballot_sync(0xffffffffu, child);
        if (child) cm_place(p, sh, base_pos, o + i + __popc(m & lt), w, k, i + __popc(m & lt));
        i += __popc(m);
    }
}

__device__ __forceinline__ void cswap(int32_t& ja, int32_t& wa, int32_t& jb, int32_t& wb)
{
    if (jb < ja) {
        int32_t t = ja; ja = jb; jb = t;
        t = wa; wa = wb; wb = t;
    }
}

__global__ void __launch_bounds__(kCoopBlock) cm_levels(CmParams p)
{
    __shared__ CmShared sh;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t nth = (int64_t)gridDim.x * blockDim.x;
    int64_t gw = tid >> 5, nw = nth >> 5;
    const int wpb = kCoopBlock / kWarp;
    for (int64_t c = tid; c < p.C; c += nth) {
        int32_t r = p.roots[c];
        p.Q[c] = r;
        p.qp[c] = (unsigned long long)c;
        p.qb[c] = p.gp[r];
        p.qd[c] = (int32_t)(p.gp[r + 1] - p.gp[r]);
        p.claim[r] = (unsigned long long)c;
    }
    if (!grid_sync(p.gb)) return;
    for (int64_t c = gw; c < p.C; c += nw) {
        int32_t r = p.roots[c];
        claim_group(p, p.gp[r], p.gp[r + 1], 32, lane, (unsigned long long)c);
    }
    if (!grid_sync(p.gb)) return;
    int64_t lo = 0, hi = p.C;
    int L = 0;
    while (hi > lo) {
        int64_t F = hi - lo;
        int64_t chunk = ceil_div(F, (int64_t)gridDim.x);
        int64_t c0 = lo + (int64_t)blockIdx.x * chunk;
        int64_t c1 = c0 + chunk < hi ? c0 + chunk : hi;
        int64_t nit = c1 > c0 ? c1 - c0 : 0;
        const bool staged = nit <= (int64_t)blockDim.x;  // then chunk vertex kl has slot kl
        if (threadIdx.x == 0) sh.s_nheavy = 0;
        if (staged) sh.scnt[threadIdx.x] = 0;
        else
            for (int64_t k = c0 + threadIdx.x; k < c1; k += blockDim.x) p.cnt[k] = 0;
        __syncthreads();
        // (A) child counts: children of u are the w with claim[w] == P(u)
        {
            const int G = group_lanes(nit);
            const int lg = threadIdx.x & (G - 1);
            const int ipp = blockDim.x / G;
            for (int64_t k = c0 + threadIdx.x / G; k < c1; k += ipp) {
                int kl = (int)(k - c0);
                unsigned long long pu = p.qp[k];
                int64_t b = p.qb[k], e = b + p.qd[k];
                if (heavy_for(e - b, G) && kl < kHeavyBuf) {
                    if (lg == 0) sh.heavy[atomicAdd(&sh.s_nheavy, 1)] = kl;
                    continue;
                }
                cm_count(p, sh, b, e, G, lg, pu, k, kl, staged);
            }
        }
        __syncthreads();
        for (int h = wid; h < sh.s_nheavy; h += wpb) {
            int kl = sh.heavy[h];
            int64_t k = c0 + kl;
            cm_count(p, sh, p.qb[k], p.qb[k] + p.qd[k], 32, lane, p.qp[k], k, kl, staged);
        }
        __syncthreads();
        // block-local exclusive scan of the child counts
        int64_t carry = 0;
        for (int64_t base = c0; base < c1; base += blockDim.x) {
            int64_t k = base + threadIdx.x;
            int64_t v = k < c1 ? (staged ? (int64_t)sh.scnt[k - c0] : p.cnt[k]) : 0;
            int64_t inc = v;
            for (int o = 1; o < 32; o <<= 1) {
                int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += t;
            }
            if (lane == 31) sh.wsum[wid] = inc;
            __syncthreads();
            if (threadIdx.x == 0) {
                int64_t run = 0;
                for (int w = 0; w < wpb; ++w) {
                    int64_t t = sh.wsum[w];
                    sh.wsum[w] = run;
                    run += t;
                }
                sh.s_tot = run;
            }
            __syncthreads();
            if (k < c1) {
                int64_t off = carry + sh.wsum[wid] + inc - v;
                if (staged) sh.soff[k - c0] = off;
                else p.cnt[k] = off;
            }
            carry += sh.s_tot;
            __syncthreads();
        }
        // look-back: publish this block's total, add up the earlier blocks'
        const unsigned long long ltag = (unsigned long long)(L + 1) & kAggTagMask;
        if (threadIdx.x == 0) {
            sh.s_fail = 0;
            sh.s_nheavy = 0;
            st_release_u64(p.agg + blockIdx.x, (ltag << kAggShift) | (unsigned long long)carry);
        }
        __syncthreads();
        int64_t before = 0;
        for (unsigned j = threadIdx.x; j < blockIdx.x; j += blockDim.x) {
            long long spins = 0;
            unsigned long long a;
            for (;;) {
                asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(a) : "l"(p.agg + j) : "memory");
                if ((a >> kAggShift) == ltag) break;
                if (++spins > p.gb.limit || ((spins & 63) == 0 && ld_volatile_i32(p.gb.err) != 0)) {
                    atomicCAS(p.gb.err, 0, (int)kDevTimeout);
                    sh.s_fail = 1;
                    break;
                }
                if (spins > 20000) __nanosleep(32);
            }
            before += (int64_t)(a & ((1ull << kAggShift) - 1ull));
        }
        for (int o = 16; o > 0; o >>= 1) before += __shfl_xor_sync(0xffffffffu, before, o);
        if (lane == 0) sh.wsum[wid] = before;
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t x = 0;
            for (int w = 0; w < wpb; ++w) x += sh.wsum[w];
            sh.s_before = x;
            if (blockIdx.x == gridDim.x - 1) p.ntot[L & 1] = x + carry;
        }
        __syncthreads();
        if (sh.s_fail) return;
        int64_t boff = sh.s_before;
        if (boff < 0 || hi + boff + carry > p.N) {  // cannot happen for a valid queue; stop before any overrun
            if (threadIdx.x == 0) atomicCAS(p.gb.err, 0, (int)kDevOverflow);
            return;
        }
        const int64_t base_pos = hi + boff;
        // (B) the children in order at base_pos + offset + idx with priority
        // ((k + 1) << 32) | idx: staged lists are sorted by adjacency offset
        // (= rank order) and copied; the others are found again from the
        // claims, which no longer change for these vertices
        for (int64_t k = c0 + threadIdx.x; k < c1; k += blockDim.x) {
            int kl = (int)(k - c0);
            if (staged && sh.scnt[kl] <= kStage) {
                int n = sh.scnt[kl];
                int64_t o = base_pos + sh.soff[kl];
                int32_t j[kStage], w[kStage];
#pragma unroll
                for (int i = 0; i < kStage; ++i) {
                    j[i] = i < n ? sh.sj[i][kl] : INT32_MAX;
                    w[i] = i < n ? sh.sw[i][kl] : 0;
                }
#pragma unroll
                for (int r = 0; r < kStage; ++r)  // odd-even transposition sort of 8
#pragma unroll
                    for (int i = r & 1; i + 1 < kStage; i += 2) cswap(j[i], w[i], j[i + 1], w[i + 1]);
#pragma unroll
                for (int i = 0; i < kStage; ++i)
                    if (i < n) cm_place(p, sh, base_pos, o + i, w[i], k, i);
                continue;
            }
            int64_t o = base_pos + (staged ? sh.soff[kl] : p.cnt[k]);
            if (p.qd[k] > kHeavyDeg && kl < kHeavyBuf) {
                sh.heavy[atomicAdd(&sh.s_nheavy, 1)] = kl;
                continue;
            }
            cm_rescan_thread(p, sh, base_pos, k, o);
        }
        __syncthreads();
        for (int h = wid; h < sh.s_nheavy; h += wpb) {
            int kl = sh.heavy[h];
            int64_t k = c0 + kl;
            int64_t o = base_pos + (staged ? sh.soff[kl] : p.cnt[k]);
            cm_rescan_warp(p, sh, base_pos, k, o, lane);
        }
        __syncthreads();
        // (C) the new vertices of this block record their adjacency range at
        //     their queue position and claim their neighbours
        if (threadIdx.x == 0) sh.s_nheavy = 0;
        __syncthreads();
        {
            const int G = group_lanes(carry);
            const int lg = threadIdx.x & (G - 1);
            const int ipp = blockDim.x / G;
            for (int64_t j = threadIdx.x / G; j < carry; j += ipp) {
                int32_t w;
                unsigned long long pw;
                if (j < kChildStage) {
                    w = sh.cw[j];
                    pw = sh.cp[j];
                } else {
                    w = p.Q[base_pos + j];
                    pw = p.qp[base_pos + j];
                }
                int64_t b = p.gp[w], e = p.gp[w + 1];
                if (lg == 0) {
                    p.qb[base_pos + j] = b;
                    p.qd[base_pos + j] = (int32_t)(e - b);
                }
                if (heavy_for(e - b, G) && j < kHeavyBuf) {
                    if (lg == 0) sh.heavy[atomicAdd(&sh.s_nheavy, 1)] = (int32_t)j;
                    continue;
                }
                claim_group(p, b, e, G, lg, pw);
            }
        }
        __syncthreads();
        for (int h = wid; h < sh.s_nheavy; h += wpb) {
            int64_t q = base_pos + sh.heavy[h];
            int64_t b = p.qb[q];
            claim_group(p, b, b + p.qd[q], 32, lane, p.qp[q]);
        }
        if (!grid_sync(p.gb)) return;
        int64_t nf = *(volatile int64_t*)(p.ntot + (L & 1));
        if (nf < 0 || hi + nf > p.N) {
            if (tid == 0) atomicCAS(p.gb.err, 0, (int)kDevOverflow);
            return;
        }
        lo = hi;
        hi = hi + nf;
        ++L;
    }
    if (tid == 0) {
        p.nlevels[0] = L;
        p.nlevels[1] = hi;
    }
}

__global__ void comp_keys(int64_t N, const int32_t* Q, const int32_t* label, const int32_t* cidx, uint64_t* keys,
                          uint32_t* vals)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        keys[k] = (uint64_t)(uint32_t)cidx[label[Q[k]]];
        vals[k] = (uint32_t)Q[k];
    }
}

__global__ void reverse_into_perm(int64_t N, const int32_t* cm_order, int32_t* perm)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x)
        perm[N - 1 - k] = cm_order[k];
}

inline unsigned grid_for(int64_t n) { return (unsigned)std::min<int64_t>(ceil_div(n, kBlock) + 1, 65535); }

}  // namespace

namespace {
// a second stream of the calling thread on the current device (created on
// first use, kept for the thread's lifetime)
cudaStream_t aux_stream()
{
    constexpr int kMaxDev = 64;
    thread_local cudaStream_t streams[kMaxDev] = {};
    int dev = 0;
    OBK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDev) throw Error{-5, "device index out of range"};
    if (!streams[dev]) OBK_CUDA(cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking));
    return streams[dev];
}
}  // namespace

void build_sym_graph(int64_t N, const int64_t* rp, const int32_t* ci, int64_t nnz, DBuf<int64_t>& gp,
                     DBuf<int32_t>& adj, cudaStream_t st)
{
    if (pattern_symmetric(N, rp, ci, nnz, st)) {
        DBuf<int64_t> deg(N + 1, st);
        drop_self_count<<<grid_for(N), kBlock, 0, st>>>(N, rp, ci, deg.p);
        OBK_CHECK_LAUNCH();
        gp.alloc(N + 1, st);
        exclusive_scan_i64(deg.p, gp.p, N, st);
        int64_t M = read_scalar(gp.p + N, st);
        adj.alloc(M > 0 ? M : 1, st);
        drop_self_copy<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(N, kBlock / 32), 65535 * 4)), kBlock, 0, st>>>(
            N, rp, ci, gp.p, adj.p);
        OBK_CHECK_LAUNCH();
        return;
    }
    // transpose pattern: the rows of each column, ascending
    DBuf<int64_t> tp;
    DBuf<uint32_t> trow, tsrc;
    transpose_pattern(N, N, rp, ci, nnz, tp, trow, tsrc, st);
    tsrc.release();
    DBuf<int64_t> deg(N + 1, st);
    merge_sym<false><<<grid_for(N), kBlock, 0, st>>>(N, rp, ci, tp.p, trow.p, nullptr, deg.p, nullptr);
    OBK_CHECK_LAUNCH();
    gp.alloc(N + 1, st);
    exclusive_scan_i64(deg.p, gp.p, N, st);
    int64_t M = read_scalar(gp.p + N, st);
    adj.alloc(M > 0 ? M : 1, st);
    merge_sym<true><<<grid_for(N), kBlock, 0, st>>>(N, rp, ci, tp.p, trow.p, gp.p, nullptr, adj.p);
    OBK_CHECK_LAUNCH();
}

void rcm_reorder(int64_t N, const int64_t* rp, const int32_t* ci, int64_t nnz, int32_t* perm,
                 long long spin_limit, int* d_err, RcmStats* stats, cudaStream_t st, StageClock* clock)
{
    auto mark = [&]() {
        if (clock) clock->mark(st);
    };
    DevInfo di = dev_info();
    // 1. symmetric graph
    DBuf<int64_t> gp;
    DBuf<int32_t> adj;
    build_sym_graph(N, rp, ci, nnz, gp, adj, st);
    int64_t M = read_scalar(gp.p + N, st);
    mark();

    // 2. ranks in (deg, index) order
    // stable sort by degree of the vertices in index order = (degree, index) order
    DBuf<uint64_t> dk(N, st);
    DBuf<uint32_t> by_rank(N, st);
    DBuf<unsigned long long> dmax(1, st);
    OBK_CUDA(cudaMemsetAsync(dmax.p, 0, sizeof(unsigned long long), st));
    deg_keys<<<grid_for(N), kBlock, 0, st>>>(N, gp.p, dk.p, by_rank.p, dmax.p);
    OBK_CHECK_LAUNCH();
    radix_sort_pairs(dk.p, by_rank.p, N, bits_for((uint64_t)read_scalar(dmax.p, st)), st);
    dk.release();
    DBuf<int32_t> r(N, st);
    rank_of<<<grid_for(N), kBlock, 0, st>>>(N, by_rank.p, r.p);
    OBK_CHECK_LAUNCH();

    // 3. adjacency lists sorted by rank
    DBuf<uint32_t> ak(M, st), av(M, st);
    if (M) {
        adj_rank_keys<<<grid_for(M), kBlock, 0, st>>>(M, adj.p, r.p, ak.p, av.p);
        OBK_CHECK_LAUNCH();
        segmented_sort_u32(gp.p, N, ak.p, av.p, st);
    }
    ak.release();
    const int32_t* adj_r = reinterpret_cast<const int32_t*>(av.p);
    mark();

    // 4. first search from the global minimum-(deg, index) vertex; if it
    //    reaches every vertex the graph is connected and no labelling is needed
    DBuf<int32_t> label(N, st), cidx(N, st);
    DBuf<int32_t> dist(N, st), qa(N, st), qb(N, st), ecc(N, st), cand_r(N, st);
    DBuf<int64_t> cnt4(4, st), nsrc(1, st);
    DBuf<int32_t> nlev(1, st);
    DBuf<unsigned> bar(kBarrierWords, st);
    // grids scale with the problem (one block per 2K vertices, at most two per
    // SM) so that small systems leave the rest of the GPU to other requests
    int64_t want = std::min<int64_t>((int64_t)di.sms * kCoopBlocksPerSm, ceil_div(N, 2048));
    int bfs_grid = coop_grid((const void*)bfs_levels, kCoopBlock, 0, want);
    auto run_bfs = [&](const int32_t* sources, int64_t ns, int grid) -> int64_t {
        OBK_CUDA(cudaMemsetAsync(dist.p, 0xff, N * sizeof(int32_t), st));
        OBK_CUDA(cudaMemsetAsync(cnt4.p, 0, 4 * sizeof(int64_t), st));
        OBK_CUDA(cudaMemsetAsync(bar.p, 0, kBarrierWords * sizeof(unsigned), st));
        BfsParams bp{N, gp.p, adj_r, sources, ns, dist.p, qa.p, qb.p, cnt4.p, nlev.p,
                     GridBarrier{bar.p, d_err, spin_limit}};
        void* args[] = {&bp};
        OBK_COOP_LAUNCH(bfs_levels, grid, kCoopBlock, args, st);
        OBK_CUDA(cudaMemsetAsync(ecc.p, 0, N * sizeof(int32_t), st));
        OBK_CUDA(cudaMemsetAsync(cand_r.p, 0x7f, N * sizeof(int32_t), st));
        ecc_per_comp<<<grid_for(N), kBlock, 0, st>>>(N, dist.p, label.p, ecc.p);
        OBK_CHECK_LAUNCH();
        last_level_min<<<grid_for(N), kBlock, 0, st>>>(N, dist.p, label.p, ecc.p, r.p, cand_r.p);
        OBK_CHECK_LAUNCH();
        int64_t reached = read_scalar(cnt4.p + 3, st);
        if (read_scalar(d_err, st) != 0) throw Error{-4, "bounded wait expired in RCM search"};
        return reached;
    };
    OBK_CUDA(cudaMemsetAsync(label.p, 0, N * sizeof(int32_t), st));
    DBuf<int32_t> s0(1, st);
    OBK_CUDA(cudaMemcpyAsync(s0.p, by_rank.p, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    int64_t reached = run_bfs(s0.p, 1, bfs_grid);
    int64_t C = 1;
    DBuf<int32_t> roots;
    if (reached == N) {
        roots.alloc(1, st);
        OBK_CUDA(cudaMemcpyAsync(roots.p, s0.p, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        OBK_CUDA(cudaMemsetAsync(cidx.p, 0, sizeof(int32_t), st));  // label 0 -> component 0
    } else {
        // connected components (label = smallest vertex index) by min-hooking
        DBuf<int> changed(1, st);
        cc_init<<<grid_for(N), kBlock, 0, st>>>(N, label.p);
        OBK_CHECK_LAUNCH();
        for (int it = 0; it < 100000; ++it) {
            OBK_CUDA(cudaMemsetAsync(changed.p, 0, sizeof(int), st));
            cc_hook<<<grid_for(N), kBlock, 0, st>>>(N, gp.p, adj.p, label.p, changed.p);
            OBK_CHECK_LAUNCH();
            cc_compress<<<grid_for(N), kBlock, 0, st>>>(N, label.p);
            OBK_CHECK_LAUNCH();
            if (read_scalar(changed.p, st) == 0) break;
        }
        // component order (by minimum-(deg, index) vertex) and first positions
        DBuf<int32_t> cmin_r(N, st), csize(N, st), flag(N, st);
        DBuf<int64_t> fscan(N + 1, st);
        OBK_CUDA(cudaMemsetAsync(cmin_r.p, 0x7f, N * sizeof(int32_t), st));
        OBK_CUDA(cudaMemsetAsync(csize.p, 0, N * sizeof(int32_t), st));
        comp_stats<<<grid_for(N), kBlock, 0, st>>>(N, label.p, r.p, cmin_r.p, csize.p);
        OBK_CHECK_LAUNCH();
        comp_start_flags<<<grid_for(N), kBlock, 0, st>>>(N, by_rank.p, label.p, cmin_r.p, flag.p);
        OBK_CHECK_LAUNCH();
        exclusive_scan_i32_to_i64(flag.p, fscan.p, N, st);
        C = read_scalar(fscan.p + N, st);
        roots.alloc(C, st);
        DBuf<int64_t> size_by_idx(C, st);
        comp_order<<<grid_for(N), kBlock, 0, st>>>(N, by_rank.p, label.p, flag.p, fscan.p, cidx.p, roots.p,
                                                   size_by_idx.p, csize.p);
        OBK_CHECK_LAUNCH();
        run_bfs(roots.p, C, bfs_grid);
    }
    adj.release();

    // 5. George-Liu pseudo-peripheral roots, all components at once
    DBuf<int32_t> ecc_root(C, st), cand(C, st), active(C, st), src(C, st);
    DBuf<int> any(1, st);
    OBK_CUDA(cudaMemsetAsync(active.p, 1, C * sizeof(int32_t), st));  // nonzero word = active
    gl_record_root<<<grid_for(C), kBlock, 0, st>>>(C, roots.p, label.p, ecc.p, cand_r.p, by_rank.p,
                                                    ecc_root.p, cand.p, active.p);
    OBK_CHECK_LAUNCH();
    // Cuthill-McKee overlaps the search: a pass from the roots a round would
    // end with runs on a second stream beside the search's BFS (each on half
    // the grid); if the search ends with exactly those roots, the pass is the
    // result.  On long level structures (many levels) the first candidates
    // usually become the roots and stay, so the first round starts a pass from
    // them and it overlaps two BFS; otherwise a pass starts from the current
    // roots once a round has moved them (the next BFS usually confirms them).
    // buffers of one Cuthill-McKee pass
    struct CmBufs {
        DBuf<unsigned long long> claim, qp, agg;
        DBuf<int64_t> cnt, nl, ntot, qb;
        DBuf<int32_t> q, qd, roots;
        DBuf<unsigned> bar;
        void alloc(int64_t n, int64_t c, int agg_n, cudaStream_t s)
        {
            claim.alloc(n, s);
            qp.alloc(n, s);
            qb.alloc(n, s);
            qd.alloc(n, s);
            agg.alloc(agg_n, s);
            cnt.alloc(n, s);
            nl.alloc(2, s);
            ntot.alloc(2, s);
            q.alloc(n, s);
            roots.alloc(c, s);
            bar.alloc(kBarrierWords, s);
        }
    };
    int half_grid = std::max(1, bfs_grid / 2);
    int cm_grid_full = coop_grid((const void*)cm_levels, kCoopBlock, 0, want);
    int cm_grid_half = coop_grid((const void*)cm_levels, kCoopBlock, 0, std::max<int64_t>(1, want / 2));
    CmBufs pass;  // the overlapped pass (second stream)
    cudaStream_t st2 = aux_stream();
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    OBK_CUDA(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
    OBK_CUDA(cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming));
    // on every exit the second stream's pass has ended before its buffers go
    struct EvGuard {
        cudaEvent_t a, b;
        bool pending;
        ~EvGuard()
        {
            if (pending) cudaEventSynchronize(b);
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } evg{ev_in, ev_out, false};
    // Cuthill-McKee from b.roots into b.q on stream s with the given grid
    auto launch_cm = [&](CmBufs& b, cudaStream_t s, int grid) {
        OBK_CUDA(cudaMemsetAsync(b.claim.p, 0xff, N * sizeof(unsigned long long), s));
        OBK_CUDA(cudaMemsetAsync(b.bar.p, 0, kBarrierWords * sizeof(unsigned), s));
        OBK_CUDA(cudaMemsetAsync(b.agg.p, 0, grid * sizeof(unsigned long long), s));
        CmParams cp{N, gp.p, adj_r, b.roots.p, C, b.claim.p, b.qp.p, b.qb.p, b.qd.p, b.q.p, b.cnt.p, b.agg.p,
                    b.ntot.p, b.nl.p, GridBarrier{b.bar.p, d_err, spin_limit}};
        void* args[] = {&cp};
        OBK_COOP_LAUNCH(cm_levels, grid, kCoopBlock, args, s);
    };
    DBuf<int> differ(1, st);
    // true when the roots differ from those of the overlapped pass
    auto roots_moved_from_pass = [&]() -> bool {
        OBK_CUDA(cudaMemsetAsync(differ.p, 0, sizeof(int), st));
        roots_differ<<<grid_for(C), kBlock, 0, st>>>(C, roots.p, pass.roots.p, differ.p);
        OBK_CHECK_LAUNCH();
        return read_scalar(differ.p, st) != 0;
    };
    auto start_pass = [&]() {
        OBK_CUDA(cudaEventRecord(ev_in, st));
        OBK_CUDA(cudaStreamWaitEvent(st2, ev_in, 0));
        evg.pending = true;
        launch_cm(pass, st2, cm_grid_half);
        OBK_CUDA(cudaEventRecord(ev_out, st2));
    };
    auto end_pass = [&]() {
        OBK_CUDA(cudaEventSynchronize(ev_out));
        evg.pending = false;
        OBK_CUDA(cudaStreamWaitEvent(st, ev_out, 0));  // later stream work sees the pass's output
    };
    auto pass_running = [&]() {
        if (!evg.pending) return false;
        cudaError_t q = cudaEventQuery(ev_out);
        if (q == cudaErrorNotReady) return true;
        OBK_CUDA(q);
        return false;
    };
    const bool long_levels = bfs_grid > 1 && read_scalar(nlev.p, st) >= kEarlyPassLevels;
    bool moved = false, cm_done = false, live = false;  // live: the pass may still be the result
    int gl_rounds = 0;
    for (;;) {
        ++gl_rounds;
        OBK_CUDA(cudaMemsetAsync(nsrc.p, 0, sizeof(int64_t), st));
        gather_active_sources<<<grid_for(C), kBlock, 0, st>>>(C, cand.p, active.p, src.p, nsrc.p);
        OBK_CHECK_LAUNCH();
        int64_t ns = read_scalar(nsrc.p, st);
        if (ns == 0) break;
        if (!live && bfs_grid > 1 && (moved || (gl_rounds == 1 && long_levels))) {
            if (!pass.q.p) pass.alloc(N, C, cm_grid_full, st);
            if (evg.pending) end_pass();  // a pass that is no longer the result: let it end first
            if (moved) {
                OBK_CUDA(cudaMemcpyAsync(pass.roots.p, roots.p, C * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
            } else {  // the roots if every active component moves to its candidate
                spec_roots<<<grid_for(C), kBlock, 0, st>>>(C, roots.p, cand.p, active.p, pass.roots.p);
                OBK_CHECK_LAUNCH();
            }
            start_pass();
            live = true;
        }
        run_bfs(src.p, ns, pass_running() ? half_grid : bfs_grid);
        OBK_CUDA(cudaMemsetAsync(any.p, 0, sizeof(int), st));
        gl_compare<<<grid_for(C), kBlock, 0, st>>>(C, roots.p, label.p, ecc.p, cand_r.p, by_rank.p,
                                                    ecc_root.p, cand.p, active.p, any.p);
        OBK_CHECK_LAUNCH();
        int changed = read_scalar(any.p, st);
        if (changed == 0) break;
        moved = true;
        if (live && roots_moved_from_pass()) live = false;  // that pass cannot be the result any more
    }
    if (live && !roots_moved_from_pass()) {
        end_pass();
        cm_done = true;
    }
    dist.release(); ecc.release(); cand_r.release(); ecc_root.release(); cand.release();
    active.release(); src.release();
    mark();

    // 6. Cuthill-McKee levels into one queue (unless the overlapped pass already
    //    ran from the final roots), then the per-component order.  A pass
    //    still running on the second stream keeps half the grid.
    CmBufs main_pass;
    CmBufs* res = &pass;
    if (!cm_done) {
        main_pass.alloc(N, C, cm_grid_full, st);
        OBK_CUDA(cudaMemcpyAsync(main_pass.roots.p, roots.p, C * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        launch_cm(main_pass, st, pass_running() ? cm_grid_half : cm_grid_full);
        res = &main_pass;
    }
    int32_t* Q = res->q.p;
    if (read_scalar(d_err, st) != 0) throw Error{-4, "bounded wait or bound check failed in Cuthill-McKee levels"};
    if (read_scalar(res->nl.p + 1, st) != N) throw Error{-5, "internal error: Cuthill-McKee order does not cover every vertex"};
    const int32_t* cm = Q;
    DBuf<uint64_t> ck;
    DBuf<uint32_t> cv;
    if (C > 1) {
        ck.alloc(N, st);
        cv.alloc(N, st);
        comp_keys<<<grid_for(N), kBlock, 0, st>>>(N, Q, label.p, cidx.p, ck.p, cv.p);
        OBK_CHECK_LAUNCH();
        radix_sort_pairs(ck.p, cv.p, N, bits_for((uint64_t)C), st);
        cm = reinterpret_cast<const int32_t*>(cv.p);
    }
    reverse_into_perm<<<grid_for(N), kBlock, 0, st>>>(N, cm, perm);
    OBK_CHECK_LAUNCH();
    if (stats) {
        stats->components = C;
        stats->levels = read_scalar(res->nl.p, st);
        stats->gl_rounds = gl_rounds;
        stats->graph_edges = M;
    }
}

}  // namespace obk
