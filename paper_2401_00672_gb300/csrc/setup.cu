// setup.cu -- validation, symmetric permutation (Eq. 3.1), row norms (Eq. 1.2)
// and the cosine-threshold row grouping of Section 3.3 taken at one row per
// block, plus the memory layout used by the sweep.
//
// Grouping, as fixed for this library (bit-identical to the CPU reference):
//   nsq_i   = ((a_1*a_1 + a_2*a_2) + ...) over ascending columns, each product
//             and sum rounded separately (no fused multiply-add)
//   dot_ij  = left fold of a_ic*a_jc over the common columns, ascending
//   cos_ij  = dot_ij / (sqrt(nsq_i) * sqrt(nsq_j)), IEEE division and sqrt
//   conflict when |cos_ij| >= thr; row i joins the smallest group holding no
//   conflicting earlier row (greedy first fit in index order); rows with
//   nsq = 0 join no group.
//
// GPU formulation: dot products are accumulated Gustavson style (one warp per
// row i walks its columns in ascending order and, for each column, adds the
// products with every earlier row of that column into a per-warp hash table),
// which keeps the per-pair ascending-column order.  First fit is computed as
// the unique fixed point of c_i = mex{c_j : j < i conflicting} by rounds of
// in-place updates until a round changes nothing.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace obk {
namespace {

constexpr int kBlock = 256;
inline unsigned grid_for(int64_t n) { return (unsigned)std::min<int64_t>(ceil_div(n, kBlock) + 1, 65535); }

#define GRID_STRIDE(i, n)                                                              \
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); \
         i += (int64_t)gridDim.x * blockDim.x)

// ---- validation --------------------------------------------------------------

__global__ void validate_rows(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci,
                              const double* v, int64_t nnz, int* bad)
{
    GRID_STRIDE(i, m)
    {
        int64_t b = rp[i], e = rp[i + 1];
        if (b > e || b < 0 || e > nnz) { atomicOr(bad, 1); continue; }
        for (int64_t k = b; k < e; ++k) {
            int32_t c = ci[k];
            if (c < 0 || (int64_t)c >= n) { atomicOr(bad, 2); break; }
            if (k > b && c <= ci[k - 1]) { atomicOr(bad, 4); break; }
            if (v && !isfinite(v[k])) { atomicOr(bad, 8); break; }  // v NULL: the pattern only
        }
    }
}

__global__ void bandwidth_kernel(int64_t N, const int64_t* rp, const int32_t* ci,
                                 unsigned long long* bw)
{
    unsigned long long mx = 0;
    GRID_STRIDE(i, N)
    {
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            long long d = (long long)i - ci[e];
            unsigned long long a = (unsigned long long)(d < 0 ? -d : d);
            mx = a > mx ? a : mx;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = t > mx ? t : mx;
    }
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(bw, mx);
}

// ---- permutation -------------------------------------------------------------

__global__ void inverse_perm(int64_t N, const int32_t* perm, int32_t* iperm)
{
    GRID_STRIDE(k, N) iperm[perm[k]] = (int32_t)k;
}

__global__ void permuted_lengths(int64_t N, const int64_t* rp, const int32_t* perm, int64_t* len)
{
    GRID_STRIDE(k, N) len[k] = rp[perm[k] + 1] - rp[perm[k]];
}

__global__ void permute_gather(int64_t N, const int64_t* rp, const int32_t* ci, const int32_t* perm,
                               const int32_t* iperm, const int64_t* rp_t, uint32_t* keys,
                               uint32_t* src)
{
    // one warp per new row
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = w; k < N; k += nw) {
        int64_t o = rp[perm[k]], len = rp[perm[k] + 1] - o, d = rp_t[k];
        for (int64_t t = lane; t < len; t += 32) {
            keys[d + t] = (uint32_t)iperm[ci[o + t]];
            src[d + t] = (uint32_t)(o + t);
        }
    }
}

// Rows of at most 32 entries in one pass: one warp per new row k gathers the
// entries of old row perm[k], relabels their columns, sorts them by the new
// column with a bitonic network across the lanes (columns of a row are
// distinct, so the order is unique) and writes them.  Lanes past the row's
// end carry the largest key and sort last.
__global__ void permute_rows_warp(int64_t N, const int64_t* rp, const int32_t* ci, const double* v,
                                  const int32_t* perm, const int32_t* iperm, const int64_t* rp_t, int32_t* ci_t,
                                  double* v_t)
{
    const unsigned full = 0xffffffffu;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = w; k < N; k += nw) {
        int64_t o = rp[perm[k]], len = rp[perm[k] + 1] - o, d = rp_t[k];
        uint32_t key = 0xffffffffu;
        double val = 0.0;
        if (lane < len) {
            key = (uint32_t)iperm[ci[o + lane]];
            val = v[o + lane];
        }
#pragma unroll
        for (int m = 2; m <= 32; m <<= 1) {
#pragma unroll
            for (int j = m >> 1; j > 0; j >>= 1) {
                uint32_t ok = __shfl_xor_sync(full, key, j);
                double ov = __shfl_xor_sync(full, val, j);
                bool up = (lane & m) == 0;      // this run sorts ascending
                bool low = (lane & j) == 0;     // the lower lane keeps the smaller key of an ascending run
                bool take = (low == up) ? ok < key : ok > key;
                if (take) {
                    key = ok;
                    val = ov;
                }
            }
        }
        if (lane < len) {
            ci_t[d + lane] = (int32_t)key;
            v_t[d + lane] = val;
        }
    }
}

__global__ void permute_finish(int64_t nnz, const uint32_t* keys, const uint32_t* src, const double* v,
                               int32_t* ci_t, double* v_t)
{
    GRID_STRIDE(e, nnz)
    {
        ci_t[e] = (int32_t)keys[e];
        v_t[e] = v[src[e]];
    }
}

// ---- norms and transposition -------------------------------------------------

// nsq[i] = ||A_i||^2 as the left fold of the rounded squares over ascending
// columns, s[i] = sqrt(nsq[i]); one thread per row, the values of a row loaded
// eight at a time before they are folded in order
__global__ void row_norms_exact(int64_t N, const int64_t* rp, const double* v, double* nsq, double* s)
{
    GRID_STRIDE(i, N)
    {
        double acc = 0.0;
        int64_t e = rp[i];
        const int64_t e1 = rp[i + 1];
        for (; e + 8 <= e1; e += 8) {
            double a[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = v[e + k];
#pragma unroll
            for (int k = 0; k < 8; ++k) acc = __dadd_rn(acc, __dmul_rn(a[k], a[k]));
        }
        for (; e < e1; ++e) acc = __dadd_rn(acc, __dmul_rn(v[e], v[e]));
        nsq[i] = acc;
        s[i] = __dsqrt_rn(acc);
    }
}

// CSC arrays from the transposed pattern; pos_of[e] = CSC position of entry e.
__global__ void csc_fill(int64_t nnz, const uint32_t* src, const uint32_t* trow, const double* v,
                         int32_t* crow, double* cval, int64_t* pos_of)
{
    GRID_STRIDE(p, nnz)
    {
        uint32_t e = src[p];
        crow[p] = (int32_t)trow[p];
        cval[p] = v[e];
        pos_of[e] = p;
    }
}

// The same for a structurally symmetric pattern, where the CSC slot of entry
// e is tsrc[e] and the entry of slot p is tsrc[p]: coalesced writes only.
__global__ void csc_fill_symmetric(int64_t nnz, const uint32_t* tsrc, const double* v, double* cval,
                                   int64_t* pos_of)
{
    GRID_STRIDE(p, nnz)
    {
        const uint32_t e = tsrc[p];
        cval[p] = v[e];
        pos_of[p] = (int64_t)e;
    }
}

// ub[i] = number of (earlier row, shared column) incidences of row i; the rank
// of entry (i, c) in column c counts the earlier rows of that column.
__global__ void pair_upper_bound(int64_t N, const int64_t* rp, const int32_t* ci, const int64_t* cptr,
                                 const int64_t* pos_of, int64_t* ub)
{
    GRID_STRIDE(i, N)
    {
        int64_t s = 0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) s += pos_of[e] - cptr[ci[e]];
        ub[i] = s;
    }
}

// hash slots for a row with at most ub candidates: a power of two, load <= 2/3
__host__ __device__ inline int64_t table_cap(int64_t ub)
{
    int64_t c = 32;
    while (c < ub + (ub + 1) / 2) c <<= 1;
    return c;
}

__global__ void big_table_sizes(int64_t N, const int64_t* ub, int64_t smem_cap, int64_t* sz)
{
    GRID_STRIDE(i, N)
    {
        int64_t c = table_cap(ub[i]);
        sz[i] = c > smem_cap ? c : 0;
    }
}

// ---- pair cosines and conflict lists ------------------------------------------

constexpr int kPairWarps = 8;
constexpr int kPairCap = 512;  // hash slots per warp in shared memory
constexpr int32_t kEmpty = -1;

struct PairParams {
    int64_t N;
    const int64_t* rp;
    const int32_t* ci;
    const double* v;
    const int64_t* cptr;
    const int32_t* crow;
    const double* cval;
    const int64_t* pos_of;
    const double* nsq;
    const double* s;
    double thr;
    const int64_t* ub;
    const int64_t* big_off;  // offsets into the global tables (rows whose table is too big)
    int32_t* big_key;
    double* big_val;
    int32_t* conf_cnt;       // out
    int64_t* conf_off;       // out
    int32_t* pool;
    int64_t pool_cap;
    unsigned long long* pool_used;
    unsigned long long* n_conflicts;
    int* err;
    unsigned long long* stats;  // STATS mode: [0] nonzero cosine-table entries, [1] sum of |cos| in 2^-32
    const int64_t* gstart;      // GRAM mode: first group-major row of each row's group
    double* pool_val;           // GRAM mode: the dot product of each listed pair
};

__device__ __forceinline__ uint32_t hslot(int32_t j, uint32_t mask)
{
    return ((uint32_t)j * 0x9E3779B1u) & mask;
}

// |cos_ij| >= thr with cos_ij = RN(dot / RN(s_j * s_i)), decided exactly.
// t = RN(RN(thr * s_i) * s_j) is within 3 units of rounding of thr * s_i * s_j,
// so |dot| more than 32 units in the last place of t above t (a relative
// margin of at least 2^-48) proves the quotient reaches thr, and as far below
// proves it rounds below thr; only the narrow band in between takes the IEEE
// division.  Non-negative doubles order like their bit patterns, so the band
// and range tests are integer compares: one FP64 multiply per candidate.
__device__ __forceinline__ bool is_conflict(double dot, double sj, double si, double thr_si, double thr)
{
    const long long kTmin = __double_as_longlong(1e-280), kTmax = __double_as_longlong(1e280);
    const long long kAmax = __double_as_longlong(1e300);
    long long ab = __double_as_longlong(dot) & 0x7fffffffffffffffLL;
    long long tb = __double_as_longlong(thr_si * sj);
    if (tb > kTmin && tb < kTmax && ab < kAmax) {
        if (ab > tb + 32) return true;
        if (ab < tb - 32) return false;
    }
    return fabs(__ddiv_rn(dot, __dmul_rn(sj, si))) >= thr;
}

// x == 0.0 for a row norm (never negative), by its bits
__device__ __forceinline__ bool zero_norm(double x)
{
    return (__double_as_longlong(x) << 1) == 0;
}

// Modes: kPairConflicts lists the earlier conflicting rows (|cos| >= thr);
// kPairStats counts the nonzero entries of the row cosine table and adds up
// their magnitudes (rounded to units of 2^-32) for Definitions 1-2, the
// diagonal (1 for every row here) included; kPairGram lists the earlier rows
// of the same group with a nonzero dot product, with that product.
enum PairMode { kPairConflicts = 0, kPairStats = 1, kPairGram = 2 };

template <int MODE>
__global__ void __launch_bounds__(kPairWarps * 32) pair_conflicts(PairParams p)
{
    constexpr bool STATS = MODE == kPairStats;
    __shared__ int32_t skey[kPairWarps][kPairCap];
    __shared__ double sval[kPairWarps][kPairCap];
    __shared__ int64_t spre[kPairWarps][32];  // incidence prefix of the current 32 entries
    __shared__ int64_t sq0[kPairWarps][32];   // first column position of each entry
    __shared__ double sa[kPairWarps][32];     // value of each entry
    int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    unsigned lt = (1u << lane) - 1u;
    int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = gw; i < p.N; i += nw) {
        if (p.nsq[i] == 0.0) {
            if (!STATS && lane == 0) { p.conf_cnt[i] = 0; p.conf_off[i] = 0; }
            continue;
        }
        int64_t cap = table_cap(p.ub[i]);
        int32_t* key;
        double* val;
        if (cap <= kPairCap) {
            key = skey[wl];
            val = sval[wl];
        } else {
            key = p.big_key + p.big_off[i];
            val = p.big_val + p.big_off[i];
        }
        uint32_t mask = (uint32_t)cap - 1u;
        for (int64_t t = lane; t < cap; t += 32) { key[t] = kEmpty; val[t] = 0.0; }
        __syncwarp();
        // The (column, earlier row) incidences of row i, in ascending column
        // order, are processed 32 at a time: one product per lane, then the
        // additions into the table in rounds, the r-th round taking each
        // lane whose row j occurred r times earlier in the chunk.  Every
        // dot_ij therefore accumulates its products in ascending column order.
        for (int64_t e0 = p.rp[i]; e0 < p.rp[i + 1]; e0 += 32) {
            int64_t e = e0 + lane;
            int64_t cnt = 0, q0 = 0;
            double a = 0.0;
            if (e < p.rp[i + 1]) {
                int32_t c = p.ci[e];
                a = p.v[e];
                q0 = p.cptr[c];
                cnt = p.pos_of[e] - q0;  // earlier rows of column c
            }
            int64_t inc = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += t;
            }
            spre[wl][lane] = inc - cnt;
            sq0[wl][lane] = q0;
            sa[wl][lane] = a;
            int64_t U = __shfl_sync(0xffffffffu, inc, 31);
            __syncwarp();
            for (int64_t t0 = 0; t0 < U; t0 += 32) {
                int64_t t = t0 + lane;
                bool valid = t < U;
                int32_t j = -1;
                double prod = 0.0;
                if (valid) {
                    int lo = 0, hi = 31;  // last entry whose incidences start at or before t
                    while (lo < hi) {
                        int mid = (lo + hi + 1) >> 1;
                        if (spre[wl][mid] <= t) lo = mid;
                        else hi = mid - 1;
                    }
                    int64_t q = sq0[wl][lo] + (t - spre[wl][lo]);
                    j = p.crow[q];
                    double w = p.cval[q];
                    if (zero_norm(p.nsq[j])) valid = false;
                    else prod = __dmul_rn(sa[wl][lo], w);
                }
                unsigned peers = __match_any_sync(0xffffffffu, valid ? j : -1 - lane);
                int rank = __popc(peers & lt);
                int maxr = __reduce_max_sync(0xffffffffu, valid ? rank : 0);
                uint32_t h = 0;
                if (valid && rank == 0) {
                    h = hslot(j, mask);
                    int64_t probes = 0;
                    for (;;) {
                        int32_t k = key[h];
                        if (k == j) break;
                        if (k == kEmpty) {
                            int32_t old = atomicCAS(key + h, kEmpty, j);
                            if (old == kEmpty || old == j) break;
                        }
                        h = (h + 1) & mask;
                        if (++probes > cap) { h = 0xffffffffu; break; }
                    }
                }
                h = __shfl_sync(0xffffffffu, h, __ffs(peers) - 1);
                if (valid && h == 0xffffffffu) {
                    atomicCAS(p.err, 0, (int)kDevOverflow);
                    valid = false;
                }
                for (int r = 0; r <= maxr; ++r) {
                    if (valid && rank == r) val[h] = __dadd_rn(val[h], prod);
                    __syncwarp();
                }
            }
            __syncwarp();
        }
        // compact the occupied slots to the front of the table (in slot order)
        int nc = 0;
        for (int64_t t0 = 0; t0 < cap; t0 += 32) {
            int64_t t = t0 + lane;
            int32_t j = t < cap ? key[t] : kEmpty;
            double a = t < cap ? val[t] : 0.0;
            unsigned m = __ballot_sync(0xffffffffu, j != kEmpty);
            __syncwarp();
            if (j != kEmpty) {
                key[nc + __popc(m & lt)] = j;
                val[nc + __popc(m & lt)] = a;
            }
            nc += __popc(m);
            __syncwarp();
        }
        if (STATS) {
            double si0 = p.s[i];
            unsigned long long c_nz = 0, c_sum = 0;
            for (int t = lane; t < nc; t += 32) {
                double cv = fabs(__ddiv_rn(val[t], __dmul_rn(p.s[key[t]], si0)));
                if (cv != 0.0) {  // C_ij and C_ji
                    c_nz += 2;
                    c_sum += 2ull * __double2ull_rn(cv * 0x1p32);
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                c_nz += __shfl_xor_sync(0xffffffffu, c_nz, o);
                c_sum += __shfl_xor_sync(0xffffffffu, c_sum, o);
            }
            if (lane == 0) {
                atomicAdd(p.stats, c_nz + 1);             // + C_ii
                atomicAdd(p.stats + 1, c_sum + (1ull << 32));
            }
            __syncwarp();
            continue;
        }
        // one decision per candidate, kept as bits (64 candidates per lane)
        double si = p.s[i];
        double thr_si = p.thr * si;
        int64_t g0 = MODE == kPairGram ? p.gstart[i] : 0;
        auto keep = [&](int t) -> bool {
            if (MODE == kPairGram) return key[t] >= g0 && val[t] != 0.0;
            return is_conflict(val[t], p.s[key[t]], si, thr_si, p.thr);
        };
        int cnt = 0;
        unsigned long long flags = 0;
        bool many = nc > 32 * 64;
        for (int t0 = 0, it = 0; t0 < nc; t0 += 32, ++it) {
            int t = t0 + lane;
            bool conf = false;
            if (t < nc) conf = keep(t);
            if (conf && !many) flags |= 1ull << it;
            cnt += __popc(__ballot_sync(0xffffffffu, conf));
        }
        unsigned long long base = 0;
        if (lane == 0) {
            base = atomicAdd(p.pool_used, (unsigned long long)cnt);
            atomicAdd(p.n_conflicts, (unsigned long long)cnt);
            p.conf_cnt[i] = cnt;
            p.conf_off[i] = (int64_t)base;
        }
        base = __shfl_sync(0xffffffffu, base, 0);
        if ((int64_t)(base + cnt) <= p.pool_cap) {
            int run = 0;
            for (int t0 = 0, it = 0; t0 < nc; t0 += 32, ++it) {
                int t = t0 + lane;
                bool conf;
                if (!many) conf = (flags >> it) & 1ull;
                else conf = t < nc && keep(t);
                unsigned b = __ballot_sync(0xffffffffu, conf);
                if (conf) {
                    p.pool[base + run + __popc(b & lt)] = key[t];
                    if (MODE == kPairGram) p.pool_val[base + run + __popc(b & lt)] = val[t];
                }
                run += __popc(b);
            }
        }
        __syncwarp();
    }
}

// ---- greedy first-fit colouring (fixed-point rounds) ---------------------------
//
// First fit in index order gives row i the smallest colour not used by its
// earlier conflicting rows.  That recurrence has exactly one solution, so any
// colouring c with c_i = mex{c_j : j < i conflicts with i} for every i is the
// sequential result.  The kernel starts from c = 0 and repeats rounds in which
// every row recomputes its mex from the current colours (in place, so later
// rows of a round already see earlier updates).  A round that changes nothing
// proves the fixed point.  After round r every row whose longest chain of
// earlier conflicts is shorter than r is final, so at most (chain length + 2)
// rounds run; on the workloads measured the rounds stay below about a hundred
// while the chains grow with the problem.

constexpr int kColorBatch = 4;

struct ColorParams {
    int64_t N;
    const double* nsq;
    const int32_t* conf_cnt;
    const int64_t* conf_off;
    const int32_t* pool;
    int32_t* color;     // rows with nsq == 0 get -1
    int* changed;       // 3 rotating round flags, zeroed
    int64_t* rounds;    // out
    int64_t run;        // consecutive rows a lane group takes at a time
    GridBarrier gb;
};

// S lanes per row: the lanes read a row's conflict list together (S
// consecutive entries at a time, kColorBatch such reads in flight) and OR
// their colour masks; S = 1 is one thread per row.
template <int S>
__global__ void __launch_bounds__(kBlock) greedy_color(ColorParams p)
{
    __shared__ int s_changed;
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t nth = (int64_t)gridDim.x * blockDim.x;
    int sub = (int)(threadIdx.x & (S - 1));
    int64_t sw = tid / S, nsw = nth / S;
    unsigned smask = S == 32 ? 0xffffffffu : (((1u << S) - 1u) << ((threadIdx.x & 31) & ~(S - 1)));
    volatile int32_t* col = p.color;
    for (int64_t i = tid; i < p.N; i += nth) col[i] = p.nsq[i] == 0.0 ? -1 : 0;
    if (!grid_sync(p.gb)) return;
    for (int64_t r = 0; r <= p.N + 1; ++r) {
        if (threadIdx.x == 0) s_changed = 0;
        if (tid == 0) p.changed[(r + 1) % 3] = 0;  // last read two rounds ago
        __syncthreads();
        int ch = 0;
        // each lane group takes runs of p.run consecutive rows in index order,
        // so a chain of conflicts between nearby rows (the usual case after
        // RCM) resolves inside one round instead of one link per round
        for (int64_t rb = sw * p.run; rb < p.N; rb += nsw * p.run)
        for (int64_t i = rb; i < rb + p.run && i < p.N; ++i) {
            int32_t ci = col[i];
            if (ci < 0) continue;  // the same for the row's S lanes
            int64_t o = p.conf_off[i];
            int n = p.conf_cnt[i];
            unsigned long long used = 0;
            for (int t0 = sub; t0 < n; t0 += S * kColorBatch) {
                int32_t cj[kColorBatch];
#pragma unroll
                for (int u = 0; u < kColorBatch; ++u) {
                    cj[u] = -1;
                    if (t0 + S * u < n) cj[u] = col[p.pool[o + t0 + S * u]];
                }
#pragma unroll
                for (int u = 0; u < kColorBatch; ++u)
                    if (cj[u] >= 0 && cj[u] < 64) used |= 1ull << cj[u];
            }
            if (S > 1) {
                unsigned lo = (unsigned)used, hi = (unsigned)(used >> 32);
#pragma unroll
                for (int d = S / 2; d > 0; d >>= 1) {
                    lo |= __shfl_xor_sync(smask, lo, d);
                    hi |= __shfl_xor_sync(smask, hi, d);
                }
                used = ((unsigned long long)hi << 32) | lo;
            }
            if (sub != 0) continue;
            int32_t g;
            if (~used != 0ull) {
                g = __ffsll((long long)~used) - 1;
            } else {  // colours 0..63 all taken: smallest free one above
                g = 64;
                for (;;) {
                    bool taken = false;
                    for (int u = 0; u < n; ++u)
                        if (col[p.pool[o + u]] == g) { taken = true; break; }
                    if (!taken) break;
                    ++g;
                }
            }
            if (g != ci) {
                col[i] = g;
                ch = 1;
            }
        }
        if (__any_sync(0xffffffffu, ch) && (threadIdx.x & 31) == 0) s_changed = 1;
        __syncthreads();
        if (threadIdx.x == 0 && s_changed) atomicOr(p.changed + (r % 3), 1);
        if (!grid_sync(p.gb)) return;
        if (*(volatile int*)(p.changed + (r % 3)) == 0) {
            if (tid == 0) *p.rounds = r + 1;
            return;
        }
    }
    if (tid == 0) atomicCAS(p.gb.err, 0, (int)kDevTimeout);  // cannot happen: N + 2 rounds always suffice
}

__global__ void max_color(int64_t N, const int32_t* color, int* gmax)
{
    int m = -1;
    GRID_STRIDE(i, N) m = color[i] > m ? color[i] : m;
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m >= 0) atomicMax(gmax, m);
}

// ---- group layout -------------------------------------------------------------

// Row order of the sweep layout: by group, then by tile (a fixed range of
// B consecutive permuted rows; the sweep gives each thread block the tiles of
// one contiguous range, so that a block's rows of every group touch one band of
// x), then by row length, then by index (stable sort on (group, tile, length)
// over rows in index order).  Equal lengths inside a warp keep every lane of
// every FP64 instruction busy.  Rows (and column segments, by the tile of their
// column) are ordered by length in buckets of 2^kLenBucketShift, then by
// index: slices of 32 stay nearly free of padding while neighbouring lanes keep
// nearby indices (and so nearby columns).
constexpr int kLenBucketShift = 1;

// key = ((group * T + tile) << lbits) | length class; rows of no group take group G
__global__ void color_keys(int64_t N, const int32_t* color, const int64_t* rp, int32_t G, int64_t tile_rows,
                           int64_t T, int lbits, uint64_t* keys, uint32_t* vals)
{
    GRID_STRIDE(i, N)
    {
        uint64_t g = (uint64_t)(color[i] >= 0 ? color[i] : G);
        uint64_t len = (uint64_t)(rp[i + 1] - rp[i]) >> kLenBucketShift;
        uint64_t lmax = (1ull << lbits) - 1;
        uint64_t seg = g * (uint64_t)T + (uint64_t)(i / tile_rows);
        keys[i] = (seg << lbits) | (len < lmax ? len : lmax);
        vals[i] = (uint32_t)i;
    }
}

// ptr[s] = first position k of the sorted keys with (keys[k] >> shift) >= s,
// for s in [0, nseg]; keys at or beyond segment nseg (rows of no group) count
// as nseg.  Each entry of ptr is written by exactly one k.
__global__ void segment_starts(int64_t n, const uint64_t* keys, int shift, int64_t nseg, int64_t* ptr)
{
    GRID_STRIDE(k, n + 1)
    {
        int64_t lo = k == 0 ? 0 : (int64_t)(keys[k - 1] >> shift) + 1;
        int64_t hi = k == n ? nseg : (int64_t)(keys[k] >> shift);
        if (hi > nseg) hi = nseg;
        for (int64_t q = lo; q <= hi; ++q) ptr[q] = k;
    }
}

// Dependency reach of each tile of rows/columns [t * B, (t + 1) * B): the
// lowest and highest tile holding a column of one of its rows or a row of one
// of its columns (the tile itself included).  One block per tile.
__global__ void tile_reach(int64_t N, int64_t B, const int64_t* rp, const int32_t* ci, const int64_t* cptr,
                           const int32_t* crow, int32_t* reach_lo, int32_t* reach_hi)
{
    __shared__ int64_t slo[kBlock / 32], shi[kBlock / 32];
    int64_t t = blockIdx.x;
    int64_t k0 = t * B, k1 = k0 + B < N ? k0 + B : N;
    int64_t lo = t, hi = t;
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        if (rp[k + 1] > rp[k]) {  // columns ascend inside a row
            lo = min(lo, (int64_t)ci[rp[k]] / B);
            hi = max(hi, (int64_t)ci[rp[k + 1] - 1] / B);
        }
        if (cptr[k + 1] > cptr[k]) {  // rows ascend inside a column
            lo = min(lo, (int64_t)crow[cptr[k]] / B);
            hi = max(hi, (int64_t)crow[cptr[k + 1] - 1] / B);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) { slo[threadIdx.x >> 5] = lo; shi[threadIdx.x >> 5] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { lo = min(lo, slo[w]); hi = max(hi, shi[w]); }
        reach_lo[t] = (int32_t)lo;
        reach_hi[t] = (int32_t)hi;
    }
}

// Segment order inside each group: by tile of the column, then by length,
// then by column (stable sort of the (group, column)-ordered segments).
__global__ void seg_keys(int64_t nseg, const int64_t* seg_ptr, const int64_t* gseg_ptr, const int32_t* seg_col,
                         int64_t G, int64_t tile_rows, int64_t T, int lbits, uint64_t* keys, uint32_t* vals)
{
    GRID_STRIDE(t, nseg)
    {
        // group of segment t: gseg_ptr is increasing, binary search
        int64_t lo = 0, hi = G;
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) >> 1;
            if (gseg_ptr[mid] <= t) lo = mid;
            else hi = mid;
        }
        uint64_t len = (uint64_t)(seg_ptr[t + 1] - seg_ptr[t]) >> kLenBucketShift;
        uint64_t lmax = (1ull << lbits) - 1;
        uint64_t sq = (uint64_t)lo * (uint64_t)T + (uint64_t)(seg_col[t] / tile_rows);
        keys[t] = (sq << lbits) | (len < lmax ? len : lmax);
        vals[t] = (uint32_t)t;
    }
}

// longest row of a CSR (max over i of ptr[i+1] - ptr[i])
__global__ void max_row_len(int64_t n, const int64_t* ptr, unsigned long long* mx)
{
    unsigned long long m = 0;
    GRID_STRIDE(i, n)
    {
        unsigned long long d = (unsigned long long)(ptr[i + 1] - ptr[i]);
        m = d > m ? d : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
        m = t > m ? t : m;
    }
    __shared__ unsigned long long wmax[kBlock / 32];
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = 0;
        for (int w = 0; w < kBlock / 32; ++w) b = wmax[w] > b ? wmax[w] : b;
        if (b) atomicMax(mx, b);  // one atomic per block
    }
}

__global__ void gm_rows(int64_t Ngm, const uint32_t* order, const int64_t* rp, const double* nsq,
                        int32_t* grp_row, int32_t* gm_of_row, int64_t* len, double* inv, float* inv32)
{
    GRID_STRIDE(k, Ngm)
    {
        int32_t i = (int32_t)order[k];
        grp_row[k] = i;
        gm_of_row[i] = (int32_t)k;
        len[k] = rp[i + 1] - rp[i];
        double d = 1.0 / nsq[i];
        inv[k] = d;
        if (inv32) inv32[k] = (float)d;
    }
}

__global__ void gm_copy(int64_t Ngm, const int32_t* grp_row, const int64_t* rp, const int32_t* ci,
                        const double* v, const int64_t* grp_rp, int32_t* gci, double* gv, float* gv32)
{
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = w; k < Ngm; k += nw) {
        int64_t o = rp[grp_row[k]], len = rp[grp_row[k] + 1] - o, d = grp_rp[k];
        for (int64_t t = lane; t < len; t += 32) {
            gci[d + t] = ci[o + t];
            gv[d + t] = v[o + t];
            if (gv32) gv32[d + t] = (float)v[o + t];
        }
    }
}

__global__ void csc_color_keys(int64_t nnz, const int32_t* crow, const int32_t* color, int32_t G,
                               uint64_t* keys, uint32_t* vals)
{
    GRID_STRIDE(p, nnz)
    {
        int32_t c = color[crow[p]];
        keys[p] = (uint64_t)(c >= 0 ? c : G);
        vals[p] = (uint32_t)p;
    }
}

__global__ void expand_cols(int64_t N, const int64_t* cptr, int32_t* col_of)
{
    GRID_STRIDE(c, N)
    for (int64_t p = cptr[c]; p < cptr[c + 1]; ++p) col_of[p] = (int32_t)c;
}

// mirror entries in (group, column, row) order; seg flags mark (group, column)
// starts.  A warp takes 32 consecutive entries: each lane's predecessor's
// (column, group) comes from the lane before it by shuffle.
__global__ void mirror_fill(int64_t M, const uint32_t* order, const int32_t* crow, const double* cval,
                            const int32_t* col_of, const int32_t* color, const int32_t* gm_of_row,
                            int32_t* mrow, double* mval, float* mval32, int32_t* flag)
{
    int lane = threadIdx.x & 31;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t q0 = w * 32; q0 < M; q0 += nw * 32) {
        int64_t q = q0 + lane;
        bool valid = q < M;
        int32_t c = -1, g = -1;
        if (valid) {
            uint32_t pp = order[q];
            int32_t i = crow[pp];
            c = col_of[pp];
            g = color[i];
            mrow[q] = gm_of_row[i];
            double a = cval[pp];
            mval[q] = a;
            if (mval32) mval32[q] = (float)a;
        }
        int32_t pc = __shfl_up_sync(0xffffffffu, c, 1);
        int32_t pg = __shfl_up_sync(0xffffffffu, g, 1);
        if (valid) {
            if (lane == 0 && q > 0) {
                uint32_t pr = order[q - 1];
                pc = col_of[pr];
                pg = color[crow[pr]];
            }
            flag[q] = (q == 0 || pc != c || pg != g) ? 1 : 0;
        }
    }
}

__global__ void mirror_segments(int64_t M, const uint32_t* order, const int32_t* crow, const int32_t* col_of,
                                const int32_t* color, const int32_t* flag, const int64_t* fscan,
                                int64_t* seg_ptr, int32_t* seg_col, int64_t* gseg_ptr)
{
    GRID_STRIDE(q, M)
    {
        if (!flag[q]) continue;
        int64_t sg = fscan[q];
        uint32_t pp = order[q];
        seg_ptr[sg] = q;
        seg_col[sg] = col_of[pp];
        int32_t g = color[crow[pp]];
        if (q == 0 || color[crow[order[q - 1]]] != g) gseg_ptr[g] = sg;
    }
}

// ---- sliced ELL (SELL-32) copies of the group-major rows and the mirror ----------

// 32 * (longest row of the slice) for every slice; slices of segment q (a
// group, or a (group, tile) pair) start at slice index sg[q], its items at item_g[q]
// The items of the sliced copies are CSR rows read through an order: item k
// is row order[k] of (ptr, idx, val), or row k when order is NULL.  Rows go in
// (group, tile, length) order straight from the permuted matrix; mirror
// segments in (group, tile, length, column) order from the (group, column)
// ordered mirror.
template <class TO>
__device__ __forceinline__ int64_t item_row(const TO* order, int64_t k)
{
    return order ? (int64_t)order[k] : k;
}

template <class TO>
__global__ void sell_lengths(int64_t ns, int64_t G, const int64_t* sg, const int64_t* item_g,
                             const int64_t* ptr, const TO* order, int64_t* slen, int64_t* row0, int32_t* nrow)
{
    GRID_STRIDE(s, ns)
    {
        int64_t lo = 0, hi = G;  // group of slice s: largest g with sg[g] <= s
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) >> 1;
            if (sg[mid] <= s) lo = mid;
            else hi = mid;
        }
        int64_t k0 = item_g[lo] + (s - sg[lo]) * 32;
        int64_t k1 = k0 + 32 < item_g[lo + 1] ? k0 + 32 : item_g[lo + 1];
        int64_t mx = 0;
        for (int64_t k = k0; k < k1; ++k) {
            int64_t r = item_row(order, k);
            mx = max(mx, ptr[r + 1] - ptr[r]);
        }
        slen[s] = 32 * mx;
        if (row0) row0[s] = k0;
        if (nrow) nrow[s] = (int32_t)(k1 - k0);
    }
}

// entries of slice s, lane l: item row0[s] + l (rows) with the padding zeros.
// A padding entry (value 0) repeats the lane's last index, or the first index
// of the slice's first item for a lane without an item, so that its load
// stays inside the band the slice's step waits for.
template <class TI, class TO>
__global__ void sell_fill(int64_t ns, const int64_t* sl_ptr, const int64_t* row0, const int32_t* nrow,
                          const int64_t* ptr, const TO* order, const TI* idx, const double* val, TI* sidx,
                          double* sval, float* sval32)
{
    GRID_STRIDE(t, ns * 32)
    {
        int64_t s = t >> 5;
        int lane = (int)(t & 31);
        int64_t base = sl_ptr[s], len = (sl_ptr[s + 1] - base) >> 5;
        bool valid = lane < nrow[s];
        int64_t k = row0[s] + lane;
        int64_t r = valid ? item_row(order, k) : 0;
        int64_t b = valid ? ptr[r] : 0, rl = valid ? ptr[r + 1] - b : 0;
        TI pad_idx = rl > 0 ? idx[b + rl - 1] : idx[ptr[item_row(order, row0[s])]];
        for (int64_t j = 0; j < len; ++j) {
            int64_t q = base + 32 * j + lane;
            bool live = j < rl;
            double a = live ? val[b + j] : 0.0;
            sidx[q] = live ? idx[b + j] : pad_idx;
            sval[q] = a;
            if (sval32) sval32[q] = (float)a;
        }
    }
}

// Mirror slices of a (group, tile) piece with at least kMirrorDoubleMin
// segments hold 64 of them: lane l takes the neighbouring segments row0 + 2l
// (column a) and row0 + 2l + 1 (column b), of about the same length in the
// length order, their entries interleaved (even positions a, odd positions b,
// the shorter one padded), so that a slice costs one round of loads and
// gathers for twice the entries and the two columns' sums run as independent
// chains.  Slices of a smaller piece hold 32 segments, one per lane; their
// second column word is kOneColumn, which tells the sweep the format (dbl[s]
// tells msell_fill).
__global__ void msell_lengths(int64_t nms, int64_t G, const int64_t* sg, const int64_t* item_g, const int64_t* ptr,
                              const uint32_t* order, const int32_t* pdbl, int64_t* slen, int64_t* row0, int32_t* nrow,
                              int32_t* dbl)
{
    GRID_STRIDE(s, nms)
    {
        int64_t lo = 0, hi = G;  // piece of slice s: largest g with sg[g] <= s
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) >> 1;
            if (sg[mid] <= s) lo = mid;
            else hi = mid;
        }
        const int64_t w = pdbl[lo] ? 64 : 32;
        const int64_t k0 = item_g[lo] + (s - sg[lo]) * w;
        const int64_t k1 = k0 + w < item_g[lo + 1] ? k0 + w : item_g[lo + 1];
        int64_t mx = 0;
        for (int64_t k = k0; k < k1; ++k) {
            const int64_t r = order[k];
            mx = max(mx, ptr[r + 1] - ptr[r]);
        }
        slen[s] = w * mx;  // 32 lanes x (1 or 2 segments) x the longest segment
        row0[s] = k0;
        nrow[s] = (int32_t)(k1 - k0);
        dbl[s] = pdbl[lo];
    }
}

// entries and lane columns (mcol[64 s + l] = a, mcol[64 s + 32 + l] = b) of the
// mirror slices; a padding entry (value 0) repeats the last index of its
// column's segment, or the first index of the slice's first segment for a
// column without one, so that its load stays inside the band
__global__ void msell_fill(int64_t nms, const int64_t* ml_ptr, const int64_t* row0, const int32_t* nrow,
                           const int32_t* dbl, const int64_t* ptr, const uint32_t* order, const int32_t* seg_col,
                           const int32_t* idx, const double* val, int32_t* sidx, double* sval, float* sval32,
                           int32_t* mcol)
{
    GRID_STRIDE(t, nms * 32)
    {
        const int64_t s = t >> 5;
        const int lane = (int)(t & 31);
        const int64_t base = ml_ptr[s], len = (ml_ptr[s + 1] - base) >> 5;
        const int n = nrow[s];
        if (!dbl[s]) {  // one segment per lane, entries in order
            const bool va = lane < n;
            const int64_t ra = va ? (int64_t)order[row0[s] + lane] : 0;
            const int64_t ba = va ? ptr[ra] : 0, la = va ? ptr[ra + 1] - ba : 0;
            const int32_t pad = la > 0 ? idx[ba + la - 1] : idx[ptr[order[row0[s]]]];
            for (int64_t j = 0; j < len; ++j) {
                const int64_t q = base + 32 * j + lane;
                const bool live = j < la;
                const double a = live ? val[ba + j] : 0.0;
                sidx[q] = live ? idx[ba + j] : pad;
                sval[q] = a;
                if (sval32) sval32[q] = (float)a;
            }
            mcol[s * 64 + lane] = va ? seg_col[ra] : -1;
            mcol[s * 64 + 32 + lane] = kOneColumn;
            continue;
        }
        const bool va = 2 * lane < n, vb = 2 * lane + 1 < n;
        const int64_t ra = va ? (int64_t)order[row0[s] + 2 * lane] : 0;
        const int64_t rb = vb ? (int64_t)order[row0[s] + 2 * lane + 1] : 0;
        const int64_t ba = va ? ptr[ra] : 0, la = va ? ptr[ra + 1] - ba : 0;
        const int64_t bb = vb ? ptr[rb] : 0, lb = vb ? ptr[rb + 1] - bb : 0;
        const int32_t first = idx[ptr[order[row0[s]]]];
        const int32_t pad_a = la > 0 ? idx[ba + la - 1] : first;
        const int32_t pad_b = lb > 0 ? idx[bb + lb - 1] : pad_a;
        for (int64_t j = 0; j < len; ++j) {
            const int64_t q = base + 32 * j + lane;
            const int64_t u = j >> 1;
            int32_t c;
            double a = 0.0;
            if ((j & 1) == 0) {
                c = pad_a;
                if (u < la) { c = idx[ba + u]; a = val[ba + u]; }
            } else {
                c = pad_b;
                if (u < lb) { c = idx[bb + u]; a = val[bb + u]; }
            }
            sidx[q] = c;
            sval[q] = a;
            if (sval32) sval32[q] = (float)a;
        }
        mcol[s * 64 + lane] = va ? seg_col[ra] : -1;
        mcol[s * 64 + 32 + lane] = vb ? seg_col[rb] : -1;
    }
}

}  // namespace

int64_t max_segment_length(int64_t n, const int64_t* ptr, cudaStream_t st)
{
    DBuf<unsigned long long> mx(1, st);
    OBK_CUDA(cudaMemsetAsync(mx.p, 0, sizeof(unsigned long long), st));
    max_row_len<<<grid_for(n), kBlock, 0, st>>>(n, ptr, mx.p);
    OBK_CHECK_LAUNCH();
    return (int64_t)read_scalar(mx.p, st);
}

void validate_csr(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                  int64_t nnz, int* d_bad, cudaStream_t st)
{
    OBK_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int), st));
    validate_rows<<<grid_for(m), kBlock, 0, st>>>(m, n, rp, ci, v, nnz, d_bad);
    OBK_CHECK_LAUNCH();
}

int64_t half_bandwidth(int64_t N, const int64_t* rp, const int32_t* ci, int64_t nnz, cudaStream_t st)
{
    (void)nnz;
    DBuf<unsigned long long> bw(1, st);
    OBK_CUDA(cudaMemsetAsync(bw.p, 0, sizeof(unsigned long long), st));
    bandwidth_kernel<<<grid_for(N), kBlock, 0, st>>>(N, rp, ci, bw.p);
    OBK_CHECK_LAUNCH();
    return (int64_t)read_scalar(bw.p, st);
}

void permute_csr(int64_t N, const int64_t* rp, const int32_t* ci, const double* v, int64_t nnz,
                 const int32_t* perm, int32_t* iperm, int64_t* rp_t, int32_t* ci_t, double* v_t,
                 cudaStream_t st)
{
    inverse_perm<<<grid_for(N), kBlock, 0, st>>>(N, perm, iperm);
    OBK_CHECK_LAUNCH();
    DBuf<int64_t> len(N, st);
    permuted_lengths<<<grid_for(N), kBlock, 0, st>>>(N, rp, perm, len.p);
    OBK_CHECK_LAUNCH();
    exclusive_scan_i64(len.p, rp_t, N, st);
    if (nnz == 0) return;
    if (max_segment_length(N, rp, st) <= 32) {
        permute_rows_warp<<<grid_for(N * 32), kBlock, 0, st>>>(N, rp, ci, v, perm, iperm, rp_t, ci_t, v_t);
        OBK_CHECK_LAUNCH();
        return;
    }
    DBuf<uint32_t> keys(nnz, st), src(nnz, st);
    permute_gather<<<grid_for(N * 32), kBlock, 0, st>>>(N, rp, ci, perm, iperm, rp_t, keys.p, src.p);
    OBK_CHECK_LAUNCH();
    segmented_sort_u32(rp_t, N, keys.p, src.p, st);
    permute_finish<<<grid_for(nnz), kBlock, 0, st>>>(nnz, keys.p, src.p, v, ci_t, v_t);
    OBK_CHECK_LAUNCH();
}

// (column lists of a CSR matrix: see kernels.cuh)
void build_csc(int64_t nrows, int64_t ncols, const int64_t* rp, const int32_t* ci, const double* v, int64_t nnz,
               DBuf<int64_t>& cptr, DBuf<int32_t>& crow, DBuf<double>& cval, DBuf<int64_t>& pos_of,
               cudaStream_t st)
{
    DBuf<uint32_t> trow, tsrc;
    bool sym = false;
    transpose_pattern(nrows, ncols, rp, ci, nnz, cptr, trow, tsrc, st, &sym, false);
    pos_of.alloc(std::max<int64_t>(nnz, 1), st);
    crow.alloc(std::max<int64_t>(nnz, 1), st);
    cval.alloc(std::max<int64_t>(nnz, 1), st);
    if (nnz && sym) {
        // the transpose has the pattern itself: its rows are the column
        // indices, and the slot map pairs each entry with its mirror both ways
        OBK_CUDA(cudaMemcpyAsync(crow.p, ci, nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        csc_fill_symmetric<<<grid_for(nnz), kBlock, 0, st>>>(nnz, tsrc.p, v, cval.p, pos_of.p);
        OBK_CHECK_LAUNCH();
    } else if (nnz) {
        csc_fill<<<grid_for(nnz), kBlock, 0, st>>>(nnz, tsrc.p, trow.p, v, crow.p, cval.p, pos_of.p);
        OBK_CHECK_LAUNCH();
    }
}

namespace {

__global__ void gm_norms(int64_t Ngm, const int32_t* grp_row, const double* nsq, double* nsq_gm, double* s_gm)
{
    GRID_STRIDE(k, Ngm)
    {
        double q = nsq[grp_row[k]];
        nsq_gm[k] = q;
        s_gm[k] = sqrt(q);
    }
}

}  // namespace

void cosine_stats(SweepLayout& L, int64_t* nz, uint64_t* sum, int* d_err, cudaStream_t st)
{
    ensure_gm_csr(L, st);
    int64_t Ngm = L.Ngm, N = L.N, nnz = L.nnz_gm;
    if (Ngm == 0) {
        *nz = 0;
        *sum = 0;
        return;
    }
    DevInfo di = dev_info();
    // the group-major rows are the nonzero rows of the permuted matrix (columns in
    // its numbering, ascending): their dot products fold in the same order
    DBuf<double> nsq(Ngm, st), s(Ngm, st);
    gm_norms<<<grid_for(Ngm), kBlock, 0, st>>>(Ngm, L.grp_row.p, L.nsq.p, nsq.p, s.p);
    OBK_CHECK_LAUNCH();
    DBuf<int64_t> cptr, pos_of;
    DBuf<int32_t> crow;
    DBuf<double> cval;
    build_csc(Ngm, N, L.grp_rp.p, L.grp_ci.p, L.grp_v.p, nnz, cptr, crow, cval, pos_of, st);
    DBuf<int64_t> ub(Ngm, st), bigsz(Ngm, st), bigoff(Ngm + 1, st);
    pair_upper_bound<<<grid_for(Ngm), kBlock, 0, st>>>(Ngm, L.grp_rp.p, L.grp_ci.p, cptr.p, pos_of.p, ub.p);
    OBK_CHECK_LAUNCH();
    big_table_sizes<<<grid_for(Ngm), kBlock, 0, st>>>(Ngm, ub.p, kPairCap, bigsz.p);
    OBK_CHECK_LAUNCH();
    exclusive_scan_i64(bigsz.p, bigoff.p, Ngm, st);
    int64_t big_total = read_scalar(bigoff.p + Ngm, st);
    DBuf<int32_t> big_key(std::max<int64_t>(big_total, 1), st);
    DBuf<double> big_val(std::max<int64_t>(big_total, 1), st);
    DBuf<unsigned long long> acc(2, st);
    OBK_CUDA(cudaMemsetAsync(acc.p, 0, 2 * sizeof(unsigned long long), st));
    PairParams pp{Ngm, L.grp_rp.p, L.grp_ci.p, L.grp_v.p, cptr.p, crow.p, cval.p, pos_of.p, nsq.p, s.p, 0.0, ub.p,
                  bigoff.p, big_key.p, big_val.p, nullptr, nullptr, nullptr, 0, nullptr, nullptr, d_err, acc.p,
                  nullptr, nullptr};
    int blocks = (int)std::min<int64_t>(ceil_div(Ngm, kPairWarps), (int64_t)di.sms * 16);
    pair_conflicts<kPairStats><<<blocks, kPairWarps * 32, 0, st>>>(pp);
    OBK_CHECK_LAUNCH();
    if (read_scalar(d_err, st) != 0) throw Error{-5, "internal error: pair table overflow"};
    unsigned long long h[2];
    OBK_CUDA(cudaMemcpyAsync(h, acc.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    OBK_CUDA(cudaStreamSynchronize(st));
    *nz = (int64_t)h[0];
    *sum = (uint64_t)h[1];
}


namespace {

__global__ void gm_group_start(int64_t Ngm, int64_t G, const int64_t* gptr, int64_t* gstart)
{
    GRID_STRIDE(k, Ngm)
    {
        int64_t lo = 0, hi = G;  // the group g with gptr[g] <= k < gptr[g+1]
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) >> 1;
            if (gptr[mid] <= k) lo = mid;
            else hi = mid;
        }
        gstart[k] = gptr[lo];
    }
}

// both directions of every listed pair: key row * Ngm + partner, value = the pair's slot
__global__ void gram_directed(int64_t Ngm, const int32_t* cnt, const int64_t* off, const int32_t* pool,
                              uint64_t* keys, uint32_t* slot)
{
    GRID_STRIDE(i, Ngm)
    {
        for (int t = 0; t < cnt[i]; ++t) {
            int64_t q = off[i] + t;
            uint64_t j = (uint64_t)pool[q];
            keys[2 * q] = (uint64_t)i * (uint64_t)Ngm + j;
            keys[2 * q + 1] = j * (uint64_t)Ngm + (uint64_t)i;
            slot[2 * q] = (uint32_t)q;
            slot[2 * q + 1] = (uint32_t)q;
        }
    }
}

__global__ void gram_fill(int64_t n, int64_t Ngm, const uint64_t* keys, const uint32_t* slot, const double* pool_val,
                          int32_t* idx, double* val, int64_t* rowcnt)
{
    GRID_STRIDE(t, n)
    {
        uint64_t k = keys[t];
        idx[t] = (int32_t)(k % (uint64_t)Ngm);
        val[t] = pool_val[slot[t]];
        atomicAdd((unsigned long long*)(rowcnt + k / (uint64_t)Ngm), 1ull);
    }
}

}  // namespace

void build_group_gram(SweepLayout& L, int* d_err, cudaStream_t st)
{
    ensure_gm_csr(L, st);
    int64_t Ngm = L.Ngm, N = L.N, nnz = L.nnz_gm;
    L.gram_ptr.alloc(Ngm + 1, st);
    OBK_CUDA(cudaMemsetAsync(L.gram_ptr.p, 0, (Ngm + 1) * sizeof(int64_t), st));
    if (Ngm == 0) {
        L.gram_idx.alloc(1, st);
        L.gram_val.alloc(1, st);
        L.has_gram = true;
        return;
    }
    DevInfo di = dev_info();
    DBuf<double> nsq(Ngm, st), s(Ngm, st);
    gm_norms<<<grid_for(Ngm), kBlock, 0, st>>>(Ngm, L.grp_row.p, L.nsq.p, nsq.p, s.p);
    OBK_CHECK_LAUNCH();
    DBuf<int64_t> cptr, pos_of;
    DBuf<int32_t> crow;
    DBuf<double> cval;
    build_csc(Ngm, N, L.grp_rp.p, L.grp_ci.p, L.grp_v.p, nnz, cptr, crow, cval, pos_of, st);
    DBuf<int64_t> ub(Ngm, st), bigsz(Ngm, st), bigoff(Ngm + 1, st), gstart(Ngm, st);
    pair_upper_bound<<<grid_for(Ngm), kBlock, 0, st>>>(Ngm, L.grp_rp.p, L.grp_ci.p, cptr.p, pos_of.p, ub.p);
    OBK_CHECK_LAUNCH();
    big_table_sizes<<<grid_for(Ngm), kBlock, 0, st>>>(Ngm, ub.p, kPairCap, bigsz.p);
    OBK_CHECK_LAUNCH();
    exclusive_scan_i64(bigsz.p, bigoff.p, Ngm, st);
    gm_group_start<<<grid_for(Ngm), kBlock, 0, st>>>(Ngm, L.G, L.gptr.p, gstart.p);
    OBK_CHECK_LAUNCH();
    int64_t big_total = read_scalar(bigoff.p + Ngm, st);
    DBuf<int32_t> big_key(std::max<int64_t>(big_total, 1), st);
    DBuf<double> big_val(std::max<int64_t>(big_total, 1), st);
    DBuf<int32_t> cnt(Ngm, st);
    DBuf<int64_t> off(Ngm, st);
    DBuf<unsigned long long> counters(2, st);
    int64_t pool_cap = 8 * Ngm + 1024;
    DBuf<int32_t> pool;
    DBuf<double> pool_val;
    unsigned long long used = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        pool.alloc(pool_cap, st);
        pool_val.alloc(pool_cap, st);
        OBK_CUDA(cudaMemsetAsync(counters.p, 0, 2 * sizeof(unsigned long long), st));
        PairParams pp{Ngm, L.grp_rp.p, L.grp_ci.p, L.grp_v.p, cptr.p, crow.p, cval.p, pos_of.p, nsq.p, s.p, 0.0,
                      ub.p, bigoff.p, big_key.p, big_val.p, cnt.p, off.p, pool.p, pool_cap, counters.p,
                      counters.p + 1, d_err, nullptr, gstart.p, pool_val.p};
        int blocks = (int)std::min<int64_t>(ceil_div(Ngm, kPairWarps), (int64_t)di.sms * 16);
        pair_conflicts<kPairGram><<<blocks, kPairWarps * 32, 0, st>>>(pp);
        OBK_CHECK_LAUNCH();
        if (read_scalar(d_err, st) != 0) throw Error{-5, "internal error: pair table overflow"};
        used = read_scalar(counters.p, st);
        if ((int64_t)used <= pool_cap) break;
        pool_cap = (int64_t)used + 1024;
    }
    int64_t M = 2 * (int64_t)used;  // directed entries
    L.gram_idx.alloc(std::max<int64_t>(M, 1), st);
    L.gram_val.alloc(std::max<int64_t>(M, 1), st);
    if (M > 0) {
        DBuf<uint64_t> keys(M, st);
        DBuf<uint32_t> slot(M, st);
        gram_directed<<<grid_for(Ngm), kBlock, 0, st>>>(Ngm, cnt.p, off.p, pool.p, keys.p, slot.p);
        OBK_CHECK_LAUNCH();
        radix_sort_pairs(keys.p, slot.p, M, bits_for((uint64_t)Ngm * (uint64_t)Ngm - 1), st);
        DBuf<int64_t> rowcnt(Ngm, st);
        OBK_CUDA(cudaMemsetAsync(rowcnt.p, 0, Ngm * sizeof(int64_t), st));
        gram_fill<<<grid_for(M), kBlock, 0, st>>>(M, Ngm, keys.p, slot.p, pool_val.p, L.gram_idx.p, L.gram_val.p,
                                                 rowcnt.p);
        OBK_CHECK_LAUNCH();
        exclusive_scan_i64(rowcnt.p, L.gram_ptr.p, Ngm, st);
    }
    OBK_CUDA(cudaStreamSynchronize(st));
    L.has_gram = true;
}

// Sliced copies of the group-major rows and of the mirror segments: slices of
// 32 are cut inside each (group, tile) segment, so the slices of one block's
// tiles are contiguous in every group.
void build_sell(SweepLayout& L, const int64_t* rp, const int32_t* ci, const double* v, bool want_fp32,
                cudaStream_t st)
{
    int64_t G = L.G, T = L.T, nsegs = G * T;
    // first slice of each group (slice index of segment g * T)
    L.h_sl_gptr.resize(G + 1);
    L.h_ml_gptr.resize(G + 1);
    for (int64_t g = 0; g <= G; ++g) {
        L.h_sl_gptr[g] = L.h_sl_tptr[g * T];
        L.h_ml_gptr[g] = L.h_ml_tptr[g * T];
    }
    auto upload = [&](DBuf<int64_t>& d, const std::vector<int64_t>& h) {
        d.alloc(h.size(), st);
        OBK_CUDA(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    };
    upload(L.sl_gptr, L.h_sl_gptr);
    upload(L.ml_gptr, L.h_ml_gptr);
    upload(L.sl_tptr, L.h_sl_tptr);
    upload(L.ml_tptr, L.h_ml_tptr);
    // rows
    int64_t ns = L.h_sl_tptr[nsegs];
    L.ns = ns;
    DBuf<int64_t> slen(std::max<int64_t>(ns, 1), st);
    L.sl_ptr.alloc(ns + 1, st);
    L.sl_row0.alloc(std::max<int64_t>(ns, 1), st);
    L.sl_nrow.alloc(std::max<int64_t>(ns, 1), st);
    if (ns) {
        sell_lengths<int32_t><<<grid_for(ns), kBlock, 0, st>>>(ns, nsegs, L.sl_tptr.p, L.gt_ptr.p, rp, L.grp_row.p,
                                                               slen.p, L.sl_row0.p, L.sl_nrow.p);
        OBK_CHECK_LAUNCH();
    }
    exclusive_scan_i64(slen.p, L.sl_ptr.p, ns, st);
    L.sell_nnz = read_scalar(L.sl_ptr.p + ns, st);
    L.sci.alloc(std::max<int64_t>(L.sell_nnz, 1), st);
    L.sv.alloc(std::max<int64_t>(L.sell_nnz, 1), st);
    if (want_fp32) L.sv32.alloc(std::max<int64_t>(L.sell_nnz, 1), st);
    if (ns) {
        sell_fill<int32_t, int32_t><<<grid_for(ns * 32), kBlock, 0, st>>>(ns, L.sl_ptr.p, L.sl_row0.p, L.sl_nrow.p,
                                                                          rp, L.grp_row.p, ci, v, L.sci.p, L.sv.p,
                                                                          want_fp32 ? L.sv32.p : nullptr);
        OBK_CHECK_LAUNCH();
    }
    // mirror segments
    int64_t nms = L.h_ml_tptr[nsegs];
    L.nms = nms;
    DBuf<int64_t> mlen(std::max<int64_t>(nms, 1), st), mrow0(std::max<int64_t>(nms, 1), st);
    DBuf<int32_t> mnrow(std::max<int64_t>(nms, 1), st);
    L.ml_ptr.alloc(nms + 1, st);
    DBuf<int32_t> mdbl(std::max<int64_t>(nms, 1), st);
    if (nms) {
        DBuf<int32_t> pdbl(std::max<int64_t>(nsegs, 1), st);
        OBK_CUDA(cudaMemcpyAsync(pdbl.p, L.h_ml_pdbl.data(), nsegs * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        msell_lengths<<<grid_for(nms), kBlock, 0, st>>>(nms, nsegs, L.ml_tptr.p, L.gts_ptr.p, L.seg_ptr.p,
                                                         L.seg_order.p, pdbl.p, mlen.p, mrow0.p, mnrow.p, mdbl.p);
        OBK_CHECK_LAUNCH();
    }
    exclusive_scan_i64(mlen.p, L.ml_ptr.p, nms, st);
    L.msell_nnz = read_scalar(L.ml_ptr.p + nms, st);
    L.mcol.alloc(std::max<int64_t>(nms * 64, 1), st);
    L.mrow.alloc(std::max<int64_t>(L.msell_nnz, 1), st);
    L.mv.alloc(std::max<int64_t>(L.msell_nnz, 1), st);
    if (want_fp32) L.mv32.alloc(std::max<int64_t>(L.msell_nnz, 1), st);
    if (nms) {
        msell_fill<<<grid_for(nms * 32), kBlock, 0, st>>>(nms, L.ml_ptr.p, mrow0.p, mnrow.p, mdbl.p, L.seg_ptr.p,
                                                          L.seg_order.p, L.seg_col.p, L.mir_row.p, L.mir_val.p,
                                                          L.mrow.p, L.mv.p, want_fp32 ? L.mv32.p : nullptr, L.mcol.p);
        OBK_CHECK_LAUNCH();
    }
}

void ensure_gm_csr(SweepLayout& L, cudaStream_t st)
{
    if (L.has_gm_csr) return;
    int64_t nnz_gm = L.nnz_gm;
    L.grp_ci.alloc(std::max<int64_t>(nnz_gm, 1), st);
    L.grp_v.alloc(std::max<int64_t>(nnz_gm, 1), st);
    if (L.want_fp32) L.grp_v32.alloc(std::max<int64_t>(nnz_gm, 1), st);
    if (L.Ngm) {
        gm_copy<<<grid_for(L.Ngm * 32), kBlock, 0, st>>>(L.Ngm, L.grp_row.p, L.src_rp, L.src_ci, L.src_v, L.grp_rp.p,
                                                         L.grp_ci.p, L.grp_v.p, L.want_fp32 ? L.grp_v32.p : nullptr);
        OBK_CHECK_LAUNCH();
    }
    L.has_gm_csr = true;
}

void group_build(int64_t N, const int64_t* rp, const int32_t* ci, const double* v, int64_t nnz,
                 double thr, long long spin_limit, int* d_err, SweepLayout& L, bool want_fp32,
                 cudaStream_t st, StageClock* clock)
{
    auto mark = [&]() {
        if (clock) clock->mark(st);
    };
    DevInfo di = dev_info();
    L.N = N;
    L.nnz = nnz;
    // 1. exact row norms
    L.nsq.alloc(N, st);
    DBuf<double> s(N, st);
    row_norms_exact<<<grid_for(N), kBlock, 0, st>>>(N, rp, v, L.nsq.p, s.p);
    OBK_CHECK_LAUNCH();

    // 2. transpose (rows ascending inside each column)
    DBuf<int64_t> cptr, pos_of;
    DBuf<int32_t> crow;
    DBuf<double> cval;
    build_csc(N, N, rp, ci, v, nnz, cptr, crow, cval, pos_of, st);

    mark();
    // 3. pair cosines -> lower conflict lists
    DBuf<int64_t> ub(N, st), bigsz(N, st), bigoff(N + 1, st);
    pair_upper_bound<<<grid_for(N), kBlock, 0, st>>>(N, rp, ci, cptr.p, pos_of.p, ub.p);
    OBK_CHECK_LAUNCH();
    big_table_sizes<<<grid_for(N), kBlock, 0, st>>>(N, ub.p, kPairCap, bigsz.p);
    OBK_CHECK_LAUNCH();
    exclusive_scan_i64(bigsz.p, bigoff.p, N, st);
    int64_t big_total = read_scalar(bigoff.p + N, st);
    DBuf<int32_t> big_key(big_total, st);
    DBuf<double> big_val(big_total, st);
    DBuf<int32_t> conf_cnt(N, st);
    DBuf<int64_t> conf_off(N, st);
    DBuf<unsigned long long> counters(2, st);
    // the candidates (earlier rows sharing a column) bound the conflicts: a
    // pool that holds them all needs one pass; past 24 per entry it starts
    // smaller and grows once if needed
    int64_t cand_total = 0;
    {
        DBuf<int64_t> ubscan(N + 1, st);
        exclusive_scan_i64(ub.p, ubscan.p, N, st);
        cand_total = read_scalar(ubscan.p + N, st);
    }
    int64_t pool_cap = std::min(cand_total, std::max<int64_t>(8 * N, 24 * nnz)) + 1024;
    DBuf<int32_t> pool;
    for (int attempt = 0; attempt < 2; ++attempt) {
        pool.alloc(pool_cap, st);
        OBK_CUDA(cudaMemsetAsync(counters.p, 0, 2 * sizeof(unsigned long long), st));
        PairParams pp{N, rp, ci, v, cptr.p, crow.p, cval.p, pos_of.p, L.nsq.p, s.p, thr, ub.p,
                      bigoff.p, big_key.p, big_val.p, conf_cnt.p, conf_off.p, pool.p, pool_cap,
                      counters.p, counters.p + 1, d_err, nullptr, nullptr, nullptr};
        int blocks = (int)std::min<int64_t>(ceil_div(N, kPairWarps), (int64_t)di.sms * 16);
        pair_conflicts<kPairConflicts><<<blocks, kPairWarps * 32, 0, st>>>(pp);
        OBK_CHECK_LAUNCH();
        if (read_scalar(d_err, st) != 0) throw Error{-5, "internal error: pair table overflow"};
        unsigned long long used = read_scalar(counters.p, st);
        L.n_conflicts = (int64_t)read_scalar(counters.p + 1, st);
        if ((int64_t)used <= pool_cap) break;
        pool_cap = (int64_t)used + 1024;
    }
    big_key.release();
    big_val.release();

    mark();
    // 4. greedy first-fit colouring
    L.group_of.alloc(N, st);
    {
        DBuf<int> changed(3, st);
        DBuf<int64_t> rounds(1, st);
        DBuf<unsigned> bar(kBarrierWords, st);
        OBK_CUDA(cudaMemsetAsync(changed.p, 0, 3 * sizeof(int), st));
        OBK_CUDA(cudaMemsetAsync(bar.p, 0, kBarrierWords * sizeof(unsigned), st));
        ColorParams cp{N, L.nsq.p, conf_cnt.p, conf_off.p, pool.p, L.group_of.p, changed.p, rounds.p, 1,
                       GridBarrier{bar.p, d_err, spin_limit}};
        // lanes per row from the mean conflict-list length
        double mean_list = N > 0 ? (double)L.n_conflicts / (double)N : 0.0;
        int lanes = mean_list <= 6.0 ? 1 : mean_list <= 24.0 ? 4 : mean_list <= 96.0 ? 8 : 32;
        const void* fn = lanes == 1   ? (const void*)greedy_color<1>
                         : lanes == 4 ? (const void*)greedy_color<4>
                         : lanes == 8 ? (const void*)greedy_color<8>
                                      : (const void*)greedy_color<32>;
        int cgrid = coop_grid(fn, kBlock, 0, ceil_div(N * lanes, (int64_t)kBlock));
        // runs of consecutive rows per lane group: after RCM most conflicts
        // join nearby rows, and a run resolves their chains in one round.
        // One lane per row (short lists): each thread takes one contiguous
        // chunk of the rows (4M kNN: 29-30 rounds and 2.5 ms instead of 36-45
        // rounds and 2.8-3.5 ms with runs of 8); more lanes per row: runs of
        // up to 8 (longer runs unbalance the rounds of long conflict lists)
        cp.run = lanes == 1 ? ceil_div(N, (int64_t)cgrid * kBlock)
                            : std::min<int64_t>(8, ceil_div(N, (int64_t)cgrid * kBlock / lanes));
        void* args[] = {&cp};
        OBK_COOP_LAUNCH(fn, cgrid, kBlock, args, st);
        if (read_scalar(d_err, st) != 0) throw Error{-4, "bounded wait expired in greedy grouping"};
        L.color_rounds = read_scalar(rounds.p, st);
    }
    DBuf<int> gmax(1, st);
    OBK_CUDA(cudaMemsetAsync(gmax.p, 0xff, sizeof(int), st));
    max_color<<<grid_for(N), kBlock, 0, st>>>(N, L.group_of.p, gmax.p);
    OBK_CHECK_LAUNCH();
    int G = read_scalar(gmax.p, st) + 1;
    L.G = G;
    pool.release();
    conf_cnt.release();
    conf_off.release();

    mark();
    // 5. group-major rows, ordered by (group, tile, length, index)
    const int64_t T = sweep_tiles(N);
    const int64_t B = ceil_div(N, T);
    L.T = T;
    L.B = B;
    const int64_t nsegs = (int64_t)G * T;
    const int sbits = bits_for((uint64_t)(nsegs + T));  // (group, tile) index, rows of no group included
    DBuf<uint64_t> gk(N, st);
    DBuf<uint32_t> gorder(N, st);
    // length classes: every length up to the longest row (capped at 1023, longer
    // rows share the last class)
    int lbits = std::min(10, bits_for((uint64_t)max_segment_length(N, rp, st)));
    color_keys<<<grid_for(N), kBlock, 0, st>>>(N, L.group_of.p, rp, G, B, T, lbits, gk.p, gorder.p);
    OBK_CHECK_LAUNCH();
    radix_sort_pairs(gk.p, gorder.p, N, sbits + lbits, st);
    DBuf<int64_t> gt_ptr(nsegs + 1, st);
    segment_starts<<<grid_for(N + 1), kBlock, 0, st>>>(N, gk.p, lbits, nsegs, gt_ptr.p);
    OBK_CHECK_LAUNCH();
    gk.release();
    std::vector<int64_t> h_gt(nsegs + 1);
    OBK_CUDA(cudaMemcpyAsync(h_gt.data(), gt_ptr.p, (nsegs + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    OBK_CUDA(cudaStreamSynchronize(st));
    L.h_gptr.resize(G + 1);
    for (int64_t g = 0; g <= G; ++g) L.h_gptr[g] = h_gt[g * T];
    L.gptr.alloc(G + 1, st);
    OBK_CUDA(cudaMemcpyAsync(L.gptr.p, L.h_gptr.data(), (G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    int64_t Ngm = L.h_gptr[G];
    L.Ngm = Ngm;
    // slices of 32 rows inside each (group, tile) segment
    L.h_sl_tptr.assign(nsegs + 1, 0);
    for (int64_t q = 0; q < nsegs; ++q) L.h_sl_tptr[q + 1] = L.h_sl_tptr[q] + ceil_div(h_gt[q + 1] - h_gt[q], (int64_t)32);
    L.gt_ptr = std::move(gt_ptr);
    // tile dependency reach (rows of the tile -> tiles of their columns, and back)
    L.reach_lo.alloc(T, st);
    L.reach_hi.alloc(T, st);
    tile_reach<<<(unsigned)T, kBlock, 0, st>>>(N, B, rp, ci, cptr.p, crow.p, L.reach_lo.p, L.reach_hi.p);
    OBK_CHECK_LAUNCH();
    {
        std::vector<int32_t> hlo(T), hhi(T);
        OBK_CUDA(cudaMemcpyAsync(hlo.data(), L.reach_lo.p, T * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        OBK_CUDA(cudaMemcpyAsync(hhi.data(), L.reach_hi.p, T * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        OBK_CUDA(cudaStreamSynchronize(st));
        L.xwin_max = L.ywin_max = 0;
        for (int64_t t = 0; t < T; ++t) {
            L.xwin_max = std::max<int64_t>(L.xwin_max, std::min<int64_t>((int64_t)(hhi[t] + 1) * B, N) - (int64_t)hlo[t] * B);
            for (int64_t g = 0; g < G; ++g)
                L.ywin_max = std::max<int64_t>(L.ywin_max, h_gt[g * T + hhi[t] + 1] - h_gt[g * T + hlo[t]]);
        }
    }
    DBuf<int32_t> gm_of_row(N, st);
    OBK_CUDA(cudaMemsetAsync(gm_of_row.p, 0xff, N * sizeof(int32_t), st));
    L.grp_row.alloc(Ngm, st);
    L.grp_inv.alloc(Ngm, st);
    if (want_fp32) L.grp_inv32.alloc(Ngm, st);
    DBuf<int64_t> glen(Ngm, st);
    gm_rows<<<grid_for(Ngm), kBlock, 0, st>>>(Ngm, gorder.p, rp, L.nsq.p, L.grp_row.p, gm_of_row.p, glen.p,
                                              L.grp_inv.p, want_fp32 ? L.grp_inv32.p : nullptr);
    OBK_CHECK_LAUNCH();
    L.grp_rp.alloc(Ngm + 1, st);
    exclusive_scan_i64(glen.p, L.grp_rp.p, Ngm, st);
    int64_t nnz_gm = read_scalar(L.grp_rp.p + Ngm, st);
    L.nnz_gm = nnz_gm;
    // the group-major copy of the entries is built on first use (ensure_gm_csr):
    // the sliced copies read the permuted matrix directly
    L.src_rp = rp;
    L.src_ci = ci;
    L.src_v = v;
    L.want_fp32 = want_fp32;
    L.has_gm_csr = false;

    mark();
    // 6. column mirror: CSC entries stably partitioned by the group of their row
    DBuf<uint64_t> mk(nnz, st);
    DBuf<uint32_t> morder(nnz, st);
    DBuf<int32_t> col_of(nnz, st);
    if (nnz) {
        csc_color_keys<<<grid_for(nnz), kBlock, 0, st>>>(nnz, crow.p, L.group_of.p, G, mk.p, morder.p);
        OBK_CHECK_LAUNCH();
        radix_sort_pairs(mk.p, morder.p, nnz, bits_for((uint64_t)G), st);
        expand_cols<<<grid_for(N), kBlock, 0, st>>>(N, cptr.p, col_of.p);
        OBK_CHECK_LAUNCH();
    }
    mk.release();
    // grouped entries come first (zero rows were keyed G)
    int64_t M = nnz_gm;
    L.mir_row.alloc(M, st);
    L.mir_val.alloc(M, st);
    if (want_fp32) L.mir_val32.alloc(M, st);
    DBuf<int32_t> flag(M, st);
    DBuf<int64_t> fscan(M + 1, st);
    if (M) {
        mirror_fill<<<grid_for(M), kBlock, 0, st>>>(M, morder.p, crow.p, cval.p, col_of.p, L.group_of.p,
                                                   gm_of_row.p, L.mir_row.p, L.mir_val.p,
                                                   want_fp32 ? L.mir_val32.p : nullptr, flag.p);
        OBK_CHECK_LAUNCH();
    }
    exclusive_scan_i32_to_i64(flag.p, fscan.p, M, st);
    int64_t nseg = read_scalar(fscan.p + M, st);
    L.nseg = nseg;
    L.seg_ptr.alloc(nseg + 1, st);
    L.seg_col.alloc(nseg, st);
    L.gseg_ptr.alloc(G + 1, st);
    OBK_CUDA(cudaMemcpyAsync(L.seg_ptr.p + nseg, &M, sizeof(int64_t), cudaMemcpyHostToDevice, st));
    OBK_CUDA(cudaMemcpyAsync(L.gseg_ptr.p + G, &nseg, sizeof(int64_t), cudaMemcpyHostToDevice, st));
    if (M) {
        mirror_segments<<<grid_for(M), kBlock, 0, st>>>(M, morder.p, crow.p, col_of.p, L.group_of.p, flag.p,
                                                       fscan.p, L.seg_ptr.p, L.seg_col.p, L.gseg_ptr.p);
        OBK_CHECK_LAUNCH();
    }
    // 7. the order of the segments in the sliced copy: by (group, tile of the
    // column, length, column); the mirror itself stays in (group, column) order
    // and the sliced copy reads it through this order
    DBuf<int64_t> gts_ptr(nsegs + 1, st);
    L.seg_order.alloc(std::max<int64_t>(nseg, 1), st);
    if (nseg >= 1) {
        DBuf<uint64_t> sk(nseg, st);
        int slbits = std::min(10, bits_for((uint64_t)max_segment_length(nseg, L.seg_ptr.p, st)));
        seg_keys<<<grid_for(nseg), kBlock, 0, st>>>(nseg, L.seg_ptr.p, L.gseg_ptr.p, L.seg_col.p, G, B, T, slbits,
                                                    sk.p, L.seg_order.p);
        OBK_CHECK_LAUNCH();
        radix_sort_pairs(sk.p, L.seg_order.p, nseg, sbits + slbits, st);
        segment_starts<<<grid_for(nseg + 1), kBlock, 0, st>>>(nseg, sk.p, slbits, nsegs, gts_ptr.p);
        OBK_CHECK_LAUNCH();
    } else {
        OBK_CUDA(cudaMemsetAsync(gts_ptr.p, 0, (nsegs + 1) * sizeof(int64_t), st));
    }
    {
        std::vector<int64_t> h_gts(nsegs + 1);
        OBK_CUDA(cudaMemcpyAsync(h_gts.data(), gts_ptr.p, (nsegs + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost,
                                 st));
        OBK_CUDA(cudaStreamSynchronize(st));
        L.h_ml_tptr.assign(nsegs + 1, 0);
        L.h_ml_pdbl.assign(nsegs, 0);
        for (int64_t q = 0; q < nsegs; ++q) {
            const int64_t items = h_gts[q + 1] - h_gts[q];
            L.h_ml_pdbl[q] = items >= kMirrorDoubleMin ? 1 : 0;
            L.h_ml_tptr[q + 1] = L.h_ml_tptr[q] + ceil_div(items, (int64_t)(L.h_ml_pdbl[q] ? 64 : 32));
        }
        L.gts_ptr = std::move(gts_ptr);
    }
    mark();
    L.h_gseg_ptr.resize(G + 1);
    OBK_CUDA(cudaMemcpyAsync(L.h_gseg_ptr.data(), L.gseg_ptr.p, (G + 1) * sizeof(int64_t),
                             cudaMemcpyDeviceToHost, st));
    OBK_CUDA(cudaStreamSynchronize(st));
    // 8. sliced ELL copies for the persistent sweep
    build_sell(L, rp, ci, v, want_fp32, st);
}

}  // namespace obk
