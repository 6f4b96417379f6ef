// sweep.cu -- the orthogonal-group Kaczmarz sweep (paper Eq. 1.2 / Eq. 1.3 /
// Eq. 3.3, Algorithm 4), the residual check and the FP32-sweep / FP64
// refinement form, in one persistent cooperative kernel per solve.
//
// One group step (rows of group g are mutually near-orthogonal):
//   phase 1  y_k = (f_k - A_k . x) / ||A_k||^2 for every row k of the group,
//            from the x at the start of the group: by default one thread per
//            row on the sliced (SELL-32) layout; for long rows a sub-warp of
//            SUB lanes per row of the group-major CSR with a shuffle reduction.
//   phase 2  x_c += sum_k A_kc y_k over the group's rows, one thread per
//            (group, column) segment of the column mirror (sliced the same
//            way): a deterministic gather, no floating-point atomics.
// Between the phases (by default) no grid barrier: each thread block owns a
// range of tiles -- consecutive permuted rows, and the columns with the same
// numbers -- and the layout keeps every (group, tile) piece of the rows and of
// the column mirror contiguous.  After RCM a tile's rows touch only columns of
// nearby tiles, so a step (one phase of one group on the block's tiles) waits
// only until the blocks owning those tiles have finished every earlier step:
// a per-block step counter published with a release store and polled with
// bounded waits.  Blocks then run ahead into later groups and sweeps as far as
// their band allows, and every x or y value is still read exactly when the
// group-after-group order of the method says (see flow_wait).  The grid
// barrier of each phase remains selectable.  For an exactly orthogonal group the
// update equals x + A_tau^+ (f_tau - A_tau x) (Eq. 1.3); with pinv_iters > 0,
// Jacobi steps on the group's Gram system make it that projection for
// near-orthogonal groups too.
//
// Residual check: ||f - A x|| / ||f|| with a fixed-order two-level reduction
// (deterministic for a given grid).  Block 0 takes the stop decision and the
// other blocks read it after a barrier.
//
// Precision form: outer FP64 loop r = f - A x, beta = ||r||; FP32 sweeps on
// A d = r / beta from d = 0 (FP32 values, x and y; row norms and groups from
// FP64); then x += beta * d in FP64.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace obk {
namespace {

// The persistent kernel runs 1024 threads per SM (64 registers each fill the
// register file), as one block of 1024 threads (the default) or two of 512;
// the layout has two tiles per SM, so a block of 1024 owns two adjacent tiles
// and a block of 512 one.
constexpr int kThreadsPerSm = 1024;
constexpr int kTilesPerSm = 2;
constexpr int kMaxWarps = 32;
constexpr int kBatch = 8;         // independent loads issued before their uses

struct SweepParams {
    int64_t N, Ngm, G;
    const int64_t* grp_rp;
    const int32_t* grp_ci;
    const double* grp_v;
    const float* grp_v32;
    const double* grp_inv;
    const float* grp_inv32;
    const int64_t* gptr;
    const int64_t* gseg_ptr;
    const int64_t* seg_ptr;
    const int32_t* seg_col;
    const int32_t* mir_row;
    const double* mir_val;
    const float* mir_val32;
    // sliced ELL (SELL-32) copies: one thread per row / per mirror segment
    int64_t ns;
    const int64_t* sl_gptr;
    const int64_t* sl_ptr;
    const int64_t* sl_row0;
    const int32_t* sl_nrow;
    const int32_t* sci;
    const double* sv;
    const float* sv32;
    const int64_t* ml_gptr;
    const int64_t* ml_ptr;
    const int32_t* mcol;
    const int32_t* mrow;
    const double* mv;
    const float* mv32;
    // Eq. 1.3 group projection by Jacobi steps (pinv_iters > 0)
    int pinv_iters;
    const int64_t* gram_ptr;
    const int32_t* gram_idx;
    const double* gram_val;
    double* y0;       // Ngm: r / ||A_i||^2 of the current group step
    double* yb;       // Ngm: second Jacobi buffer
    const double* f;  // group-major
    double* x;        // N
    double* y;        // Ngm
    double* r64;      // Ngm (precision form)
    float* b32;       // Ngm
    float* y32;       // Ngm
    float* d32;       // N
    double fnorm, zero_f2, tol, stagnation;
    int64_t maxit;
    int check_every, precision, inner_sweeps, max_outer;  // check_every < 0: adaptive schedule
    // band-local step counters instead of grid barriers (SUB == 1, no Jacobi steps)
    int dataflow;
    int64_t T;                  // tiles of the layout
    const int64_t* sl_tptr;     // G*T + 1: first row slice of each (group, tile)
    const int64_t* ml_tptr;     // G*T + 1: first mirror slice of each (group, tile)
    const int32_t* reach_lo;    // T: lowest tile a step of the tile depends on
    const int32_t* reach_hi;    // T: highest such tile
    unsigned long long* flow;   // gridDim.x step counters, zeroed before the launch
    const int64_t* gt_ptr;      // G*T + 1: first group-major row of each (group, tile)
    int64_t tile_rows;          // B
    int64_t smem_bytes;         // dynamic shared memory of the launch (staging windows)
    int staging;
    int l2_stream;  // slices larger than half the L2: evict-first loads                // 1 = stage windows in shared memory when worth it, 0 or 2 = never
    double* partial;  // gridDim.x
    double* ctrl;     // [0] rr, [1] beta, [2..11] history
    int64_t* out;     // [0] sweeps, [1] status, [2] outer, [3] stop, [4] sweep ns, [5] inner,
                      // [6] next checked sweep (adaptive schedule), [7] residual checks done
    GridBarrier gb;
};

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int SUB>
__device__ __forceinline__ unsigned sub_mask()
{
    if constexpr (SUB == 32) {
        return 0xffffffffu;
    } else {
        int lane = threadIdx.x & 31;
        return ((1u << SUB) - 1u) << (lane & ~(SUB - 1));
    }
}

template <int SUB, class T>
__device__ __forceinline__ T sub_reduce(T v)
{
    unsigned m = sub_mask<SUB>();
#pragma unroll
    for (int o = SUB / 2; o > 0; o >>= 1) v += __shfl_xor_sync(m, v, o);
    return v;
}

// ---- exact-length row and segment kernels -------------------------------------
//
// A warp-wide FP64 instruction occupies the SM's FP64 pipe for the same time
// whether 1 or 32 lanes are active, and even when every lane is predicated
// off.  Rows and column segments are therefore sorted by length inside each
// group, and the loops below run exactly as many multiply-adds as a row (or
// segment) has entries: full batches, then a warp-uniform switch on the
// remainder.  Loads are batched ahead of their uses so that a row costs a few
// memory round trips, not two per entry.

// acc - sum_{j<B} a[q+j] * xv[ci[q+j]]
template <int B, class T>
__device__ __forceinline__ T sub_batch(const int32_t* ci, const T* vals, const T* xv, int64_t q, T acc)
{
    int32_t idx[B];
    T a[B];
#pragma unroll
    for (int j = 0; j < B; ++j) {
        idx[j] = ci[q + j];
        a[j] = vals[q + j];
    }
    T xg[B];
#pragma unroll
    for (int j = 0; j < B; ++j) xg[j] = xv[idx[j]];
#pragma unroll
    for (int j = 0; j < B; ++j) acc = fma(-a[j], xg[j], acc);
    return acc;
}

// Dot product of one row with xv by a sub-warp of SUB > 1 lanes (long rows):
// lanes stride by SUB, batched loads, shuffle reduction afterwards.
template <int SUB, class T>
__device__ __forceinline__ T row_dot_wide(const int64_t* rp, const int32_t* ci, const T* vals, const T* xv,
                                          int64_t k, int sub)
{
    int64_t b = rp[k], e = rp[k + 1];
    T acc = 0;
    for (int64_t q0 = b + sub; q0 < e; q0 += (int64_t)SUB * kBatch) {
        int32_t idx[kBatch];
        T a[kBatch];
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            int64_t q = q0 + (int64_t)j * SUB;
            idx[j] = q < e ? ci[q] : -1;
            a[j] = q < e ? vals[q] : T(0);
        }
        T xg[kBatch];
#pragma unroll
        for (int j = 0; j < kBatch; ++j) xg[j] = idx[j] >= 0 ? xv[idx[j]] : T(0);
#pragma unroll
        for (int j = 0; j < kBatch; ++j) acc = fma(a[j], xg[j], acc);
    }
    return acc;
}

// rhs_k - A_k . xv with SUB lanes per row; the result is valid in lane sub == 0
template <int SUB, class T>
__device__ __forceinline__ T row_residual_sub(const SweepParams& p, const T* vals, const T* xv, int64_t k, T rhs,
                                              int sub)
{
    static_assert(SUB > 1, "one lane per row uses the sliced layout");
    T acc = row_dot_wide<SUB, T>(p.grp_rp, p.grp_ci, vals, xv, k, sub);
    acc = sub_reduce<SUB>(acc);
    return rhs - acc;
}

// phase 1: y_k = (rhs_k - A_k . xv) * inv_k for group-major rows [r0, r1)
template <int SUB, class T, class TR>
__device__ __forceinline__ void phase1(const SweepParams& p, int64_t r0, int64_t r1, const T* vals,
                                       const T* inv, const TR* rhs, const T* xv, T* y)
{
    int64_t sw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / SUB;
    int64_t nsw = ((int64_t)gridDim.x * blockDim.x) / SUB;
    int sub = threadIdx.x & (SUB - 1);
    for (int64_t k = r0 + sw; k < r1; k += nsw) {
        T r = row_residual_sub<SUB, T>(p, vals, xv, k, (T)rhs[k], sub);
        if (sub == 0) y[k] = r * inv[k];
    }
}

// ---- sliced ELL (one thread per row / per segment) ------------------------------
//
// A slice holds 32 rows of one group (similar lengths: rows are sorted by
// length inside a group) with entry j of lane l at base + 32 j + l, so every
// load instruction of a warp reads 32 consecutive values, each FP64
// instruction does 32 useful multiply-adds (up to the padding of the shorter
// rows), and the residual f_k starts the accumulator: no shuffle reduction
// and no separate subtraction.

// The slices' indices and values are read once per sweep: loaded without an
// L1 line, and, when the sliced matrix is larger than half the L2
// (SweepParams::l2_stream), with an evict-first L2 policy, so that the lines of
// x and y that the gathers reuse stay cached.  A matrix that fits in L2 keeps
// the normal policy and is read from L2 by the next sweep.  (The matrix is
// read-only inside the kernel.)
__device__ __forceinline__ uint64_t stream_policy(bool evict_first)
{
    uint64_t pol;
    if (evict_first) asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    else asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ int32_t ld_stream(const int32_t* p, uint64_t pol)
{
    int32_t v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float ld_stream(const float* p, uint64_t pol)
{
    float v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ double ld_stream(const double* p, uint64_t pol)
{
    double v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}

// acc + S * sum_{j<B} a[q + 32 j] * v[idx[q + 32 j] - off]   (S = -1 or +1; off
// is the first index held by v when v is a window staged in shared memory)
template <int B, int S, class T>
__device__ __forceinline__ T sell_batch(const int32_t* idx, const T* vals, const T* v, int64_t q, T acc,
                                        int32_t off, uint64_t pol)
{
    int32_t c[B];
    T a[B];
#pragma unroll
    for (int j = 0; j < B; ++j) {
        c[j] = ld_stream(idx + q + 32 * j, pol);
        a[j] = ld_stream(vals + q + 32 * j, pol);
    }
    T g[B];
#pragma unroll
    for (int j = 0; j < B; ++j) g[j] = v[c[j] - off];
#pragma unroll
    for (int j = 0; j < B; ++j) acc = fma(S > 0 ? a[j] : -a[j], g[j], acc);
    return acc;
}

// one lane's row (or segment) of a slice: len entries from position q
template <int S, class T>
__device__ __forceinline__ T sell_lane(const int32_t* idx, const T* vals, const T* v, int64_t q, int64_t len, T acc,
                                       int32_t off, uint64_t pol)
{
    int64_t j = 0;
    for (; j + kBatch <= len; j += kBatch, q += 32 * kBatch) acc = sell_batch<kBatch, S, T>(idx, vals, v, q, acc, off, pol);
    switch ((int)(len - j)) {  // the same for the whole warp
        case 7: acc = sell_batch<7, S, T>(idx, vals, v, q, acc, off, pol); break;
        case 6: acc = sell_batch<6, S, T>(idx, vals, v, q, acc, off, pol); break;
        case 5: acc = sell_batch<5, S, T>(idx, vals, v, q, acc, off, pol); break;
        case 4: acc = sell_batch<4, S, T>(idx, vals, v, q, acc, off, pol); break;
        case 3: acc = sell_batch<3, S, T>(idx, vals, v, q, acc, off, pol); break;
        case 2: acc = sell_batch<2, S, T>(idx, vals, v, q, acc, off, pol); break;
        case 1: acc = sell_batch<1, S, T>(idx, vals, v, q, acc, off, pol); break;
        default: break;
    }
    return acc;
}

// Slices go to warps in warp-major order over the blocks (warp w of block b is
// number w * gridDim + b): in every round of the grid stride, consecutive
// slices -- neighbours in memory and of about the same length -- land on
// different blocks, so the GPU streams one contiguous stretch of the layout at
// a time and a partial last round spreads over all SMs.
__device__ __forceinline__ int64_t sell_warp()
{
    return (int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
}

// one row slice s: y_k = (rhs_k - A_k . xv) * inv_k for its (up to) 32 rows
template <class T, class TR>
__device__ __forceinline__ void row_slice(const SweepParams& p, int64_t s, const T* sval, const T* inv,
                                          const TR* rhs, const T* xv, T* y, int32_t xoff = 0)
{
    int lane = threadIdx.x & 31;
    int64_t base = p.sl_ptr[s], len = (p.sl_ptr[s + 1] - base) >> 5;
    bool valid = lane < p.sl_nrow[s];
    int64_t k = p.sl_row0[s] + lane;
    T acc = valid ? (T)rhs[k] : T(0);
    acc = sell_lane<-1, T>(p.sci, sval, xv, base + lane, len, acc, xoff, stream_policy(p.l2_stream));
    if (valid) y[k] = acc * inv[k];
}

// one row slice s whose entries [b0, b1) and first row k0 were located ahead
template <class T, class TR>
__device__ __forceinline__ void row_slice_at(const SweepParams& p, int64_t s, int64_t b0, int64_t b1, int64_t k0,
                                             const T* sval, const T* inv, const TR* rhs, const T* xv, T* y)
{
    const int lane = threadIdx.x & 31;
    const bool valid = lane < p.sl_nrow[s];
    const int64_t k = k0 + lane;
    T acc = valid ? (T)rhs[k] : T(0);
    acc = sell_lane<-1, T>(p.sci, sval, xv, b0 + lane, (b1 - b0) >> 5, acc, 0, stream_policy(p.l2_stream));
    if (valid) y[k] = acc * inv[k];
}

// Mirror slices: lane l holds two columns, a and b (neighbouring segments),
// their entries interleaved: even positions a, odd positions b.  Each column's
// sum starts from x at the column and adds its entries in order, as for one
// segment per lane; the two sums are independent chains.
template <int B, class T>
__device__ __forceinline__ void mirror_batch(const int32_t* idx, const T* vals, const T* y, int64_t q, T& acc_a,
                                             T& acc_b, int32_t off, uint64_t pol)
{
    static_assert(B % 2 == 0, "entries come in (a, b) pairs");
    int32_t c[B];
    T a[B];
#pragma unroll
    for (int j = 0; j < B; ++j) {
        c[j] = ld_stream(idx + q + 32 * j, pol);
        a[j] = ld_stream(vals + q + 32 * j, pol);
    }
    T g[B];
#pragma unroll
    for (int j = 0; j < B; ++j) g[j] = y[c[j] - off];
#pragma unroll
    for (int j = 0; j < B; j += 2) {
        acc_a = fma(a[j], g[j], acc_a);
        acc_b = fma(a[j + 1], g[j + 1], acc_b);
    }
}

template <class T>
__device__ __forceinline__ void mirror_lane(const int32_t* idx, const T* vals, const T* y, int64_t q, int64_t len,
                                            T& acc_a, T& acc_b, int32_t off, uint64_t pol)
{
    int64_t j = 0;
    for (; j + kBatch <= len; j += kBatch, q += 32 * kBatch)
        mirror_batch<kBatch, T>(idx, vals, y, q, acc_a, acc_b, off, pol);
    switch ((int)(len - j)) {  // even, the same for the whole warp
        case 6: mirror_batch<6, T>(idx, vals, y, q, acc_a, acc_b, off, pol); break;
        case 4: mirror_batch<4, T>(idx, vals, y, q, acc_a, acc_b, off, pol); break;
        case 2: mirror_batch<2, T>(idx, vals, y, q, acc_a, acc_b, off, pol); break;
        default: break;
    }
}

// one mirror slice whose lane columns ca, cb (cb = kOneColumn: one column
// per lane) and entries [b0, b1) are known: xv_c += sum_k A_kc y_k for its
// (up to) 32 or 64 columns
template <class T>
__device__ __forceinline__ void col_slice_at(const SweepParams& p, int32_t ca, int32_t cb, int64_t b0, int64_t b1,
                                             const T* mval, const T* y, T* xv, int32_t yoff = 0)
{
    const int lane = threadIdx.x & 31;
    const uint64_t pol = stream_policy(p.l2_stream);
    T acc_a = ca >= 0 ? xv[ca] : T(0);
    if (cb != kOneColumn) {  // the same for the whole warp
        T acc_b = cb >= 0 ? xv[cb] : T(0);
        mirror_lane<T>(p.mrow, mval, y, b0 + lane, (b1 - b0) >> 5, acc_a, acc_b, yoff, pol);
        if (cb >= 0) xv[cb] = acc_b;
    } else {
        acc_a = sell_lane<1, T>(p.mrow, mval, y, b0 + lane, (b1 - b0) >> 5, acc_a, yoff, pol);
    }
    if (ca >= 0) xv[ca] = acc_a;
}

// one mirror slice s
template <class T>
__device__ __forceinline__ void col_slice(const SweepParams& p, int64_t s, const T* mval, const T* y, T* xv,
                                          int32_t yoff = 0)
{
    const int lane = threadIdx.x & 31;
    col_slice_at<T>(p, p.mcol[s * 64 + lane], p.mcol[s * 64 + 32 + lane], p.ml_ptr[s], p.ml_ptr[s + 1], mval, y, xv,
                    yoff);
}

// phase 1 over all row slices of group g (whole grid)
template <class T, class TR>
__device__ __forceinline__ void phase1_sell(const SweepParams& p, int64_t g, const T* sval, const T* inv,
                                            const TR* rhs, const T* xv, T* y)
{
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t s1 = p.sl_gptr[g + 1];
    for (int64_t s = p.sl_gptr[g] + sell_warp(); s < s1; s += nw) row_slice<T, TR>(p, s, sval, inv, rhs, xv, y);
}

// phase 2 over all mirror slices of group g (whole grid)
template <class T>
__device__ __forceinline__ void phase2_sell(const SweepParams& p, int64_t g, const T* mval, const T* y, T* xv)
{
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t s1 = p.ml_gptr[g + 1];
    for (int64_t s = p.ml_gptr[g] + sell_warp(); s < s1; s += nw) col_slice<T>(p, s, mval, y, xv);
}

// xv_c + sum_{j<B} a[q+j] * y[row[q+j]]
template <int B, class T>
__device__ __forceinline__ T add_batch(const int32_t* mrow, const T* mval, const T* y, int64_t q, T acc)
{
    int32_t r[B];
    T a[B];
#pragma unroll
    for (int j = 0; j < B; ++j) {
        r[j] = mrow[q + j];
        a[j] = mval[q + j];
    }
    T yg[B];
#pragma unroll
    for (int j = 0; j < B; ++j) yg[j] = y[r[j]];
#pragma unroll
    for (int j = 0; j < B; ++j) acc = fma(a[j], yg[j], acc);
    return acc;
}

// phase 2: xv_c += sum over the segment's rows (ascending) of A_kc y_k, one
// thread per (group, column) segment, segments [s0, s1)
template <class T>
__device__ __forceinline__ void phase2(const SweepParams& p, int64_t s0, int64_t s1, const T* mval,
                                       const T* y, T* xv)
{
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t nth = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = s0 + tid; t < s1; t += nth) {
        int64_t q = p.seg_ptr[t], e = p.seg_ptr[t + 1];
        int32_t c = p.seg_col[t];
        T acc = xv[c];
        for (; q + 4 <= e; q += 4) acc = add_batch<4, T>(p.mir_row, mval, y, q, acc);
        switch ((int)(e - q)) {
            case 3: acc = add_batch<3, T>(p.mir_row, mval, y, q, acc); break;
            case 2: acc = add_batch<2, T>(p.mir_row, mval, y, q, acc); break;
            case 1: acc = add_batch<1, T>(p.mir_row, mval, y, q, acc); break;
            default: break;
        }
        xv[c] = acc;
    }
}

// deterministic block sum (fixed shuffle tree, warps in order); result in thread 0
__device__ double block_sum(double v)
{
    __shared__ double ws[kMaxWarps];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) ws[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += ws[k];
    __syncthreads();
    return s;
}

// sum of squared residuals (FP64) of all group-major rows into partial[block];
// with store_r the residuals are kept in r64
template <int SUB>
__device__ void residual_partial(const SweepParams& p, bool store_r)
{
    if constexpr (SUB == 1) {
        int lane = threadIdx.x & 31;
        int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
        double local = 0.0;
        for (int64_t s = sell_warp(); s < p.ns; s += nw) {
            int64_t base = p.sl_ptr[s], len = (p.sl_ptr[s + 1] - base) >> 5;
            bool valid = lane < p.sl_nrow[s];
            int64_t k = p.sl_row0[s] + lane;
            double acc = valid ? p.f[k] : 0.0;
            acc = sell_lane<-1, double>(p.sci, p.sv, p.x, base + lane, len, acc, 0, stream_policy(p.l2_stream));
            if (valid) {
                if (store_r) p.r64[k] = acc;
                local = fma(acc, acc, local);
            }
        }
        double sum = block_sum(local);
        if (threadIdx.x == 0) p.partial[blockIdx.x] = sum;
    } else {
        int64_t sw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / SUB;
        int64_t nsw = ((int64_t)gridDim.x * blockDim.x) / SUB;
        int sub = threadIdx.x & (SUB - 1);
        double local = 0.0;
        for (int64_t k = sw; k < p.Ngm; k += nsw) {
            double r = row_residual_sub<SUB, double>(p, p.grp_v, p.x, k, p.f[k], sub);
            if (sub == 0) {
                if (store_r) p.r64[k] = r;
                local = fma(r, r, local);
            }
        }
        double s = block_sum(local);
        if (threadIdx.x == 0) p.partial[blockIdx.x] = s;
    }
}

// Total of the per-block partial sums, computed by block 0 with a fixed
// reduction tree (thread t sums partials t, t + blockDim, ... in order, then
// the block sum), so the result is the same on every run for a given grid.
// Called by every thread of block 0; the total is returned to thread 0.
__device__ double total_partials(const SweepParams& p)
{
    double s = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) s += p.partial[b];
    s = block_sum(s);
    return s + p.zero_f2;
}

// Adaptive residual-check schedule: from the last two checks (sweeps s_prev < s,
// residuals rr_prev > rr) the linear rate predicts k more sweeps to reach tol;
// the next check comes after min(k, s) sweeps (the gap at most doubles), or
// after one sweep when no rate is available.  The CPU reference applies the
// same rule.
__device__ __forceinline__ int64_t next_check(int64_t s, double rr, int64_t s_prev, double rr_prev, double tol)
{
    int64_t step = 1;
    if (s_prev > 0 && rr < rr_prev && rr > tol && rr > 0.0) {
        double rate = pow(rr / rr_prev, 1.0 / (double)(s - s_prev));
        if (rate > 0.0 && rate < 1.0) {
            double k = ceil(log(tol / rr) / log(rate));
            if (k > (double)s) k = (double)s;
            if (k > 1.0) step = (int64_t)k;
        }
    } else if (s_prev == 0) {
        step = 1;
    }
    return s + step;
}

// One Jacobi step of the group's Gram system (A_tau A_tau^T) y = r_tau for the
// rows of group g: dst_k = y0_k - (1/||A_k||^2) sum_u (A_k . A_u) src_u over
// the row's partners in the group (ascending), with y0 = r / ||A_k||^2 the
// phase-1 value, saved from src at the first step.
__device__ __forceinline__ void jacobi_step(const SweepParams& p, int64_t g, const double* src, double* dst,
                                            bool first)
{
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t nth = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = p.gptr[g] + tid; k < p.gptr[g + 1]; k += nth) {
        double y0 = src[k];
        if (first) p.y0[k] = y0;
        else y0 = p.y0[k];
        double acc = 0.0;
        for (int64_t a = p.gram_ptr[k]; a < p.gram_ptr[k + 1]; ++a) acc = fma(p.gram_val[a], src[p.gram_idx[a]], acc);
        dst[k] = fma(-p.grp_inv[k], acc, y0);
    }
}

// one group step's two phases: sliced layout for SUB == 1, sub-warps per CSR row otherwise
template <int SUB, class T, class TR>
__device__ __forceinline__ void group_phase1(const SweepParams& p, int64_t g, const T* vals, const T* svals,
                                             const T* inv, const TR* rhs, const T* xv, T* y)
{
    if constexpr (SUB == 1) phase1_sell<T, TR>(p, g, svals, inv, rhs, xv, y);
    else phase1<SUB, T, TR>(p, p.gptr[g], p.gptr[g + 1], vals, inv, rhs, xv, y);
}
template <int SUB, class T>
__device__ __forceinline__ void group_phase2(const SweepParams& p, int64_t g, const T* mvals, const T* smvals,
                                             const T* y, T* xv)
{
    if constexpr (SUB == 1) phase2_sell<T>(p, g, smvals, y, xv);
    else phase2<T>(p, p.gseg_ptr[g], p.gseg_ptr[g + 1], mvals, y, xv);
}

// ---- band-local step counters (dataflow between the phases) --------------------
//
// Steps are numbered over the whole launch: step 2 (s G + g) is phase 1 of
// group g in the s-th sweep since the launch, step 2 (s G + g) + 1 its phase 2
// (the same numbering on every block).  flow[b] = j means block b has finished
// all its steps before j.  Before a step j with work, a block publishes what
// it has finished and waits until flow[b'] >= j for every block b' owning a
// tile in the reach of its own tiles.  That order is exactly the one the grid
// barriers give, for every value the step touches:
//  * phase 1 of group g on tile t reads x_c for the columns c of its rows; the
//    tiles of those columns are in the reach of t, and their owners have
//    finished every earlier step, so every earlier update of x_c is visible,
//    and no later one has started: an update of x_c at a later step waits for
//    the tiles of the rows of column c, t among them;
//  * phase 2 of group g on tile t reads y_k for the rows k of group g that
//    touch its columns, written by phase 1 of g on their tiles (in the reach of
//    t), and overwrites x_c only after every earlier phase 1 reading x_c ended
//    (same tiles);
//  * phase 1 of the next sweep overwrites y_k only after every phase 2 reading
//    it ended: the tiles of the columns of row k are in the reach of k's tile.
// A block with nothing to do in a step skips it without waiting; its counter
// moves on at its next wait.  The block with the fewest finished steps always
// finds its waits satisfied, so the launch cannot deadlock; every wait is still
// bounded (as in grid_sync) and checks the error word, so a block that gave up
// makes the others give up too.
struct FlowState {
    int64_t t0, t1;          // tiles [t0, t1) owned by this block
    int64_t tlo, thi;        // tiles its steps depend on
    int blo, bhi;            // blocks this block's steps wait for
    unsigned long long step; // next step
    unsigned long long pub;  // last value published in flow[blockIdx.x]
    int ok;
};

__device__ __forceinline__ int block_of_tile(int64_t t, int64_t T)
{
    return (int)(((t + 1) * (int64_t)gridDim.x - 1) / T);
}

__device__ void flow_init(const SweepParams& p, FlowState& f)
{
    if (threadIdx.x == 0) {
        f.t0 = (int64_t)blockIdx.x * p.T / gridDim.x;
        f.t1 = ((int64_t)blockIdx.x + 1) * p.T / gridDim.x;
        int64_t lo = f.t0, hi = f.t1 - 1;
        for (int64_t t = f.t0; t < f.t1; ++t) {
            lo = min(lo, (int64_t)p.reach_lo[t]);
            hi = max(hi, (int64_t)p.reach_hi[t]);
        }
        f.tlo = lo;
        f.thi = hi;
        f.blo = block_of_tile(lo, p.T);
        f.bhi = block_of_tile(hi, p.T);
        f.step = 0;
        f.pub = 0;
        f.ok = 1;
    }
    __syncthreads();
}

// Publish the finished steps, then wait until every block in the reach has
// finished the steps before f.step.  Called by all threads; false on timeout.
__device__ bool flow_wait(const SweepParams& p, FlowState& f)
{
    __syncthreads();  // the block's earlier writes are complete
    if (threadIdx.x < 32) {
        const unsigned full = 0xffffffffu;
        int lane = threadIdx.x;
        unsigned long long j = f.step;
        if (lane == 0 && f.pub < j) {
            __threadfence();
            st_release_gpu_u64(p.flow + blockIdx.x, j);
        }
        long long spins = 0;
        int ok = 1;
        for (;;) {
            bool mine = true;
            for (int b = f.blo + lane; b <= f.bhi; b += 32) mine = mine && ld_volatile_u64(p.flow + b) >= j;
            if (__all_sync(full, mine)) break;
            ++spins;
            bool bad = spins > p.gb.limit;
            if ((spins & 63) == 0) bad = bad || __any_sync(full, ld_volatile_i32(p.gb.err) != 0);
            if (bad) {
                if (lane == 0) atomicCAS(p.gb.err, 0, (int)kDevTimeout);
                ok = 0;
                break;
            }
            if (spins > 16) __nanosleep(32);
        }
        // acquire the values seen (the same load the grid barrier uses), so the
        // neighbours' writes before their release are visible to this block
        for (int b = f.blo + lane; b <= f.bhi; b += 32) (void)ld_acquire_gpu_u64(p.flow + b);
        __threadfence();
        if (lane == 0) {
            f.pub = j > f.pub ? j : f.pub;
            f.ok = ok;
        }
    }
    __syncthreads();
    return f.ok != 0;
}

// The block finished step f.step (with work): publish it and move on.
__device__ __forceinline__ void flow_done(const SweepParams& p, FlowState& f)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        st_release_gpu_u64(p.flow + blockIdx.x, f.step + 1);
        f.pub = f.step + 1;
        f.step = f.step + 1;
    }
    __syncthreads();
}

// Publish every step finished so far (skipped ones included), so that no
// other block waits on this one while it is elsewhere (a grid barrier).
__device__ __forceinline__ void flow_flush(const SweepParams& p, FlowState& f)
{
    __syncthreads();
    if (threadIdx.x == 0 && f.pub < f.step) {
        __threadfence();
        st_release_gpu_u64(p.flow + blockIdx.x, f.step);
        f.pub = f.step;
    }
    __syncthreads();
}

__device__ __forceinline__ void flow_skip(FlowState& f)
{
    __syncthreads();
    if (threadIdx.x == 0) f.step = f.step + 1;
    __syncthreads();
}

__device__ __forceinline__ void cp_async_16(void* dst_smem, const void* src)
{
    unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" : : "r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" : : : "memory"); }

// Copy src[a0, w1) into the block's shared-memory window (all threads), where
// a0 = w0 rounded down to a 16-byte boundary of src, and return a0: the window
// holds src[i] at win[i - a0].  Whole 16-byte chunks go by asynchronous copies
// (all in flight at once), the ragged end element by element.  src must be
// 16-byte aligned; the window needs w1 - a0 elements.
template <class T>
__device__ __forceinline__ int64_t stage(T* win, const T* src, int64_t w0, int64_t w1)
{
    constexpr int64_t E = 16 / sizeof(T);  // elements per chunk
    int64_t a0 = w0 & ~(E - 1);
    int64_t a1 = w1 & ~(E - 1);            // chunks [a0, a1), elements [a1, w1)
    for (int64_t i = a0 + (int64_t)threadIdx.x * E; i < a1; i += (int64_t)blockDim.x * E)
        cp_async_16(win + (i - a0), src + i);
    for (int64_t i = max(a1, a0) + threadIdx.x; i < w1; i += blockDim.x) win[i - a0] = src[i];
    cp_async_wait_all();
    __syncthreads();
    return a0;
}

// A step stages its window in shared memory when the window fits and holds
// no more values than the step gathers (a copy of a value is a coalesced
// load, a gather a random one); otherwise it gathers from global memory.
__device__ __forceinline__ bool worth_staging(int64_t window, int64_t gathers, int64_t cap)
{
    return window <= cap && window <= gathers;
}

// One sweep (all groups) on the block's tiles with band-local waits; false on timeout.
//  phase 1 of group g reads x at the columns of the block's rows: the columns
//    of tiles [tlo, thi], staged as x[tlo * B, (thi + 1) * B);
//  phase 2 reads y at the group-major rows of group g in tiles [tlo, thi] (the
//    rows touching the block's columns), contiguous in the layout.
template <class T, class TR>
__device__ bool flow_sweep(const SweepParams& p, FlowState& f, const T* sval, const T* mval, const T* inv,
                           const TR* rhs, T* xv, T* y)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    T* win = reinterpret_cast<T*>(dsm);
    const int64_t cap = p.smem_bytes / (int64_t)sizeof(T);
    const int nw = blockDim.x >> 5;
    const int w = threadIdx.x >> 5;
    const int64_t x0 = f.tlo * p.tile_rows;
    const int64_t x1 = min((f.thi + 1) * p.tile_rows, p.N);
    for (int64_t g = 0; g < p.G; ++g) {
        int64_t s0 = p.sl_tptr[g * p.T + f.t0], s1 = p.sl_tptr[g * p.T + f.t1];
        if (s0 < s1) {
            if (!flow_wait(p, f)) return false;
            if (p.staging == 1 && worth_staging(x1 - x0 + 4, p.sl_ptr[s1] - p.sl_ptr[s0], cap)) {
                int64_t a0 = stage<T>(win, xv, x0, x1);
                for (int64_t s = s0 + w; s < s1; s += nw) row_slice<T, TR>(p, s, sval, inv, rhs, win, y, (int32_t)a0);
            } else {
                // each slice's bounds and first row are loaded one slice ahead
                int64_t s = s0 + w, nb0 = 0, nb1 = 0, nk0 = 0;
                if (s < s1) {
                    nb0 = p.sl_ptr[s];
                    nb1 = p.sl_ptr[s + 1];
                    nk0 = p.sl_row0[s];
                }
                for (; s < s1; s += nw) {
                    const int64_t b0 = nb0, b1 = nb1, k0 = nk0;
                    if (s + nw < s1) {
                        nb0 = p.sl_ptr[s + nw];
                        nb1 = p.sl_ptr[s + nw + 1];
                        nk0 = p.sl_row0[s + nw];
                    }
                    row_slice_at<T, TR>(p, s, b0, b1, k0, sval, inv, rhs, xv, y);
                }
            }
            flow_done(p, f);
        } else {
            flow_skip(f);
        }
        int64_t m0 = p.ml_tptr[g * p.T + f.t0], m1 = p.ml_tptr[g * p.T + f.t1];
        if (m0 < m1) {
            if (!flow_wait(p, f)) return false;
            int64_t y0 = p.gt_ptr[g * p.T + f.tlo], y1 = p.gt_ptr[g * p.T + f.thi + 1];
            if (p.staging == 1 && worth_staging(y1 - y0 + 4, p.ml_ptr[m1] - p.ml_ptr[m0], cap)) {
                int64_t a0 = stage<T>(win, y, y0, y1);
                for (int64_t s = m0 + w; s < m1; s += nw) col_slice<T>(p, s, mval, win, xv, (int32_t)a0);
            } else {
                // A mirror slice is a chain of three loads (its bounds and
                // columns, then its entries and x at the columns, then the
                // gathers of y) for a few entries per lane: the next slice's
                // bounds and columns are loaded while this one runs.
                const int lane = threadIdx.x & 31;
                int64_t s = m0 + w, nb0 = 0, nb1 = 0;
                int32_t nca = -1, ncb = -1;
                if (s < m1) {
                    nb0 = p.ml_ptr[s];
                    nb1 = p.ml_ptr[s + 1];
                    nca = p.mcol[s * 64 + lane];
                    ncb = p.mcol[s * 64 + 32 + lane];
                }
                for (; s < m1; s += nw) {
                    const int64_t b0 = nb0, b1 = nb1;
                    const int32_t ca = nca, cb = ncb;
                    if (s + nw < m1) {
                        nb0 = p.ml_ptr[s + nw];
                        nb1 = p.ml_ptr[s + nw + 1];
                        nca = p.mcol[(s + nw) * 64 + lane];
                        ncb = p.mcol[(s + nw) * 64 + 32 + lane];
                    }
                    col_slice_at<T>(p, ca, cb, b0, b1, mval, y, xv);
                }
            }
            flow_done(p, f);
        } else {
            flow_skip(f);
        }
    }
    flow_flush(p, f);
    return true;
}

template <int SUB, int BLOCK>
__global__ void __launch_bounds__(BLOCK, kThreadsPerSm / BLOCK) obk_solve_kernel(SweepParams p)
{
    __shared__ FlowState flow;
    const bool df = SUB == 1 && p.dataflow != 0 && p.pinv_iters == 0;
    if (df) flow_init(p, flow);
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    volatile int64_t* vout = p.out;
    // initial residual
    residual_partial<SUB>(p, p.precision == 1);
    if (!grid_sync(p.gb)) return;
    double tot0 = blockIdx.x == 0 ? total_partials(p) : 0.0;
    if (lead) {
        double tot = tot0;
        double rr = p.fnorm > 0.0 ? sqrt(tot) / p.fnorm : sqrt(tot);
        p.ctrl[0] = rr;
        p.ctrl[1] = sqrt(tot);
        vout[0] = 0;
        vout[2] = 0;
        vout[4] = 0;
        if (rr <= p.tol) { vout[1] = 0; vout[3] = 1; }
        else { vout[1] = 1; vout[3] = 0; }
    }
    if (!grid_sync(p.gb)) return;

    if (p.precision == 0) {
        int64_t s = 0;
        int64_t nchk = 0;
        // adaptive schedule state (lead thread only): last checked sweep and its residual
        int64_t s_prev = 0;
        double rr_prev = p.ctrl[0];
        if (lead) vout[6] = 1;
        if (!grid_sync(p.gb)) return;
        while (vout[3] == 0) {
            unsigned long long t0 = lead ? globaltimer() : 0;
            if (df) {
                if (!flow_sweep<double, double>(p, flow, p.sv, p.mv, p.grp_inv, p.f, p.x, p.y)) return;
            } else for (int64_t g = 0; g < p.G; ++g) {
                group_phase1<SUB, double, double>(p, g, p.grp_v, p.sv, p.grp_inv, p.f, p.x, p.y);
                const double* yg = p.y;
                if (p.pinv_iters > 0) {  // y <- solution of the group's Gram system
                    double* src = p.y;
                    double* dst = p.yb;
                    for (int k = 0; k < p.pinv_iters; ++k) {
                        if (!grid_sync(p.gb)) return;
                        jacobi_step(p, g, src, dst, k == 0);
                        double* t_ = src;
                        src = dst;
                        dst = t_;
                    }
                    yg = src;
                }
                if (!grid_sync(p.gb)) return;
                group_phase2<SUB, double>(p, g, p.mir_val, p.mv, yg, p.x);
                if (!grid_sync(p.gb)) return;
            }
            ++s;
            if (lead) { vout[4] += (int64_t)(globaltimer() - t0); vout[0] = s; }
            bool check = p.check_every > 0 ? ((s % p.check_every) == 0 || s >= p.maxit)
                                           : (s >= vout[6] || s >= p.maxit);
            if (check) {
                // with band-local waits the blocks may be at different steps:
                // the residual needs every block's sweeps finished
                if (df && !grid_sync(p.gb)) return;
                residual_partial<SUB>(p, false);
                if (!grid_sync(p.gb)) return;
                double totc = blockIdx.x == 0 ? total_partials(p) : 0.0;
                if (lead) {
                    double tot = totc;
                    double rr = p.fnorm > 0.0 ? sqrt(tot) / p.fnorm : sqrt(tot);
                    p.ctrl[0] = rr;
                    vout[7] += 1;
                    int stop = 0;
                    if (rr <= p.tol) { vout[1] = 0; stop = 1; }
                    else if (s >= p.maxit) stop = 1;
                    else if (p.stagnation > 0.0) {
                        double* hist = p.ctrl + 2;
                        if (nchk >= 10 && fabs(rr - hist[nchk % 10]) < p.stagnation) stop = 1;
                        hist[nchk % 10] = rr;
                    }
                    ++nchk;
                    vout[3] = stop;
                    vout[6] = next_check(s, rr, s_prev, rr_prev, p.tol);
                    s_prev = s;
                    rr_prev = rr;
                }
                if (!grid_sync(p.gb)) return;
            }
        }
        return;
    }

    // precision form: FP32 inner sweeps inside FP64 refinement
    int64_t sweeps = 0;
    int64_t outer = 0;
    int s_in = p.inner_sweeps > 0 ? p.inner_sweeps : 8;
    double rr_prev = p.ctrl[0];
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t nth = (int64_t)gridDim.x * blockDim.x;
    while (vout[3] == 0) {
        double beta = *(volatile double*)(p.ctrl + 1);
        for (int64_t k = tid; k < p.Ngm; k += nth) p.b32[k] = (float)(p.r64[k] / beta);
        for (int64_t c = tid; c < p.N; c += nth) p.d32[c] = 0.0f;
        if (!grid_sync(p.gb)) return;
        unsigned long long t0 = lead ? globaltimer() : 0;
        int nin = s_in;
        if (sweeps + nin > p.maxit) nin = (int)(p.maxit - sweeps);
        for (int it = 0; it < nin; ++it) {
            if (df) {
                if (!flow_sweep<float, float>(p, flow, p.sv32, p.mv32, p.grp_inv32, p.b32, p.d32, p.y32)) return;
                continue;
            }
            for (int64_t g = 0; g < p.G; ++g) {
                group_phase1<SUB, float, float>(p, g, p.grp_v32, p.sv32, p.grp_inv32, p.b32, p.d32, p.y32);
                if (!grid_sync(p.gb)) return;
                group_phase2<SUB, float>(p, g, p.mir_val32, p.mv32, p.y32, p.d32);
                if (!grid_sync(p.gb)) return;
            }
        }
        if (df && !grid_sync(p.gb)) return;  // every block's inner sweeps are done
        sweeps += nin;
        if (lead) { vout[4] += (int64_t)(globaltimer() - t0); vout[0] = sweeps; }
        for (int64_t c = tid; c < p.N; c += nth) p.x[c] = fma(beta, (double)p.d32[c], p.x[c]);
        ++outer;
        if (!grid_sync(p.gb)) return;
        residual_partial<SUB>(p, true);
        if (!grid_sync(p.gb)) return;
        double totr = blockIdx.x == 0 ? total_partials(p) : 0.0;
        if (lead) {
            double tot = totr;
            double rr = p.fnorm > 0.0 ? sqrt(tot) / p.fnorm : sqrt(tot);
            p.ctrl[0] = rr;
            p.ctrl[1] = sqrt(tot);
            vout[2] = outer;
            int stop = 0;
            if (rr <= p.tol) { vout[1] = 0; stop = 1; }
            else if (sweeps >= p.maxit || outer >= p.max_outer) stop = 1;
            vout[3] = stop;
            // inner sweep count for the next step: aim for the reduction that
            // FP32 can deliver (about 1e-6) or what tol still needs
            if (p.inner_sweeps <= 0 && rr > 0.0 && rr_prev > 0.0 && rr < rr_prev) {
                double rate = pow(rr / rr_prev, 1.0 / (double)nin);
                double target = fmax(1e-6, 0.5 * p.tol / rr);
                if (rate < 1.0 && rate > 0.0) {
                    double want = ceil(log(target) / log(rate));
                    int w = (int)fmin(fmax(want, 2.0), 64.0);
                    vout[5] = w;
                } else {
                    vout[5] = 64;
                }
            } else {
                vout[5] = s_in;
            }
            rr_prev = rr;
        }
        if (!grid_sync(p.gb)) return;
        s_in = (int)vout[5];
        if (p.inner_sweeps > 0) s_in = p.inner_sweeps;
    }
}

// ---- launch ---------------------------------------------------------------------

template <int SUB, int BLOCK>
void launch_solve(SweepParams& p, int64_t want_smem, cudaStream_t st)
{
    DevInfo di = dev_info();
    const void* k = (const void*)obk_solve_kernel<SUB, BLOCK>;
    // dynamic shared memory for the staged windows of the band-local sweep:
    // what the largest window needs, within the opt-in limit
    cudaFuncAttributes fa;
    OBK_CUDA(cudaFuncGetAttributes(&fa, k));
    int64_t room = (int64_t)di.smem_optin - (int64_t)fa.sharedSizeBytes;
    room &= ~(int64_t)15;
    int64_t smem = SUB == 1 && p.dataflow && p.staging == 1 ? std::max<int64_t>(0, std::min<int64_t>(want_smem, room))
                                                             : 0;
    smem &= ~(int64_t)15;
    // the attribute is the same on every call (threads of the request loop may
    // launch concurrently with different sizes, all within it)
    OBK_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)room));
    p.smem_bytes = smem;
    // blocks for the tiles of the layout (one tile per 2K rows, two per SM):
    // small systems take a few SMs and leave the others to concurrent
    // requests; a block of 1024 threads takes two tiles, and a smaller
    // co-resident grid gives each block more
    constexpr int64_t kTilesPerBlock = BLOCK / (kThreadsPerSm / kTilesPerSm);
    int64_t want = std::max<int64_t>(1, ceil_div(std::max<int64_t>(p.T, 1), kTilesPerBlock));
    int grid = coop_grid(k, BLOCK, (size_t)smem, want);
    DBuf<double> partial(grid, st);
    DBuf<unsigned long long> flow(grid, st);
    OBK_CUDA(cudaMemsetAsync(flow.p, 0, flow.bytes(), st));
    p.partial = partial.p;
    p.flow = flow.p;
    void* args[] = {&p};
    ::obk::count_launch();
    OBK_CUDA(cudaLaunchCooperativeKernel(k, grid, BLOCK, args, (size_t)smem, st));
    OBK_CUDA(cudaStreamSynchronize(st));
}

}  // namespace

int default_sync_mode(const SweepLayout& L)
{
    DevInfo di = dev_info();
    return L.T >= (int64_t)di.sms * kTilesPerSm && L.G <= 16 ? 2 : 1;
}

int64_t sweep_tiles(int64_t N)
{
    DevInfo di = dev_info();
    return std::max<int64_t>(1, std::min<int64_t>((int64_t)di.sms * kTilesPerSm, ceil_div(N, 2048)));
}

// Lanes per row in phase 1.  FP64 issue is scarce on this GPU (a warp-wide
// FP64 instruction occupies the FP64 pipe for the same time whatever the
// number of active lanes).  One lane per row on the sliced layout wastes none
// of it (no shuffle reduction, no separate subtraction, coalesced loads) and
// measured fastest for rows of up to a few dozen entries; long rows get a
// sub-warp each so that a row's loads are spread over lanes.
int choose_sub(double avg_row)
{
    // (a measured choice from obk_autotune takes precedence, see capi.cu)
    if (avg_row <= 64) return 1;
    if (avg_row <= 160) return 8;
    return 32;
}

SolveResult run_solve(const SweepLayout& L, const double* f_gm, double fnorm2, double zero_f2,
                      double* x, const SolveArgs& a, int* d_err, cudaStream_t st)
{
    SolveResult res;
    DBuf<double> y(std::max<int64_t>(L.Ngm, 1), st), ctrl(16, st);
    DBuf<int64_t> out(8, st);
    DBuf<unsigned> bar(kBarrierWords, st);
    DBuf<double> r64;
    DBuf<float> b32, y32, d32;
    if (a.precision == 1) {
        r64.alloc(std::max<int64_t>(L.Ngm, 1), st);
        b32.alloc(std::max<int64_t>(L.Ngm, 1), st);
        y32.alloc(std::max<int64_t>(L.Ngm, 1), st);
        d32.alloc(std::max<int64_t>(L.N, 1), st);
        if (!L.sv32.p && L.nnz_gm > 0) throw Error{-1, "precision form needs the FP32 layout"};
    }
    OBK_CUDA(cudaMemsetAsync(ctrl.p, 0, 16 * sizeof(double), st));
    OBK_CUDA(cudaMemsetAsync(out.p, 0, 8 * sizeof(int64_t), st));
    OBK_CUDA(cudaMemsetAsync(bar.p, 0, kBarrierWords * sizeof(unsigned), st));
    OBK_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), st));
    DBuf<double> y0, yb;
    if (a.precision == 0 && a.pinv_iters > 0) {
        if (!L.has_gram) throw Error{-5, "internal error: Gram entries not built"};
        y0.alloc(std::max<int64_t>(L.Ngm, 1), st);
        yb.alloc(std::max<int64_t>(L.Ngm, 1), st);
    }
    SweepParams p{};
    p.N = L.N;
    p.Ngm = L.Ngm;
    p.G = L.G;
    p.grp_rp = L.grp_rp.p;
    p.grp_ci = L.grp_ci.p;
    p.grp_v = L.grp_v.p;
    p.grp_v32 = L.grp_v32.p;
    p.grp_inv = L.grp_inv.p;
    p.grp_inv32 = L.grp_inv32.p;
    p.gptr = L.gptr.p;
    p.gseg_ptr = L.gseg_ptr.p;
    p.seg_ptr = L.seg_ptr.p;
    p.seg_col = L.seg_col.p;
    p.mir_row = L.mir_row.p;
    p.mir_val = L.mir_val.p;
    p.mir_val32 = L.mir_val32.p;
    p.ns = L.ns;
    p.sl_gptr = L.sl_gptr.p;
    p.sl_ptr = L.sl_ptr.p;
    p.sl_row0 = L.sl_row0.p;
    p.sl_nrow = L.sl_nrow.p;
    p.sci = L.sci.p;
    p.sv = L.sv.p;
    p.sv32 = L.sv32.p;
    p.ml_gptr = L.ml_gptr.p;
    p.ml_ptr = L.ml_ptr.p;
    p.mcol = L.mcol.p;
    p.mrow = L.mrow.p;
    p.mv = L.mv.p;
    p.mv32 = L.mv32.p;
    p.pinv_iters = a.precision == 0 ? a.pinv_iters : 0;
    p.gram_ptr = L.gram_ptr.p;
    p.gram_idx = L.gram_idx.p;
    p.gram_val = L.gram_val.p;
    p.y0 = y0.p;
    p.yb = yb.p;
    p.f = f_gm;
    p.x = x;
    p.y = y.p;
    p.r64 = r64.p;
    p.b32 = b32.p;
    p.y32 = y32.p;
    p.d32 = d32.p;
    p.fnorm = sqrt(fnorm2);
    p.zero_f2 = zero_f2;
    p.tol = a.tol;
    p.stagnation = a.stagnation;
    p.maxit = a.maxit;
    p.check_every = a.check_every;
    p.precision = a.precision;
    p.inner_sweeps = a.inner_sweeps;
    p.max_outer = a.max_outer > 0 ? a.max_outer : 100;
    p.dataflow = a.sync_mode == 2 ? 1 : 0;
    p.T = L.T;
    p.sl_tptr = L.sl_tptr.p;
    p.ml_tptr = L.ml_tptr.p;
    p.reach_lo = L.reach_lo.p;
    p.reach_hi = L.reach_hi.p;
    p.gt_ptr = L.gt_ptr.p;
    p.tile_rows = L.B;
    p.staging = a.staging;
    {
        const double sliced = (double)(L.sell_nnz + L.msell_nnz) * (4.0 + (a.precision == 1 ? 4.0 : 8.0));
        p.l2_stream = sliced > 0.5 * (double)dev_info().l2_bytes ? 1 : 0;
    }
    p.ctrl = ctrl.p;
    p.out = out.p;
    p.gb = GridBarrier{bar.p, d_err, a.spin_limit};
    int sub = a.sub;
    if (sub == 0) sub = choose_sub(L.Ngm ? (double)L.nnz_gm / (double)L.Ngm : 1.0);
    if (sub > 1 && L.nnz_gm > 0 && (!L.has_gm_csr || (a.precision == 1 && !L.grp_v32.p)))
        throw Error{-5, "internal error: group-major rows not built"};
    int64_t elt = a.precision == 1 ? (int64_t)sizeof(float) : (int64_t)sizeof(double);
    int64_t want_smem = (std::max(L.ywin_max, L.xwin_max) + 4) * elt;  // + the 16-byte rounding of a window
    bool big = a.block != 512;
    switch (sub) {
        case 1: big ? launch_solve<1, 1024>(p, want_smem, st) : launch_solve<1, 512>(p, want_smem, st); break;
        case 2: big ? launch_solve<2, 1024>(p, want_smem, st) : launch_solve<2, 512>(p, want_smem, st); break;
        case 4: big ? launch_solve<4, 1024>(p, want_smem, st) : launch_solve<4, 512>(p, want_smem, st); break;
        case 8: big ? launch_solve<8, 1024>(p, want_smem, st) : launch_solve<8, 512>(p, want_smem, st); break;
        case 16: big ? launch_solve<16, 1024>(p, want_smem, st) : launch_solve<16, 512>(p, want_smem, st); break;
        default: big ? launch_solve<32, 1024>(p, want_smem, st) : launch_solve<32, 512>(p, want_smem, st); break;
    }
    int err = read_scalar(d_err, st);
    if (err != 0) throw Error{-4, "bounded wait expired in the sweep kernel"};
    int64_t h_out[8];
    double h_ctrl[2];
    OBK_CUDA(cudaMemcpyAsync(h_out, out.p, sizeof(h_out), cudaMemcpyDeviceToHost, st));
    OBK_CUDA(cudaMemcpyAsync(h_ctrl, ctrl.p, sizeof(h_ctrl), cudaMemcpyDeviceToHost, st));
    OBK_CUDA(cudaStreamSynchronize(st));
    res.sweeps = h_out[0];
    res.status = (int)h_out[1];
    res.outer = h_out[2];
    res.sweep_ms = (double)h_out[4] * 1e-6;
    res.rel_res = h_ctrl[0];
    return res;
}

}  // namespace obk

namespace obk {
namespace {
__global__ void fill_ones(double* p, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = 1.0;
}
}  // namespace

double time_sweep(const SweepLayout& L, int sub, int precision, int block, int staging, int sync_mode, int* d_err,
                  cudaStream_t st)
{
    // scratch system state: x = 0, f = 1 (every sweep does its full work)
    DBuf<double> x(std::max<int64_t>(L.N, 1), st), f(std::max<int64_t>(L.Ngm, 1), st);
    OBK_CUDA(cudaMemsetAsync(x.p, 0, x.bytes(), st));
    fill_ones<<<(unsigned)std::min<int64_t>(ceil_div(f.n, 256), 4096), 256, 0, st>>>(f.p, (int64_t)f.n);
    OBK_CHECK_LAUNCH();
    cudaEvent_t e[4];
    for (auto& ev : e) OBK_CUDA(cudaEventCreate(&ev));
    double per = 0.0;
    try {
        SolveArgs a;
        a.precision = precision;
        a.check_every = 1 << 30;
        a.tol = -1.0;  // never met: exactly maxit sweeps
        a.sub = sub;
        a.block = block;
        a.staging = staging;
        a.sync_mode = sync_mode;
        a.max_outer = 1;
        a.inner_sweeps = 0;
        // the first repetition warms up; the shortest of the three measured
        // ones of each length is taken, so that one slow launch (another
        // process on the GPU, a clock change) cannot make the difference small
        // or negative
        float t2 = 0.f, t8 = 0.f, b2 = 1e30f, b8 = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            a.maxit = 2;
            if (precision == 1) a.inner_sweeps = 2;
            OBK_CUDA(cudaEventRecord(e[0], st));
            run_solve(L, f.p, (double)L.Ngm, 0.0, x.p, a, d_err, st);
            OBK_CUDA(cudaEventRecord(e[1], st));
            a.maxit = 8;
            if (precision == 1) a.inner_sweeps = 8;
            OBK_CUDA(cudaEventRecord(e[2], st));
            run_solve(L, f.p, (double)L.Ngm, 0.0, x.p, a, d_err, st);
            OBK_CUDA(cudaEventRecord(e[3], st));
            OBK_CUDA(cudaEventSynchronize(e[3]));
            OBK_CUDA(cudaEventElapsedTime(&t2, e[0], e[1]));
            OBK_CUDA(cudaEventElapsedTime(&t8, e[2], e[3]));
            if (rep > 0) {
                b2 = std::min(b2, t2);
                b8 = std::min(b8, t8);
            }
        }
        per = (double)(b8 - b2) / 6.0;
        if (!(per > 0.0)) per = (double)b8 / 8.0;  // an upper bound: launch included
    } catch (...) {
        for (auto& ev : e) cudaEventDestroy(ev);
        throw;
    }
    for (auto& ev : e) cudaEventDestroy(ev);
    return per;
}

}  // namespace obk
