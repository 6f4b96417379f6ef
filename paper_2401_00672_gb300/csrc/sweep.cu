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
// A grid barrier separates the phases.  For an exactly orthogonal group the
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

constexpr int kBlock = 512;       // threads per block of the persistent kernel
constexpr int kBlocksPerSm = 2;   // co-resident blocks per SM
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

// acc + S * sum_{j<B} a[q + 32 j] * v[idx[q + 32 j]]   (S = -1 or +1)
template <int B, int S, class T>
__device__ __forceinline__ T sell_batch(const int32_t* idx, const T* vals, const T* v, int64_t q, T acc)
{
    int32_t c[B];
    T a[B];
#pragma unroll
    for (int j = 0; j < B; ++j) {
        c[j] = idx[q + 32 * j];
        a[j] = vals[q + 32 * j];
    }
    T g[B];
#pragma unroll
    for (int j = 0; j < B; ++j) g[j] = v[c[j]];
#pragma unroll
    for (int j = 0; j < B; ++j) acc = fma(S > 0 ? a[j] : -a[j], g[j], acc);
    return acc;
}

// one lane's row (or segment) of a slice: len entries from position q
template <int S, class T>
__device__ __forceinline__ T sell_lane(const int32_t* idx, const T* vals, const T* v, int64_t q, int64_t len, T acc)
{
    int64_t j = 0;
    for (; j + kBatch <= len; j += kBatch, q += 32 * kBatch) acc = sell_batch<kBatch, S, T>(idx, vals, v, q, acc);
    switch ((int)(len - j)) {  // the same for the whole warp
        case 7: acc = sell_batch<7, S, T>(idx, vals, v, q, acc); break;
        case 6: acc = sell_batch<6, S, T>(idx, vals, v, q, acc); break;
        case 5: acc = sell_batch<5, S, T>(idx, vals, v, q, acc); break;
        case 4: acc = sell_batch<4, S, T>(idx, vals, v, q, acc); break;
        case 3: acc = sell_batch<3, S, T>(idx, vals, v, q, acc); break;
        case 2: acc = sell_batch<2, S, T>(idx, vals, v, q, acc); break;
        case 1: acc = sell_batch<1, S, T>(idx, vals, v, q, acc); break;
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

// phase 1 over the row slices of group g: y_k = (rhs_k - A_k . xv) * inv_k
template <class T, class TR>
__device__ __forceinline__ void phase1_sell(const SweepParams& p, int64_t g, const T* sval, const T* inv,
                                            const TR* rhs, const T* xv, T* y)
{
    int lane = threadIdx.x & 31;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t s1 = p.sl_gptr[g + 1];
    for (int64_t s = p.sl_gptr[g] + sell_warp(); s < s1; s += nw) {
        int64_t base = p.sl_ptr[s], len = (p.sl_ptr[s + 1] - base) >> 5;
        bool valid = lane < p.sl_nrow[s];
        int64_t k = p.sl_row0[s] + lane;
        T acc = valid ? (T)rhs[k] : T(0);
        acc = sell_lane<-1, T>(p.sci, sval, xv, base + lane, len, acc);
        if (valid) y[k] = acc * inv[k];
    }
}

// phase 2 over the mirror slices of group g: xv_c += sum_k A_kc y_k
template <class T>
__device__ __forceinline__ void phase2_sell(const SweepParams& p, int64_t g, const T* mval, const T* y, T* xv)
{
    int lane = threadIdx.x & 31;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t s1 = p.ml_gptr[g + 1];
    for (int64_t s = p.ml_gptr[g] + sell_warp(); s < s1; s += nw) {
        int64_t base = p.ml_ptr[s], len = (p.ml_ptr[s + 1] - base) >> 5;
        int32_t c = p.mcol[s * 32 + lane];
        T acc = c >= 0 ? xv[c] : T(0);
        acc = sell_lane<1, T>(p.mrow, mval, y, base + lane, len, acc);
        if (c >= 0) xv[c] = acc;
    }
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
    __shared__ double ws[kBlock / 32];
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
            acc = sell_lane<-1, double>(p.sci, p.sv, p.x, base + lane, len, acc);
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

template <int SUB>
__global__ void __launch_bounds__(kBlock, kBlocksPerSm) obk_solve_kernel(SweepParams p)
{
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
            for (int64_t g = 0; g < p.G; ++g) {
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
            for (int64_t g = 0; g < p.G; ++g) {
                group_phase1<SUB, float, float>(p, g, p.grp_v32, p.sv32, p.grp_inv32, p.b32, p.d32, p.y32);
                if (!grid_sync(p.gb)) return;
                group_phase2<SUB, float>(p, g, p.mir_val32, p.mv32, p.y32, p.d32);
                if (!grid_sync(p.gb)) return;
            }
        }
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

template <int SUB>
void launch_solve(SweepParams& p, cudaStream_t st)
{
    DevInfo di = dev_info();
    const void* k = (const void*)obk_solve_kernel<SUB>;
    // one block per 2K grouped rows, at most kBlocksPerSm per SM: small systems
    // take a few SMs and leave the others to concurrent requests
    int64_t want = std::min<int64_t>((int64_t)di.sms * kBlocksPerSm, ceil_div(std::max<int64_t>(p.Ngm, 1), 2048));
    int grid = coop_grid(k, kBlock, 0, want);
    DBuf<double> partial(grid, st);
    p.partial = partial.p;
    void* args[] = {&p};
    OBK_COOP_LAUNCH(k, grid, kBlock, args, st);
    OBK_CUDA(cudaStreamSynchronize(st));
}

}  // namespace

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
        if (!L.grp_v32.p && L.nnz_gm > 0) throw Error{-1, "precision form needs the FP32 layout"};
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
    p.ctrl = ctrl.p;
    p.out = out.p;
    p.gb = GridBarrier{bar.p, d_err, a.spin_limit};
    int sub = a.sub;
    if (sub == 0) sub = choose_sub(L.Ngm ? (double)L.nnz_gm / (double)L.Ngm : 1.0);
    switch (sub) {
        case 1: launch_solve<1>(p, st); break;
        case 2: launch_solve<2>(p, st); break;
        case 4: launch_solve<4>(p, st); break;
        case 8: launch_solve<8>(p, st); break;
        case 16: launch_solve<16>(p, st); break;
        default: launch_solve<32>(p, st); break;
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

double time_sweep(const SweepLayout& L, int sub, int precision, int* d_err, cudaStream_t st)
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
        a.max_outer = 1;
        a.inner_sweeps = 0;
        float t2 = 0.f, t8 = 0.f;
        for (int rep = 0; rep < 2; ++rep) {  // the first repetition warms up
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
        }
        per = (double)(t8 - t2) / 6.0;
    } catch (...) {
        for (auto& ev : e) cudaEventDestroy(ev);
        throw;
    }
    for (auto& ev : e) cudaEventDestroy(ev);
    return per;
}

}  // namespace obk
