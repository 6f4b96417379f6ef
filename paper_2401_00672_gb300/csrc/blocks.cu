// blocks.cu -- the paper-literal block form of OBK-RCM (Section 3.3,
// Algorithm 4): the RCM-ordered matrix A~ cut into k uniform row blocks, the
// cosines between the blocks' centroids, the classes of orthogonal block pairs
// (Oclass) and of the remaining blocks (Nclass), and block projections
// x += A_b^+ (f_b - A_b x) (Eq. 3.3) computed by CGLS from zero (which
// converges to the minimum-norm correction).
//
// Iteration j projects onto the two blocks of Oclass pair j mod P, one after
// the other, then onto the Nclass block j mod Q; the relative residual is
// checked after every iteration.
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace obk {
namespace {

constexpr int kBlk = 256;   // simple kernels
constexpr int kCg = 512;    // the cooperative CGLS kernel
constexpr int kResTile = 4096;

inline unsigned grid_of(int64_t n) { return (unsigned)std::min<int64_t>(ceil_div(n, kBlk) + 1, 65535); }

#define GSTRIDE(i, n)                                                                      \
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n);            \
         i += (int64_t)gridDim.x * blockDim.x)

// rows of block b: the first k - 1 blocks take floor(N / k) rows in order, the last the rest
__host__ __device__ inline void block_rows(int64_t N, int k, int b, int64_t* b0, int64_t* b1)
{
    int64_t w = N / k;
    *b0 = (int64_t)b * w;
    *b1 = b == k - 1 ? N : *b0 + w;
}

// column range [lo, hi] of each block (lo > hi for a block without entries)
__global__ void block_col_range(int64_t N, int k, const int64_t* rp, const int32_t* ci, unsigned long long* lo,
                                unsigned long long* hi)
{
    int64_t w = N / k;
    GSTRIDE(i, N)
    {
        if (rp[i + 1] == rp[i]) continue;
        int b = (int)std::min<int64_t>(i / w, (int64_t)k - 1);
        atomicMin(lo + b, (unsigned long long)ci[rp[i]]);
        atomicMax(hi + b, (unsigned long long)ci[rp[i + 1] - 1]);
    }
}

// first CSC position of column c holding a row >= r (rows ascending)
__device__ __forceinline__ int64_t col_lower(const int64_t* cptr, const int32_t* crow, int64_t c, int64_t r)
{
    int64_t a = cptr[c], e = cptr[c + 1];
    while (a < e) {
        int64_t mid = (a + e) >> 1;
        if (crow[mid] < r) a = mid + 1;
        else e = mid;
    }
    return a;
}

// centroid slices: cen[off[b] + c - lo[b]] = (sum of the block's column-c
// entries, rows ascending) / rows of the block, as a left fold
__global__ void centroid_slices(int k, int64_t N, const unsigned long long* lo, const int64_t* off, int64_t total,
                                const int64_t* cptr, const int32_t* crow, const double* cval, double* cen)
{
    GSTRIDE(t, total)
    {
        int a = 0, e = k;  // block: largest b with off[b] <= t
        while (e - a > 1) {
            int mid = (a + e) >> 1;
            if (off[mid] <= t) a = mid;
            else e = mid;
        }
        int b = a;
        int64_t c = (int64_t)lo[b] + (t - off[b]);
        int64_t b0, b1;
        block_rows(N, k, b, &b0, &b1);
        double s = 0.0;
        for (int64_t q = col_lower(cptr, crow, c, b0); q < cptr[c + 1] && crow[q] < b1; ++q) s = s + cval[q];
        cen[t] = s / (double)(b1 - b0);
    }
}

__global__ void centroid_norms(int k, const int64_t* off, const double* cen, double* nrm)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= k) return;
    double q = 0.0;
    for (int64_t t = off[b]; t < off[b + 1]; ++t) q = q + cen[t] * cen[t];
    nrm[b] = sqrt(q);
}

// orth[i k + j] = 1 when |cos(centroid_i, centroid_j)| < thr (i < j); the dot
// product folds over the common columns in ascending order
__global__ void centroid_pairs(int k, const unsigned long long* lo, const unsigned long long* hi, const int64_t* off,
                               const double* cen, const double* nrm, double thr, unsigned char* orth)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= k * k) return;
    int i = t / k, j = t % k;
    if (i >= j) return;
    double g = 0.0;
    if (lo[i] <= hi[i] && lo[j] <= hi[j]) {
        int64_t c0 = (int64_t)std::max(lo[i], lo[j]), c1 = (int64_t)std::min(hi[i], hi[j]);
        for (int64_t c = c0; c <= c1; ++c)
            g = g + cen[off[i] + c - (int64_t)lo[i]] * cen[off[j] + c - (int64_t)lo[j]];
    }
    double den = nrm[i] * nrm[j];
    double cosv = den > 0.0 ? g / den : 0.0;
    orth[t] = fabs(cosv) < thr ? 1 : 0;
}

// Algorithm 4's classes (one thread): each block not yet in a class is paired
// with the first later block, not yet in a class, orthogonal to it
__global__ void make_classes(int k, const unsigned char* orth, int32_t* pairs, int32_t* nclass, int32_t* counts,
                             unsigned char* used)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int b = 0; b < k; ++b) used[b] = 0;
    int np = 0, nq = 0;
    for (int i = 0; i < k; ++i) {
        if (used[i]) continue;
        for (int j = i + 1; j < k; ++j)
            if (!used[j] && orth[i * k + j]) {
                pairs[2 * np] = i;
                pairs[2 * np + 1] = j;
                ++np;
                used[i] = used[j] = 1;
                break;
            }
    }
    for (int i = 0; i < k; ++i)
        if (!used[i]) nclass[nq++] = i;
    counts[0] = np;
    counts[1] = nq;
}

// ---- CGLS block projection (persistent, cooperative) --------------------------

struct CgParams {
    int64_t b0, b1, lo, hi;  // the block's rows and column range
    const int64_t* rp;
    const int32_t* ci;
    const double* v;
    const int64_t* cptr;
    const int32_t* crow;
    const double* cval;
    const double* f;         // f~ (N)
    double* x;               // x~ (N)
    double* d;               // R = hi - lo + 1
    double* p;               // R
    double* sv;              // R
    int64_t* cs;             // R: first CSC position of the column inside the block
    double* r;               // B
    double* q;               // B
    double* partial;         // 2 gridDim
    int inner_max;
    double inner_tol;
    int64_t* steps;          // out
    GridBarrier gb;
};

__device__ double cg_block_sum(double v)
{
    __shared__ double ws[kCg / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) ws[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += ws[k];
    __syncthreads();
    return s;
}

// Sum of every thread's value over the grid, the same (fixed order) in every
// block; `slot` alternates between two partial arrays so that a block writing
// the next reduction never overtakes one still reading this one.
__device__ bool cg_allreduce(const CgParams& P, double v, int slot, double* out)
{
    __shared__ double s_tot;
    double s = cg_block_sum(v);
    double* part = P.partial + (size_t)slot * gridDim.x;
    if (threadIdx.x == 0) part[blockIdx.x] = s;
    if (!grid_sync(P.gb)) return false;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) t += ((volatile double*)part)[b];
        s_tot = t;
    }
    __syncthreads();
    *out = s_tot;
    return true;
}

__global__ void __launch_bounds__(kCg) cgls_project(CgParams P)
{
    const int64_t B = P.b1 - P.b0, R = P.hi - P.lo + 1;
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t nth = (int64_t)gridDim.x * blockDim.x;
    int slot = 0;
    // r = f_b - A_b x, d = 0, and each column's first entry inside the block
    for (int64_t t = tid; t < B; t += nth) {
        int64_t i = P.b0 + t;
        double a = 0.0;
        for (int64_t e = P.rp[i]; e < P.rp[i + 1]; ++e) a = fma(P.v[e], P.x[P.ci[e]], a);
        P.r[t] = P.f[i] - a;
    }
    for (int64_t c = tid; c < R; c += nth) {
        P.d[c] = 0.0;
        P.cs[c] = col_lower(P.cptr, P.crow, P.lo + c, P.b0);
    }
    if (!grid_sync(P.gb)) return;
    // sv = A_b^T r, p = sv, gamma = ||sv||^2
    double loc = 0.0;
    for (int64_t c = tid; c < R; c += nth) {
        double s = 0.0;
        for (int64_t q = P.cs[c]; q < P.cptr[P.lo + c + 1] && P.crow[q] < P.b1; ++q)
            s = fma(P.cval[q], P.r[P.crow[q] - P.b0], s);
        P.sv[c] = s;
        P.p[c] = s;
        loc = fma(s, s, loc);
    }
    double gamma;
    if (!cg_allreduce(P, loc, slot, &gamma)) return;
    slot ^= 1;
    const double gamma0 = gamma, stop2 = P.inner_tol * P.inner_tol * gamma0;
    int64_t it = 0;
    while (it < P.inner_max && gamma > stop2 && gamma > 0.0) {
        // q = A_b p
        loc = 0.0;
        for (int64_t t = tid; t < B; t += nth) {
            int64_t i = P.b0 + t;
            double a = 0.0;
            for (int64_t e = P.rp[i]; e < P.rp[i + 1]; ++e) a = fma(P.v[e], P.p[P.ci[e] - P.lo], a);
            P.q[t] = a;
            loc = fma(a, a, loc);
        }
        double qq;
        if (!cg_allreduce(P, loc, slot, &qq)) return;
        slot ^= 1;
        if (qq == 0.0) break;
        double alpha = gamma / qq;
        for (int64_t c = tid; c < R; c += nth) P.d[c] = fma(alpha, P.p[c], P.d[c]);
        for (int64_t t = tid; t < B; t += nth) P.r[t] = fma(-alpha, P.q[t], P.r[t]);
        if (!grid_sync(P.gb)) return;
        // sv = A_b^T r
        loc = 0.0;
        for (int64_t c = tid; c < R; c += nth) {
            double s = 0.0;
            for (int64_t q = P.cs[c]; q < P.cptr[P.lo + c + 1] && P.crow[q] < P.b1; ++q)
                s = fma(P.cval[q], P.r[P.crow[q] - P.b0], s);
            P.sv[c] = s;
            loc = fma(s, s, loc);
        }
        double gn;
        if (!cg_allreduce(P, loc, slot, &gn)) return;
        slot ^= 1;
        double beta = gn / gamma;
        for (int64_t c = tid; c < R; c += nth) P.p[c] = fma(beta, P.p[c], P.sv[c]);
        gamma = gn;
        ++it;
        if (!grid_sync(P.gb)) return;
    }
    for (int64_t c = tid; c < R; c += nth) P.x[P.lo + c] += P.d[c];
    if (tid == 0) *P.steps += it;
}

// ||f - A x||^2 and ||f||^2 per tile of kResTile rows (fixed order), then the total
__global__ void res_tiles(int64_t N, const int64_t* rp, const int32_t* ci, const double* v, const double* f,
                          const double* x, double* part)
{
    __shared__ double wr[kBlk / 32], wf[kBlk / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t r0 = (int64_t)blockIdx.x * kResTile, r1 = std::min<int64_t>(r0 + kResTile, N);
    double sr = 0.0, sf = 0.0;
    for (int64_t i = r0 + w; i < r1; i += kBlk / 32) {
        double acc = 0.0;
        for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += 32) acc = fma(v[e], x[ci[e]], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        double r = f[i] - acc;
        sr = fma(r, r, sr);
        sf = fma(f[i], f[i], sf);
    }
    if (lane == 0) { wr[w] = sr; wf[w] = sf; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < kBlk / 32; ++k) { a += wr[k]; b += wf[k]; }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

__global__ void res_final(const double* part, int64_t ntiles, double* out)
{
    if (blockIdx.x || threadIdx.x) return;
    double a = 0.0, b = 0.0;
    for (int64_t t = 0; t < ntiles; ++t) { a += part[2 * t]; b += part[2 * t + 1]; }
    *out = b > 0.0 ? sqrt(a) / sqrt(b) : sqrt(a);
}

}  // namespace

BlockResult run_blocks(int64_t N, const int64_t* rp, const int32_t* ci, const double* v, const int64_t* cptr,
                       const int32_t* crow, const double* cval, const double* ft, double* xt, const BlockArgs& a,
                       int* d_err, cudaStream_t st)
{
    BlockResult res;
    const int k = a.k;
    DevInfo di = dev_info();
    // 1. classes from the centroid cosines
    DBuf<unsigned long long> lo(k, st), hi(k, st);
    OBK_CUDA(cudaMemsetAsync(lo.p, 0xff, k * sizeof(unsigned long long), st));
    OBK_CUDA(cudaMemsetAsync(hi.p, 0, k * sizeof(unsigned long long), st));
    block_col_range<<<grid_of(N), kBlk, 0, st>>>(N, k, rp, ci, lo.p, hi.p);
    OBK_CHECK_LAUNCH();
    std::vector<unsigned long long> hlo(k), hhi(k);
    OBK_CUDA(cudaMemcpyAsync(hlo.data(), lo.p, k * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    OBK_CUDA(cudaMemcpyAsync(hhi.data(), hi.p, k * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    OBK_CUDA(cudaStreamSynchronize(st));
    std::vector<int64_t> hoff(k + 1, 0);
    for (int b = 0; b < k; ++b) hoff[b + 1] = hoff[b] + (hlo[b] <= hhi[b] ? (int64_t)(hhi[b] - hlo[b] + 1) : 0);
    int64_t total = hoff[k];
    DBuf<int64_t> off(k + 1, st);
    OBK_CUDA(cudaMemcpyAsync(off.p, hoff.data(), (k + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    DBuf<double> cen(std::max<int64_t>(total, 1), st), nrm(k, st);
    if (total) {
        centroid_slices<<<grid_of(total), kBlk, 0, st>>>(k, N, lo.p, off.p, total, cptr, crow, cval, cen.p);
        OBK_CHECK_LAUNCH();
    }
    centroid_norms<<<(unsigned)ceil_div(k, 64), 64, 0, st>>>(k, off.p, cen.p, nrm.p);
    OBK_CHECK_LAUNCH();
    DBuf<unsigned char> orth((int64_t)k * k, st), used(k, st);
    OBK_CUDA(cudaMemsetAsync(orth.p, 0, (size_t)k * k, st));
    centroid_pairs<<<(unsigned)ceil_div((int64_t)k * k, 128), 128, 0, st>>>(k, lo.p, hi.p, off.p, cen.p, nrm.p,
                                                                             a.thr, orth.p);
    OBK_CHECK_LAUNCH();
    DBuf<int32_t> pairs(2 * k + 2, st), nclass(k + 1, st), counts(2, st);
    make_classes<<<1, 1, 0, st>>>(k, orth.p, pairs.p, nclass.p, counts.p, used.p);
    OBK_CHECK_LAUNCH();
    std::vector<int32_t> hpairs(2 * k + 2), hncl(k + 1), hcnt(2);
    OBK_CUDA(cudaMemcpyAsync(hcnt.data(), counts.p, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    OBK_CUDA(cudaMemcpyAsync(hpairs.data(), pairs.p, (2 * k + 2) * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    OBK_CUDA(cudaMemcpyAsync(hncl.data(), nclass.p, (k + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    OBK_CUDA(cudaStreamSynchronize(st));
    const int np = hcnt[0], nq = hcnt[1];
    res.n_pairs = np;
    res.n_nclass = nq;
    cen.release();

    // 2. scratch for the projections (sized for the widest block)
    int64_t maxB = 0, maxR = 1;
    for (int b = 0; b < k; ++b) {
        int64_t b0, b1;
        block_rows(N, k, b, &b0, &b1);
        maxB = std::max(maxB, b1 - b0);
        if (hlo[b] <= hhi[b]) maxR = std::max<int64_t>(maxR, (int64_t)(hhi[b] - hlo[b] + 1));
    }
    DBuf<double> d(maxR, st), p(maxR, st), sv(maxR, st), r(std::max<int64_t>(maxB, 1), st),
        q(std::max<int64_t>(maxB, 1), st);
    DBuf<int64_t> cs(maxR, st), steps(1, st);
    OBK_CUDA(cudaMemsetAsync(steps.p, 0, sizeof(int64_t), st));
    DBuf<unsigned> bar(kBarrierWords, st);
    int64_t want = std::min<int64_t>((int64_t)di.sms * 2, ceil_div(std::max(maxB, maxR), (int64_t)2 * kCg));
    int grid = coop_grid((const void*)cgls_project, kCg, 0, want);
    DBuf<double> partial(2 * (int64_t)grid, st);
    auto project = [&](int b) {
        if (hlo[b] > hhi[b]) return;  // a block without entries changes nothing
        int64_t b0, b1;
        block_rows(N, k, b, &b0, &b1);
        OBK_CUDA(cudaMemsetAsync(bar.p, 0, kBarrierWords * sizeof(unsigned), st));
        CgParams P{b0, b1, (int64_t)hlo[b], (int64_t)hhi[b], rp, ci, v, cptr, crow, cval, ft, xt,
                   d.p, p.p, sv.p, cs.p, r.p, q.p, partial.p, a.inner_max, a.inner_tol, steps.p,
                   GridBarrier{bar.p, d_err, a.spin_limit}};
        void* args[] = {&P};
        OBK_COOP_LAUNCH(cgls_project, grid, kCg, args, st);
    };
    // 3. the iteration, residual after each
    int64_t ntiles = ceil_div(std::max<int64_t>(N, 1), (int64_t)kResTile);
    DBuf<double> rpart(2 * ntiles, st), rr(1, st);
    auto residual = [&]() -> double {
        res_tiles<<<(unsigned)ntiles, kBlk, 0, st>>>(N, rp, ci, v, ft, xt, rpart.p);
        OBK_CHECK_LAUNCH();
        res_final<<<1, 32, 0, st>>>(rpart.p, ntiles, rr.p);
        OBK_CHECK_LAUNCH();
        double x = read_scalar(rr.p, st);
        if (read_scalar(d_err, st) != 0) throw Error{-4, "bounded wait expired in a block projection"};
        return x;
    };
    double rel = residual();
    res.status = rel <= a.tol ? 0 : 1;
    for (int64_t j = 0; res.status != 0 && j < a.maxit; ++j) {
        if (np > 0) {
            int pp = (int)(j % np);
            project(hpairs[2 * pp]);
            project(hpairs[2 * pp + 1]);
        }
        if (nq > 0) project(hncl[j % nq]);
        res.iters = j + 1;
        rel = residual();
        if (rel <= a.tol) res.status = 0;
    }
    res.rel_res = rel;
    res.cgls_steps = read_scalar(steps.p, st);
    return res;
}

}  // namespace obk
