// batch.cu -- many small systems per launch: one thread block per system.
//
// Each block solves one prepared system completely: it gathers f into
// group-major order, permutes x0, computes ||f|| and the all-zero rows' share,
// runs the orthogonal-group sweeps (Eq. 1.3 / Eq. 3.3, Algorithm 4) with x and
// y held in shared memory and __syncthreads between the two phases of a
// group, checks the residual after every check_every-th sweep (or on the
// adaptive cadence), and writes x = P^T x~ (then x^(1:n)) to the output.
// Per-group data (group-major CSR, column mirror) is read from global memory.
#include <math.h>

#include <algorithm>

#include "batch.cuh"
#include "common.cuh"

namespace obk {
namespace {

constexpr int kBatchBlock = 512;

__device__ double block_reduce_sum(double v, double* ws)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) ws[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += ws[k];
    __syncthreads();
    if (threadIdx.x == 0) ws[0] = s;
    __syncthreads();
    s = ws[0];
    __syncthreads();
    return s;
}

// rhs - A_k . xs (one thread, exact-length loop over the row)
__device__ __forceinline__ double row_res(const BatchSystem& d, const double* xs, int64_t k, double rhs)
{
    double acc = rhs;
    for (int64_t q = d.grp_rp[k]; q < d.grp_rp[k + 1]; ++q) acc = fma(-d.grp_v[q], xs[d.grp_ci[q]], acc);
    return acc;
}

__device__ int64_t next_check_b(int64_t s, double rr, int64_t s_prev, double rr_prev, double tol)
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

__global__ void __launch_bounds__(kBatchBlock) batch_kernel(const BatchSystem* systems, int count)
{
    extern __shared__ double smem[];
    __shared__ double ws[kBatchBlock / 32];
    __shared__ int s_stop;
    if ((int)blockIdx.x >= count) return;
    const BatchSystem& d = systems[blockIdx.x];
    double* xs = smem;            // N
    double* ys = smem + d.N;      // Ngm
    double* fs = ys + d.Ngm;      // Ngm (f in group-major order)
    // load: x~0 = P x^0, f in group-major order
    for (int64_t k = threadIdx.x; k < d.N; k += blockDim.x) {
        int32_t o = d.perm[k];
        xs[k] = (d.x0 && o < d.n) ? d.x0[o] : 0.0;
    }
    for (int64_t k = threadIdx.x; k < d.Ngm; k += blockDim.x) {
        int32_t o = d.src_gm[k];
        fs[k] = o < d.m ? d.f[o] : 0.0;
    }
    double ff = 0.0, zf = 0.0;
    for (int64_t i = threadIdx.x; i < d.m; i += blockDim.x) ff = fma(d.f[i], d.f[i], ff);
    for (int64_t t = threadIdx.x; t < d.n_zero; t += blockDim.x) {
        int32_t o = d.zero_src[t];
        double v = o < d.m ? d.f[o] : 0.0;
        zf = fma(v, v, zf);
    }
    double fnorm2 = block_reduce_sum(ff, ws);
    double zero_f2 = block_reduce_sum(zf, ws);
    double fnorm = sqrt(fnorm2);
    __syncthreads();

    auto residual = [&]() -> double {
        double loc = 0.0;
        for (int64_t k = threadIdx.x; k < d.Ngm; k += blockDim.x) {
            double r = row_res(d, xs, k, fs[k]);
            loc = fma(r, r, loc);
        }
        double tot = block_reduce_sum(loc, ws) + zero_f2;
        return fnorm > 0.0 ? sqrt(tot) / fnorm : sqrt(tot);
    };

    double rr = residual();
    int status = rr <= d.tol ? 0 : 1;
    int64_t s = 0, nchk = 0, next = 1, s_prev = 0;
    double rr_prev = rr;
    double hist[10];
    while (status != 0 && s < d.maxit) {
        for (int64_t g = 0; g < d.G; ++g) {
            for (int64_t k = d.gptr[g] + threadIdx.x; k < d.gptr[g + 1]; k += blockDim.x)
                ys[k] = row_res(d, xs, k, fs[k]) * d.grp_inv[k];
            __syncthreads();
            for (int64_t t = d.gseg_ptr[g] + threadIdx.x; t < d.gseg_ptr[g + 1]; t += blockDim.x) {
                int32_t c = d.seg_col[t];
                double acc = xs[c];
                for (int64_t q = d.seg_ptr[t]; q < d.seg_ptr[t + 1]; ++q) acc = fma(d.mir_val[q], ys[d.mir_row[q]], acc);
                xs[c] = acc;
            }
            __syncthreads();
        }
        ++s;
        bool check = d.check_every > 0 ? ((s % d.check_every) == 0 || s >= d.maxit) : (s >= next || s >= d.maxit);
        if (check) {
            rr = residual();
            if (threadIdx.x == 0) {
                int stop = 0;
                if (rr <= d.tol) stop = 2;
                else if (s >= d.maxit) stop = 1;
                else if (d.stagnation > 0.0) {
                    if (nchk >= 10 && fabs(rr - hist[nchk % 10]) < d.stagnation) stop = 1;
                    hist[nchk % 10] = rr;
                }
                s_stop = stop;
            }
            ++nchk;
            next = next_check_b(s, rr, s_prev, rr_prev, d.tol);
            s_prev = s;
            rr_prev = rr;
            __syncthreads();
            int stop = s_stop;
            __syncthreads();
            if (stop == 2) status = 0;
            if (stop) break;
        }
    }
    // x = P^T x~, then x^(1:n)
    for (int64_t k = threadIdx.x; k < d.N; k += blockDim.x) {
        int32_t o = d.perm[k];
        if (o < d.n) d.x_out[o] = xs[k];
    }
    if (threadIdx.x == 0) {
        d.result[0] = (double)status;
        d.result[1] = (double)s;
        d.result[2] = rr;
    }
}

}  // namespace

size_t batch_smem_bytes(int64_t N, int64_t Ngm) { return (size_t)(N + 2 * Ngm) * sizeof(double); }

size_t batch_smem_limit()
{
    DevInfo di = dev_info();
    return di.smem_optin > 1024 ? di.smem_optin - 1024 : 0;  // leave room for the static shared memory
}

void launch_batch(const BatchSystem* d_systems, int count, size_t smem, cudaStream_t st)
{
    OBK_CUDA(cudaFuncSetAttribute((const void*)batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)batch_smem_limit()));
    batch_kernel<<<(unsigned)count, kBatchBlock, smem, st>>>(d_systems, count);
    OBK_CHECK_LAUNCH();
}

}  // namespace obk
