// peaks.cu -- measured throughput ceilings of the current GPU for the
// rooflines the library's kernels are judged against: FP64 and FP32
// multiply-add rates (the sweep's arithmetic), random 8-byte gathers from an
// L2-resident array (the sweep's x and y accesses) and the L2 streaming read
// rate.  Not part of the method; a measurement helper for benchmarks.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/obk.h"
#include "common.cuh"

namespace {

constexpr int kPeakBlock = 256;
constexpr int kChains = 8;  // independent multiply-add chains per thread

template <class T>
__global__ void __launch_bounds__(kPeakBlock) fma_chains(T* out, int iters, T b, T c)
{
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == (T)-12345.0) out[0] = s;  // never true: keeps the chains live
    if (threadIdx.x == 0 && blockIdx.x == 0) out[1] = s;
}

// Integer multiply-add chains (64-bit or 32-bit): the index arithmetic of the
// sparse kernels.
template <class T>
__global__ void __launch_bounds__(kPeakBlock) imad_chains(T* out, int iters, T b, T c)
{
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = a[k] * b + c;
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s ^= a[k];
    if (s == (T)12345) out[0] = s;
}

// Each thread gathers `iters` 8-byte words at pseudo-random positions of an
// array of n words (n a power of two) that fits in L2: the position comes from
// an integer hash, so no index array is read.
__global__ void __launch_bounds__(kPeakBlock) l2_gather(const double* __restrict__ x, uint32_t mask, int iters,
                                                        double* out)
{
    uint32_t h = (blockIdx.x * kPeakBlock + threadIdx.x) * 2654435761u + 12345u;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = 0; i < iters; i += 4) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            h ^= h << 13;
            h ^= h >> 17;
            h ^= h << 5;
            acc[k] += x[h & mask];
        }
    }
    double s = acc[0] + acc[1] + acc[2] + acc[3];
    if (s == -12345.0) out[0] = s;
}

// Grid-stride coalesced reads of an L2-resident array, `reps` times over.
// (the words are combined with integer XOR, so no FP64 add bounds the rate)
__global__ void __launch_bounds__(kPeakBlock) l2_stream(const ulonglong4_32a* __restrict__ x, int64_t n4, int reps,
                                                        double* out)
{
    unsigned long long s = 0;
    int64_t tid = (int64_t)blockIdx.x * kPeakBlock + threadIdx.x, nth = (int64_t)gridDim.x * kPeakBlock;
    for (int r = 0; r < reps; ++r)
        for (int64_t i = tid; i < n4; i += nth) {
            ulonglong4_32a v = x[i];
            s ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    if (s == 0x123456789abcdefull) out[0] = (double)s;
}

template <class F>
float best_ms(F launch, cudaStream_t st, int reps)
{
    cudaEvent_t e0, e1;
    OBK_CUDA(cudaEventCreate(&e0));
    OBK_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int r = 0; r < reps + 1; ++r) {  // the first run warms up
        OBK_CUDA(cudaEventRecord(e0, st));
        launch();
        OBK_CUDA(cudaEventRecord(e1, st));
        OBK_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        OBK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (r > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

}  // namespace

extern "C" obk_status obk_measure_peaks(obk_peaks* out)
{
    OBK_API_BEGIN
    obk::set_last_error("");
    if (!out) throw obk::Error{OBK_ERR_INVALID, "out is NULL"};
    obk::DevInfo di = obk::dev_info();
    cudaStream_t st;
    OBK_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    try {
        const int blocks = di.sms * 8;  // 2048 threads per SM
        const int64_t threads = (int64_t)blocks * kPeakBlock;
        obk::DBuf<double> sink(4, st);
        obk::DBuf<float> sink32(4, st);
        const int it64 = 4096, it32 = 32768;
        float ms64 = best_ms([&] {
            fma_chains<double><<<blocks, kPeakBlock, 0, st>>>(sink.p, it64, 0.9999999, 1e-7);
            OBK_CHECK_LAUNCH();
        }, st, 3);
        float ms32 = best_ms([&] {
            fma_chains<float><<<blocks, kPeakBlock, 0, st>>>(sink32.p, it32, 0.9999f, 1e-4f);
            OBK_CHECK_LAUNCH();
        }, st, 3);
        obk::DBuf<unsigned long long> isink(4, st);
        obk::DBuf<unsigned> isink32(4, st);
        const int iti = 8192;
        float msi64 = best_ms([&] {
            imad_chains<unsigned long long><<<blocks, kPeakBlock, 0, st>>>(isink.p, iti, 6364136223846793005ull,
                                                                          1442695040888963407ull);
            OBK_CHECK_LAUNCH();
        }, st, 3);
        float msi32 = best_ms([&] {
            imad_chains<unsigned><<<blocks, kPeakBlock, 0, st>>>(isink32.p, iti, 1664525u, 1013904223u);
            OBK_CHECK_LAUNCH();
        }, st, 3);
        out->int64_mad_tops = (double)threads * kChains * iti / (msi64 * 1e-3) / 1e12;
        out->int32_mad_tops = (double)threads * kChains * iti / (msi32 * 1e-3) / 1e12;
        out->fp64_fma_tflops = 2.0 * threads * kChains * it64 / (ms64 * 1e-3) / 1e12;
        out->fp32_fma_tflops = 2.0 * threads * kChains * it32 / (ms32 * 1e-3) / 1e12;

        // L2-resident arrays: 8 MB for the gathers (the 1M-row x), 32 MB streamed
        const int64_t ng = 1 << 20, ns = 4 << 20;
        obk::DBuf<double> xg(ng, st), xs(ns, st);
        OBK_CUDA(cudaMemsetAsync(xg.p, 0, xg.bytes(), st));
        OBK_CUDA(cudaMemsetAsync(xs.p, 0, xs.bytes(), st));
        const int git = 512;
        float msg = best_ms([&] {
            l2_gather<<<blocks, kPeakBlock, 0, st>>>(xg.p, (uint32_t)(ng - 1), git, sink.p);
            OBK_CHECK_LAUNCH();
        }, st, 3);
        out->l2_gather_g_per_s = (double)threads * git / (msg * 1e-3) / 1e9;
        const int reps = 200;
        float mss = best_ms([&] {
            l2_stream<<<blocks, kPeakBlock, 0, st>>>(reinterpret_cast<const ulonglong4_32a*>(xs.p), ns / 4, reps, sink.p);
            OBK_CHECK_LAUNCH();
        }, st, 3);
        out->l2_read_gbs = (double)ns * 8.0 * reps / (mss * 1e-3) / 1e9;
        OBK_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
        throw;
    }
    OBK_CUDA(cudaStreamDestroy(st));
    return OBK_OK;
    OBK_API_END
}
