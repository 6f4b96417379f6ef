// noalloc.cu -- obk_residual_noalloc: the residual check for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the moment they need a residual: a
// process whose device memory is entirely reserved by another allocator or
// pool, or a latency-critical loop where an allocation (which may synchronise
// the device) is not acceptable.  This entry point computes the same
// quantity as obk_residual (same tiles, same summation order) but keeps its
// scratch -- two partial sums per tile of 4096 rows -- in a fixed-size array
// that lives in device memory for as long as the library is loaded.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>
#include <string>

#include "../../include/obk.h"
#include "common.cuh"

namespace {

constexpr int kBlock = 256;
constexpr int kTile = 4096;                 // rows per partial sum (as in obk_residual)
constexpr int64_t kMaxTiles = 16384;        // -> at most 67,108,864 rows
constexpr int64_t kMaxRows = kMaxTiles * kTile;
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device: part[2t] = sum of r_i^2 and
// part[2t+1] = sum of f_i^2 over tile t.  256 KB per device that loads the
// library, held until the process exits.  In host code this name is only a
// stand-in; kernels receive the device address from cudaGetSymbolAddress.
static __device__ __align__(256) double g_residual_scratch[2 * kMaxTiles];

__global__ void residual_tiles_static(int64_t m, const int64_t* rp, const int32_t* ci, const double* v,
                                      const double* f, const double* x, double* part)
{
    __shared__ double wr[kBlock / 32], wf[kBlock / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t r0 = (int64_t)blockIdx.x * kTile, r1 = r0 + kTile < m ? r0 + kTile : m;
    double sr = 0.0, sf = 0.0;
    for (int64_t i = r0 + w; i < r1; i += kBlock / 32) {
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
        for (int k = 0; k < kBlock / 32; ++k) { a += wr[k]; b += wf[k]; }
        part[2 * blockIdx.x] = a;      // every tile of this call writes both of its
        part[2 * blockIdx.x + 1] = b;  // slots, so nothing needs clearing first
    }
}

__global__ void residual_final_static(const double* part, int64_t ntiles, double* out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int64_t t = 0; t < ntiles; ++t) { a += part[2 * t]; b += part[2 * t + 1]; }
        *out = b > 0.0 ? sqrt(a) / sqrt(b) : sqrt(a);
    }
}

std::mutex g_mu;
double* g_scratch_of_device[kMaxDevices] = {};

bool on_device(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" obk_status obk_residual_noalloc(const int64_t* row_ptr, const int32_t* col_idx, const double* val,
                                           int64_t m, int64_t n, const double* f, const double* x,
                                           double* rel_res, void* stream)
{
    if (!row_ptr || !f || !x || !rel_res || m <= 0 || n <= 0) {
        obk::set_last_error("obk_residual_noalloc: NULL pointer or non-positive size");
        return OBK_ERR_INVALID;
    }
    if (m > kMaxRows) {
        obk::set_last_error("obk_residual_noalloc: m = " + std::to_string(m) + " exceeds the maximum of " +
                            std::to_string(kMaxRows) + " rows of its fixed scratch");
        return OBK_ERR_INVALID;
    }
    if (!on_device(row_ptr) || !on_device(f) || !on_device(x) || !on_device(rel_res) ||
        (col_idx && !on_device(col_idx)) || (val && !on_device(val))) {
        obk::set_last_error("obk_residual_noalloc: every array must be in device memory");
        return OBK_ERR_INVALID;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        obk::set_last_error("obk_residual_noalloc: no usable current device");
        return OBK_ERR_CUDA;
    }
    double* scratch = nullptr;
    {
        // set-up, once per device with that device current: the device address
        // of the file-scope scratch array
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_of_device[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_residual_scratch);
            if (e != cudaSuccess || !p) {
                (void)cudaGetLastError();
                obk::set_last_error(std::string("obk_residual_noalloc: cudaGetSymbolAddress failed: ") +
                                    cudaGetErrorString(e));
                return OBK_ERR_CUDA;
            }
            g_scratch_of_device[dev] = static_cast<double*>(p);
        }
        scratch = g_scratch_of_device[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int64_t ntiles = (m + kTile - 1) / kTile;
    residual_tiles_static<<<(unsigned)ntiles, kBlock, 0, st>>>(m, row_ptr, col_idx, val, f, x, scratch);
    obk::count_launch();
    residual_final_static<<<1, 32, 0, st>>>(scratch, ntiles, rel_res);
    obk::count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        obk::set_last_error(std::string("obk_residual_noalloc: launch failed: ") + cudaGetErrorString(e));
        return OBK_ERR_CUDA;
    }
    return OBK_OK;
}
