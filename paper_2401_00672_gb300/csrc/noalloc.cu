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
#include "residual.cuh"

namespace {

constexpr int kBlock = obk::kResBlock;
constexpr int kTile = obk::kResTile;        // rows per partial sum (as in obk_residual)
constexpr int64_t kMaxTiles = 16384;        // -> at most 67,108,864 rows
constexpr int64_t kMaxRows = kMaxTiles * kTile;
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device: part[2t] = sum of r_i^2 and
// part[2t+1] = sum of f_i^2 over tile t.  256 KB per device that loads the
// library, held until the process exits.  In host code this name is only a
// stand-in; kernels receive the device address from cudaGetSymbolAddress.
static __device__ __align__(256) double g_residual_scratch[2 * kMaxTiles];

// The same per-tile body and final sum as obk_residual (residual.cuh), so the
// two entry points return identical values.
__global__ void residual_tiles_static(int64_t m, const int64_t* rp, const int32_t* ci, const double* v,
                                      const double* f, const double* x, double* part)
{
    obk::residual_tile_sums(m, rp, ci, v, f, x, part, blockIdx.x);
}

__global__ void residual_final_static(const double* part, int64_t ntiles, double* out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *out = obk::residual_from_tiles(part, ntiles);
}

std::mutex g_mu;
double* g_scratch_of_device[kMaxDevices] = {};

// True when p is memory that kernels on device `dev` can address directly:
// device memory of that device, or managed memory.
bool on_device(const void* p, int dev)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" obk_status obk_residual_noalloc(const int64_t* row_ptr, const int32_t* col_idx, const double* val,
                                           int64_t m, int64_t n, const double* f, const double* x,
                                           double* rel_res, void* stream)
{
    OBK_API_BEGIN
    obk::set_last_error("");
    if (!row_ptr || !col_idx || !val || !f || !x || !rel_res || m <= 0 || n <= 0)
        throw obk::Error{OBK_ERR_INVALID, "obk_residual_noalloc: NULL pointer or non-positive size"};
    if (m > kMaxRows)
        throw obk::Error{OBK_ERR_INVALID, "obk_residual_noalloc: m = " + std::to_string(m) +
                                              " exceeds the maximum of " + std::to_string(kMaxRows) +
                                              " rows of its fixed scratch"};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        (void)cudaGetLastError();
        throw obk::Error{OBK_ERR_CUDA, "obk_residual_noalloc: no usable current device"};
    }
    if (!on_device(row_ptr, dev) || !on_device(col_idx, dev) || !on_device(val, dev) || !on_device(f, dev) ||
        !on_device(x, dev) || !on_device(rel_res, dev))
        throw obk::Error{OBK_ERR_INVALID,
                         "obk_residual_noalloc: every array must be in device memory of the current device"};
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
                throw obk::Error{OBK_ERR_CUDA, std::string("obk_residual_noalloc: cudaGetSymbolAddress failed: ") +
                                                   cudaGetErrorString(e)};
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
    if (e != cudaSuccess)
        throw obk::Error{OBK_ERR_CUDA, std::string("obk_residual_noalloc: launch failed: ") + cudaGetErrorString(e)};
    return OBK_OK;
    OBK_API_END
}
