// residual.cuh -- the relative residual ||f - A x||_2 / ||f||_2 (the stop test
// of the solve, Sec. 3.5 read as a residual) on a plain CSR matrix, shared by
// obk_residual and obk_residual_noalloc so that both compute it with the same
// arithmetic in the same order.
//
// Tile t covers rows [t * kResTile, (t + 1) * kResTile); one block of
// kResBlock threads per tile, one warp per row with the lanes over the row's
// entries and a fixed shuffle tree; the block sums its rows' r^2 and f^2 in
// warp order.  part[2t] = sum r^2, part[2t + 1] = sum f^2 of tile t.  The
// final value adds the tiles' partial sums in tile order.
#pragma once

#include <math.h>
#include <stdint.h>

namespace obk {

constexpr int kResTile = 4096;
constexpr int kResBlock = 256;

// Body of the per-tile kernel: called by all kResBlock threads of block `tile`.
// Column indices are not checked here: every col_idx entry must be in [0, n).
__device__ __forceinline__ void residual_tile_sums(int64_t m, const int64_t* rp, const int32_t* ci,
                                                   const double* v, const double* f, const double* x,
                                                   double* part, int64_t tile)
{
    __shared__ double wr[kResBlock / 32], wf[kResBlock / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t r0 = tile * kResTile, r1 = r0 + kResTile < m ? r0 + kResTile : m;
    double sr = 0.0, sf = 0.0;
    for (int64_t i = r0 + w; i < r1; i += kResBlock / 32) {
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
        for (int k = 0; k < kResBlock / 32; ++k) { a += wr[k]; b += wf[k]; }
        part[2 * tile] = a;  // every tile writes both of its slots: nothing needs clearing first
        part[2 * tile + 1] = b;
    }
}

// The relative residual from the tiles' partial sums (absolute when f = 0).
__device__ __forceinline__ double residual_from_tiles(const double* part, int64_t ntiles)
{
    double a = 0.0, b = 0.0;
    for (int64_t t = 0; t < ntiles; ++t) { a += part[2 * t]; b += part[2 * t + 1]; }
    return b > 0.0 ? sqrt(a) / sqrt(b) : sqrt(a);
}

}  // namespace obk
