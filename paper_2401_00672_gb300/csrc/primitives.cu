// primitives.cu -- building blocks of the setup: exclusive scans, a stable LSD
// radix sort, per-segment sorts (register sorting networks for short segments)
// and the CSR pattern transpose (structurally symmetric fast path or counting
// scatter), plus the host helpers for waits and cooperative grid sizes.
#include "common.cuh"

namespace obk {

namespace {

constexpr int kScanBlock = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanBlock * kScanItems;

// Block-wide exclusive scan of one value per thread (int64).
__device__ int64_t block_exclusive_scan(int64_t v, int64_t* total)
{
    __shared__ int64_t warp_sums[kScanBlock / kWarp];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_sums[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int64_t w = lane < kScanBlock / kWarp ? warp_sums[lane] : 0;
        int64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < kScanBlock / kWarp) warp_sums[lane] = wi - w;
        if (lane == kScanBlock / kWarp - 1) *total = wi;
    }
    __syncthreads();
    int64_t r = inc - v + warp_sums[wid];
    __syncthreads();
    return r;
}

template <class Tin>
__global__ void scan_tile_sums(const Tin* in, int64_t n, int64_t* tile_sums)
{
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)k * kScanBlock + threadIdx.x;
        if (i < n) s += (int64_t)in[i];
    }
    __shared__ int64_t tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// Single-block exclusive scan of the tile sums (any length, sequential tiles).
__global__ void scan_tile_offsets(int64_t* sums, int64_t ntiles)
{
    __shared__ int64_t tot;
    int64_t carry = 0;
    for (int64_t base = 0; base < ntiles; base += kScanBlock) {
        int64_t i = base + threadIdx.x;
        int64_t v = i < ntiles ? sums[i] : 0;
        int64_t ex = block_exclusive_scan(v, &tot);
        if (i < ntiles) sums[i] = ex + carry;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[ntiles] = carry;
}

template <class Tin>
__global__ void scan_tile_apply(const Tin* in, int64_t* out, int64_t n, const int64_t* offs,
                                int64_t ntiles)
{
    // each thread owns kScanItems consecutive elements of the tile
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t loc[kScanItems];
    int64_t s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        loc[k] = i < n ? (int64_t)in[i] : 0;
        s += loc[k];
    }
    __shared__ int64_t tot;
    int64_t ex = block_exclusive_scan(s, &tot) + offs[blockIdx.x];
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        if (i < n) out[i] = ex;
        ex += loc[k];
    }
    if (blockIdx.x == ntiles - 1 && threadIdx.x == 0) out[n] = offs[ntiles];
}

// the whole scan when it fits in one tile: one launch instead of three
template <class Tin>
__global__ void scan_single_tile(const Tin* in, int64_t* out, int64_t n)
{
    int64_t base = (int64_t)threadIdx.x * kScanItems;
    int64_t loc[kScanItems];
    int64_t s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        loc[k] = i < n ? (int64_t)in[i] : 0;
        s += loc[k];
    }
    __shared__ int64_t tot;
    int64_t ex = block_exclusive_scan(s, &tot);
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        if (i < n) out[i] = ex;
        ex += loc[k];
    }
    if (threadIdx.x == 0) out[n] = tot;
}

template <class Tin>
void exclusive_scan_impl(const Tin* in, int64_t* out, int64_t n, cudaStream_t st)
{
    if (n == 0) {
        OBK_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), st));
        return;
    }
    if (n <= kScanTile) {
        scan_single_tile<Tin><<<1, kScanBlock, 0, st>>>(in, out, n);
        OBK_CHECK_LAUNCH();
        return;
    }
    int64_t ntiles = ceil_div(n, kScanTile);
    DBuf<int64_t> sums(ntiles + 1, st);
    scan_tile_sums<Tin><<<(unsigned)ntiles, kScanBlock, 0, st>>>(in, n, sums.p);
    OBK_CHECK_LAUNCH();
    scan_tile_offsets<<<1, kScanBlock, 0, st>>>(sums.p, ntiles);
    OBK_CHECK_LAUNCH();
    scan_tile_apply<Tin><<<(unsigned)ntiles, kScanBlock, 0, st>>>(in, out, n, sums.p, ntiles);
    OBK_CHECK_LAUNCH();
}

// ---- stable LSD radix sort, 8-bit digits ---------------------------------

constexpr int kSortBlock = 256;
constexpr int kSortItems = 16;  // keys per thread per tile (processed in rounds)
constexpr int kSortTile = kSortBlock * kSortItems;
constexpr int kRadix = 256;

__global__ void radix_hist(const uint64_t* keys, int64_t n, int shift, int64_t* hist, int64_t ntiles)
{
    __shared__ unsigned cnt[kRadix];
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) cnt[d] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int k = 0; k < kSortItems; ++k) {
        int64_t i = base + (int64_t)k * kSortBlock + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 0xff], 1u);
    }
    __syncthreads();
    // digit-major layout: hist[d * ntiles + tile]
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) hist[(int64_t)d * ntiles + blockIdx.x] = cnt[d];
}

// Stable scatter: keys of a tile are ranked in input order.  The tile is
// processed in rounds of kSortBlock consecutive keys; within a round a key's
// rank is (keys of the same digit in earlier rounds of this tile) + (same digit
// in earlier warps of this round) + (same digit in earlier lanes of its warp).
__global__ void radix_scatter(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                              uint32_t* vals_out, int64_t n, int shift, const int64_t* offs,
                              int64_t ntiles)
{
    constexpr int kWarps = kSortBlock / kWarp;
    __shared__ int64_t base_off[kRadix];
    __shared__ unsigned warp_cnt[kWarps][kRadix];
    __shared__ unsigned round_tot[kRadix];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x)
        base_off[d] = offs[(int64_t)d * ntiles + blockIdx.x];
    int64_t tile0 = (int64_t)blockIdx.x * kSortTile;
    unsigned lt_mask = (1u << lane) - 1u;
    for (int r = 0; r < kSortItems; ++r) {
        int64_t round0 = tile0 + (int64_t)r * kSortBlock;
        if (round0 >= n) break;  // uniform across the block
        for (int t = threadIdx.x; t < kWarps * kRadix; t += blockDim.x) (&warp_cnt[0][0])[t] = 0;
        __syncthreads();
        int64_t i = round0 + threadIdx.x;
        bool valid = i < n;
        uint64_t key = valid ? keys_in[i] : 0;
        uint32_t val = valid ? vals_in[i] : 0;
        unsigned d = valid ? (unsigned)((key >> shift) & 0xff) : (unsigned)kRadix;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned rank_in_warp = __popc(peers & lt_mask);
        if (valid && rank_in_warp == 0) warp_cnt[wid][d] = __popc(peers);
        __syncthreads();
        for (int dd = threadIdx.x; dd < kRadix; dd += blockDim.x) {
            unsigned run = 0;
            for (int w = 0; w < kWarps; ++w) {
                unsigned c = warp_cnt[w][dd];
                warp_cnt[w][dd] = run;
                run += c;
            }
            round_tot[dd] = run;
        }
        __syncthreads();
        if (valid) {
            int64_t pos = base_off[d] + warp_cnt[wid][d] + rank_in_warp;
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
        for (int dd = threadIdx.x; dd < kRadix; dd += blockDim.x) base_off[dd] += round_tot[dd];
        __syncthreads();
    }
}


// ---- segmented sort of (u32 key, u32 value) by key inside each segment ------
//
// Segments [ptr[s], ptr[s+1]).  Short segments are sorted by one thread in
// registers with Batcher's odd-even merge sort network (8, 16, 32 or 64 inputs,
// padded with the largest value), medium ones by one block with a bitonic
// network in shared memory, and the rare long ones by the global radix sort
// on (segment, key).  Pairs compare as (key, value), which is key order when
// the keys of a segment are distinct.

constexpr int kSegShort = 32;
constexpr int kSegMid = 64;
constexpr int kSegMedium = 2048;

__device__ __forceinline__ void cmp_swap(uint64_t& a, uint64_t& b)
{
    uint64_t lo = a < b ? a : b;
    b = a < b ? b : a;
    a = lo;
}

// Batcher's odd-even merge sort of a[LO, LO + N) (N a power of two), written as
// template recursion so that every index is a compile-time constant and a[]
// stays in registers.  merge<LO, N, R> merges the elements R apart.
template <int W, int LO, int N, int R>
struct OddEvenMerge {
    __device__ __forceinline__ static void run(uint64_t (&a)[W])
    {
        if constexpr (2 * R < N) {
            OddEvenMerge<W, LO, N, 2 * R>::run(a);
            OddEvenMerge<W, LO + R, N, 2 * R>::run(a);
#pragma unroll
            for (int i = LO + R; i + R < LO + N; i += 2 * R) cmp_swap(a[i], a[i + R]);
        } else {
            cmp_swap(a[LO], a[LO + R]);
        }
    }
};

template <int W, int LO, int N>
struct OddEvenSort {
    __device__ __forceinline__ static void run(uint64_t (&a)[W])
    {
        if constexpr (N > 1) {
            OddEvenSort<W, LO, N / 2>::run(a);
            OddEvenSort<W, LO + N / 2, N / 2>::run(a);
            OddEvenMerge<W, LO, N, 1>::run(a);
        }
    }
};

template <int W>
__device__ __forceinline__ void oddeven_sort(uint64_t (&a)[W])
{
    OddEvenSort<W, 0, W>::run(a);
}

template <int W>
__device__ __forceinline__ void sort_segment(int64_t b, int64_t len, uint32_t* keys, uint32_t* vals)
{
    uint64_t a[W];
#pragma unroll
    for (int t = 0; t < W; ++t)
        a[t] = t < len ? ((uint64_t)keys[b + t] << 32) | (uint64_t)vals[b + t] : ~0ull;
    oddeven_sort<W>(a);
#pragma unroll
    for (int t = 0; t < W; ++t)
        if (t < len) {
            keys[b + t] = (uint32_t)(a[t] >> 32);
            vals[b + t] = (uint32_t)a[t];
        }
}

__global__ void segsort_short(const int64_t* ptr, int64_t nseg, uint32_t* keys, uint32_t* vals,
                              int32_t* longs, int32_t* nlong, int32_t* huge, int32_t* nhuge, int32_t* mids,
                              int32_t* nmid)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    int64_t b = ptr[s], e = ptr[s + 1], len = e - b;
    if (len <= 1) return;
    if (len > kSegMedium) { huge[atomicAdd(nhuge, 1)] = (int32_t)s; return; }
    if (len > kSegMid) { longs[atomicAdd(nlong, 1)] = (int32_t)s; return; }
    if (len > kSegShort) { mids[atomicAdd(nmid, 1)] = (int32_t)s; return; }
    if (len <= 8) sort_segment<8>(b, len, keys, vals);
    else if (len <= 16) sort_segment<16>(b, len, keys, vals);
    else sort_segment<32>(b, len, keys, vals);
}

// segments of 33..64 pairs (listed), one thread each
__global__ void segsort_mid(const int64_t* ptr, const int32_t* mids, int32_t nmid, uint32_t* keys, uint32_t* vals)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nmid) return;
    int64_t s = mids[t];
    sort_segment<64>(ptr[s], ptr[s + 1] - ptr[s], keys, vals);
}

__global__ void segsort_medium(const int64_t* ptr, const int32_t* longs, uint32_t* keys, uint32_t* vals)
{
    __shared__ unsigned long long buf[kSegMedium];
    int64_t s = longs[blockIdx.x];
    int64_t b = ptr[s], len = ptr[s + 1] - b;
    int P = 1;
    while (P < len) P <<= 1;
    for (int t = threadIdx.x; t < P; t += blockDim.x)
        buf[t] = t < len ? (((unsigned long long)keys[b + t]) << 32) | vals[b + t] : ~0ull;
    __syncthreads();
    for (int kk = 2; kk <= P; kk <<= 1)
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < P; t += blockDim.x) {
                int o = t ^ j;
                if (o > t) {
                    bool up = (t & kk) == 0;
                    unsigned long long a = buf[t], c = buf[o];
                    if ((a > c) == up) { buf[t] = c; buf[o] = a; }
                }
            }
            __syncthreads();
        }
    for (int t = threadIdx.x; t < len; t += blockDim.x) {
        keys[b + t] = (uint32_t)(buf[t] >> 32);
        vals[b + t] = (uint32_t)buf[t];
    }
}

__global__ void segsort_huge_gather(const int64_t* ptr, const int32_t* huge, const int64_t* hoff,
                                    int32_t nh, const uint32_t* keys, uint64_t* k64, uint32_t* pos)
{
    for (int h = blockIdx.x; h < nh; h += gridDim.x) {
        int64_t b = ptr[huge[h]], len = ptr[huge[h] + 1] - b, o = hoff[h];
        for (int64_t t = threadIdx.x; t < len; t += blockDim.x) {
            k64[o + t] = ((uint64_t)h << 32) | keys[b + t];
            pos[o + t] = (uint32_t)(b + t);
        }
    }
}

__global__ void segsort_huge_scatter(const int64_t* ptr, const int32_t* huge, const int64_t* hoff,
                                     int32_t nh, const uint64_t* k64, const uint32_t* pos,
                                     const uint32_t* vals_src, uint32_t* keys, uint32_t* vals)
{
    for (int h = blockIdx.x; h < nh; h += gridDim.x) {
        int64_t b = ptr[huge[h]], len = ptr[huge[h] + 1] - b, o = hoff[h];
        for (int64_t t = threadIdx.x; t < len; t += blockDim.x) {
            keys[b + t] = (uint32_t)k64[o + t];
            vals[b + t] = vals_src[pos[o + t]];
        }
    }
}

__global__ void segsort_huge_sizes(const int64_t* ptr, const int32_t* huge, int32_t nh, int64_t* sz)
{
    int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h < nh) sz[h] = ptr[huge[h] + 1] - ptr[huge[h]];
}

}  // namespace

void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st)
{
    exclusive_scan_impl<int64_t>(in, out, n, st);
}

void exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t st)
{
    exclusive_scan_impl<int32_t>(in, out, n, st);
}

void radix_sort_pairs(uint64_t* keys, uint32_t* vals, int64_t n, int bits, cudaStream_t st)
{
    if (n <= 1) return;
    int64_t ntiles = ceil_div(n, kSortTile);
    DBuf<uint64_t> k2(n, st);
    DBuf<uint32_t> v2(n, st);
    DBuf<int64_t> hist(kRadix * ntiles + 1, st);
    DBuf<int64_t> offs(kRadix * ntiles + 1, st);
    uint64_t* kin = keys;
    uint32_t* vin = vals;
    uint64_t* kout = k2.p;
    uint32_t* vout = v2.p;
    int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        radix_hist<<<(unsigned)ntiles, kSortBlock, 0, st>>>(kin, n, shift, hist.p, ntiles);
        OBK_CHECK_LAUNCH();
        exclusive_scan_i64(hist.p, offs.p, kRadix * ntiles, st);
        radix_scatter<<<(unsigned)ntiles, kSortBlock, 0, st>>>(kin, vin, kout, vout, n, shift, offs.p,
                                                              ntiles);
        OBK_CHECK_LAUNCH();
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    if (kin != keys) {
        OBK_CUDA(cudaMemcpyAsync(keys, kin, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
        OBK_CUDA(cudaMemcpyAsync(vals, vin, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    }
}

namespace {
struct PinnedSlot {
    void* p = nullptr;
    ~PinnedSlot()
    {
        if (p) cudaFreeHost(p);
    }
};
}  // namespace

void* pinned_scratch()
{
    thread_local PinnedSlot slot;
    if (!slot.p) OBK_CUDA(cudaMallocHost(&slot.p, 64));
    return slot.p;
}

int coop_grid(const void* kernel, int block, size_t smem, int64_t want_blocks)
{
    DevInfo di = dev_info();
    int per_sm = 0;
    OBK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem));
    if (per_sm < 1) throw Error{-5, "kernel cannot be made resident (occupancy 0)"};
    int64_t cap = (int64_t)per_sm * di.sms;
    int64_t g = want_blocks < cap ? want_blocks : cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace obk

namespace obk {

void segmented_sort_u32(const int64_t* ptr, int64_t nseg, uint32_t* keys, uint32_t* vals,
                        cudaStream_t st)
{
    if (nseg <= 0) return;
    DBuf<int32_t> longs(nseg, st), huge(nseg, st), mids(nseg, st), cnt(3, st);
    OBK_CUDA(cudaMemsetAsync(cnt.p, 0, 3 * sizeof(int32_t), st));
    segsort_short<<<(unsigned)ceil_div(nseg, 256), 256, 0, st>>>(ptr, nseg, keys, vals, longs.p, cnt.p,
                                                                 huge.p, cnt.p + 1, mids.p, cnt.p + 2);
    OBK_CHECK_LAUNCH();
    int32_t h_cnt[3];
    OBK_CUDA(cudaMemcpyAsync(h_cnt, cnt.p, sizeof(h_cnt), cudaMemcpyDeviceToHost, st));
    OBK_CUDA(cudaStreamSynchronize(st));
    if (h_cnt[2] > 0) {
        segsort_mid<<<(unsigned)ceil_div(h_cnt[2], 128), 128, 0, st>>>(ptr, mids.p, h_cnt[2], keys, vals);
        OBK_CHECK_LAUNCH();
    }
    if (h_cnt[0] > 0) {
        segsort_medium<<<(unsigned)h_cnt[0], 512, 0, st>>>(ptr, longs.p, keys, vals);
        OBK_CHECK_LAUNCH();
    }
    int32_t nh = h_cnt[1];
    if (nh > 0) {
        DBuf<int64_t> sz(nh, st), hoff(nh + 1, st);
        segsort_huge_sizes<<<(unsigned)ceil_div(nh, 256), 256, 0, st>>>(ptr, huge.p, nh, sz.p);
        OBK_CHECK_LAUNCH();
        exclusive_scan_i64(sz.p, hoff.p, nh, st);
        int64_t tot = read_scalar(hoff.p + nh, st);
        DBuf<uint64_t> k64(tot, st);
        DBuf<uint32_t> pos(tot, st);
        segsort_huge_gather<<<256, 256, 0, st>>>(ptr, huge.p, hoff.p, nh, keys, k64.p, pos.p);
        OBK_CHECK_LAUNCH();
        radix_sort_pairs(k64.p, pos.p, tot, 32 + bits_for((uint64_t)nh), st);
        // the scatter reads values through their source positions: keep a copy
        int64_t nvals = read_scalar(ptr + nseg, st);
        DBuf<uint32_t> vsrc(nvals, st);
        OBK_CUDA(cudaMemcpyAsync(vsrc.p, vals, nvals * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
        segsort_huge_scatter<<<256, 256, 0, st>>>(ptr, huge.p, hoff.p, nh, k64.p, pos.p, vsrc.p, keys,
                                                  vals);
        OBK_CHECK_LAUNCH();
    }
}

namespace {

__global__ void column_counts(const int32_t* ci, int64_t nnz, unsigned* cnt)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt + ci[e], 1u);
}

// one thread per row; a row's entries in batches of kScatterBatch so that
// their atomics are in flight together
constexpr int kScatterBatch = 8;

__global__ void column_scatter(int64_t nrows, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                               const int64_t* __restrict__ cptr, unsigned* __restrict__ cur,
                               uint32_t* __restrict__ trow, uint32_t* __restrict__ tsrc)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nrows;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t e1 = rp[i + 1];
        for (int64_t e0 = rp[i]; e0 < e1; e0 += kScatterBatch) {
            int32_t c[kScatterBatch];
#pragma unroll
            for (int t = 0; t < kScatterBatch; ++t) c[t] = e0 + t < e1 ? ci[e0 + t] : -1;
            unsigned k[kScatterBatch];
#pragma unroll
            for (int t = 0; t < kScatterBatch; ++t) k[t] = c[t] >= 0 ? atomicAdd(cur + c[t], 1u) : 0u;
#pragma unroll
            for (int t = 0; t < kScatterBatch; ++t)
                if (c[t] >= 0) {
                    int64_t slot = cptr[c[t]] + (int64_t)k[t];
                    trow[slot] = (uint32_t)i;
                    tsrc[slot] = (uint32_t)(e0 + t);
                }
        }
    }
}

// Structurally symmetric square pattern: column c lists the same rows as row c
// lists columns, so entry e = (i, c) sits at CSC slot q = rp[c] + (rank of i in
// row c), and the entry at slot q of row c, (c, i), sits at CSC slot e.  The
// pattern is symmetric exactly when every entry above the diagonal (c > i)
// has its mirror (c, i) in row c and there are as many entries below the
// diagonal as above (the mirror map is then a bijection; columns are distinct
// in a row).  So only the entries above the diagonal search for their mirror
// (one binary search, kSymBatch of a row in flight), each search fills both
// slots, and a diagonal entry is its own slot.  Entries above / below the
// diagonal are counted into cnt[0] / cnt[1]; a missing mirror sets *asym and
// the caller falls back to the general path.  With tsrc NULL the kernel only
// tests the pattern.
constexpr int kSymBatch = 4;

__global__ void symmetric_slots(int64_t n, int64_t stride, const int64_t* __restrict__ rp,
                                const int32_t* __restrict__ ci, uint32_t* __restrict__ tsrc, int* asym,
                                unsigned long long* cnt)
{
    unsigned long long above = 0, below = 0;
    bool stop = false;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k * stride < n && !stop;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = k * stride;
        int64_t e1 = rp[i + 1];
        for (int64_t e0 = rp[i]; e0 < e1; e0 += kSymBatch) {
            if (*(volatile int*)asym) {  // already known not to be symmetric
                stop = true;
                break;
            }
            int32_t c[kSymBatch];
            int64_t lo[kSymBatch], hi[kSymBatch];
#pragma unroll
            for (int t = 0; t < kSymBatch; ++t) {
                c[t] = e0 + t < e1 ? ci[e0 + t] : -1;
                lo[t] = 0;
                hi[t] = 0;
                if (c[t] > i) {
                    lo[t] = rp[c[t]];
                    hi[t] = rp[c[t] + 1];
                    ++above;
                } else if (c[t] == i) {
                    if (tsrc) tsrc[e0 + t] = (uint32_t)(e0 + t);
                } else if (c[t] >= 0) {
                    ++below;
                }
            }
            // first position in [lo, hi) whose column is >= i
            int64_t end[kSymBatch];
#pragma unroll
            for (int t = 0; t < kSymBatch; ++t) end[t] = hi[t];
            bool more = true;
            while (more) {
                more = false;
#pragma unroll
                for (int t = 0; t < kSymBatch; ++t)
                    if (lo[t] < hi[t]) {
                        int64_t mid = (lo[t] + hi[t]) >> 1;
                        if ((int64_t)ci[mid] < i) lo[t] = mid + 1;
                        else hi[t] = mid;
                        more = true;
                    }
            }
#pragma unroll
            for (int t = 0; t < kSymBatch; ++t)
                if (c[t] > i) {
                    int64_t q = lo[t];
                    if (q < end[t] && (int64_t)ci[q] == i) {
                        if (tsrc) {
                            tsrc[q] = (uint32_t)(e0 + t);
                            tsrc[e0 + t] = (uint32_t)q;
                        }
                    } else {
                        *asym = 1;
                    }
                }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        above += __shfl_xor_sync(0xffffffffu, above, o);
        below += __shfl_xor_sync(0xffffffffu, below, o);
    }
    if ((threadIdx.x & 31) == 0 && (above | below)) {
        atomicAdd(cnt, above);
        atomicAdd(cnt + 1, below);
    }
}

__global__ void copy_cols_u32(const int32_t* ci, int64_t nnz, uint32_t* out)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = (uint32_t)ci[e];
}

__global__ void widen_counts(const unsigned* cnt, int64_t n, int64_t* out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int64_t)cnt[i];
}

}  // namespace

namespace {
// Structural symmetry test of a square pattern (sorted, distinct columns per
// row); with tsrc non-NULL it also fills the transpose slots of a symmetric
// pattern.  A sample of about 8K rows goes first: most asymmetric patterns fail
// it before the full pass.
bool symmetric_pass(int64_t n, const int64_t* rp, const int32_t* ci, uint32_t* tsrc, cudaStream_t st)
{
    constexpr int kT = 256;
    auto grid = [](int64_t m) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(m, kT), 65535)); };
    DBuf<int> asym(1, st);
    DBuf<unsigned long long> cnt(2, st);
    OBK_CUDA(cudaMemsetAsync(asym.p, 0, sizeof(int), st));
    OBK_CUDA(cudaMemsetAsync(cnt.p, 0, 2 * sizeof(unsigned long long), st));
    int64_t stride = std::max<int64_t>(1, n / 8192);
    if (stride > 1) {
        symmetric_slots<<<grid(ceil_div(n, stride)), kT, 0, st>>>(n, stride, rp, ci, tsrc, asym.p, cnt.p);
        OBK_CHECK_LAUNCH();
        OBK_CUDA(cudaMemsetAsync(cnt.p, 0, 2 * sizeof(unsigned long long), st));
    }
    if (stride == 1 || read_scalar(asym.p, st) == 0) {
        symmetric_slots<<<grid(n), kT, 0, st>>>(n, 1, rp, ci, tsrc, asym.p, cnt.p);
        OBK_CHECK_LAUNCH();
    }
    struct {
        unsigned long long c[2];
        int a;
    } r{};
    OBK_CUDA(cudaMemcpyAsync(&r.c, cnt.p, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    OBK_CUDA(cudaMemcpyAsync(&r.a, asym.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    OBK_CUDA(cudaStreamSynchronize(st));
    return r.a == 0 && r.c[0] == r.c[1];
}
}  // namespace

bool pattern_symmetric(int64_t n, const int64_t* rp, const int32_t* ci, int64_t nnz, cudaStream_t st)
{
    if (nnz == 0) return true;
    return symmetric_pass(n, rp, ci, nullptr, st);
}

void transpose_pattern(int64_t nrows, int64_t ncols, const int64_t* rp, const int32_t* ci, int64_t nnz,
                       DBuf<int64_t>& cptr, DBuf<uint32_t>& trow, DBuf<uint32_t>& tsrc, cudaStream_t st,
                       bool* symmetric, bool need_trow)
{
    if (symmetric) *symmetric = false;
    constexpr int kT = 256;
    auto grid = [](int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kT), 65535)); };
    cptr.alloc(ncols + 1, st);
    trow.alloc(std::max<int64_t>(nnz, 1), st);
    tsrc.alloc(std::max<int64_t>(nnz, 1), st);
    if (nrows == ncols && nnz > 0) {
        // structurally symmetric patterns (the common case for square systems)
        // need no counting or sorting: the transpose has the pattern itself
        if (symmetric_pass(nrows, rp, ci, tsrc.p, st)) {
            OBK_CUDA(cudaMemcpyAsync(cptr.p, rp, (nrows + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
            if (need_trow) {
                copy_cols_u32<<<grid(nnz), kT, 0, st>>>(ci, nnz, trow.p);
                OBK_CHECK_LAUNCH();
            }
            if (symmetric) *symmetric = true;
            return;
        }
    }
    DBuf<unsigned> cnt(std::max<int64_t>(ncols, 1), st);
    DBuf<int64_t> wide(std::max<int64_t>(ncols, 1), st);
    OBK_CUDA(cudaMemsetAsync(cnt.p, 0, std::max<int64_t>(ncols, 1) * sizeof(unsigned), st));
    if (nnz) {
        column_counts<<<grid(nnz), kT, 0, st>>>(ci, nnz, cnt.p);
        OBK_CHECK_LAUNCH();
    }
    widen_counts<<<grid(ncols), kT, 0, st>>>(cnt.p, ncols, wide.p);
    OBK_CHECK_LAUNCH();
    exclusive_scan_i64(wide.p, cptr.p, ncols, st);
    if (nnz) {
        OBK_CUDA(cudaMemsetAsync(cnt.p, 0, std::max<int64_t>(ncols, 1) * sizeof(unsigned), st));
        column_scatter<<<grid(nrows), kT, 0, st>>>(nrows, rp, ci, cptr.p, cnt.p, trow.p, tsrc.p);
        OBK_CHECK_LAUNCH();
        // a column's rows are distinct: sorting them restores row order
        segmented_sort_u32(cptr.p, ncols, trow.p, tsrc.p, st);
    }
}

}  // namespace obk
