// common.cuh -- shared device/host helpers of the OBK-RCM CUDA library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <new>
#include <string>

namespace obk {

// ---- error plumbing ----------------------------------------------------

// Thrown inside the library, converted to an obk_status at the C boundary.
struct Error {
    int status;
    std::string msg;
};

void set_last_error(const std::string& msg);

// Every extern "C" entry point wraps its body in OBK_API_BEGIN / OBK_API_END:
// no exception crosses the C boundary; each becomes an obk_status and a
// message for obk_last_error().
inline int api_fail(const Error& e)
{
    set_last_error(e.msg);
    return e.status;
}
#define OBK_API_BEGIN try {
#define OBK_API_END                                                                          \
    }                                                                                        \
    catch (const ::obk::Error& e) { return (obk_status)::obk::api_fail(e); }                 \
    catch (const std::bad_alloc&) {                                                          \
        return (obk_status)::obk::api_fail(::obk::Error{-2, "host allocation failed"});      \
    }                                                                                        \
    catch (...) { return (obk_status)::obk::api_fail(::obk::Error{-5, "unexpected internal error"}); }

#define OBK_CUDA(call)                                                                 \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            throw ::obk::Error{-5, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
    } while (0)

// Every kernel launch of the library is followed by OBK_CHECK_LAUNCH (or goes
// through OBK_COOP_LAUNCH), which also counts it for obk_kernel_launches().
void count_launch();
#define OBK_CHECK_LAUNCH()              \
    do {                                \
        ::obk::count_launch();          \
        OBK_CUDA(cudaGetLastError());   \
    } while (0)
#define OBK_COOP_LAUNCH(k, g, b, a, s)                                        \
    do {                                                                      \
        ::obk::count_launch();                                                \
        OBK_CUDA(cudaLaunchCooperativeKernel((const void*)(k), g, b, a, 0, s)); \
    } while (0)

constexpr int kWarp = 32;

// Error word written by device code (0 = fine).
enum DevErr : int { kDevOk = 0, kDevTimeout = 1, kDevOverflow = 2 };

// Default bound on device-side spin waits (iterations of a poll loop, each at
// least one L2 round trip): a few seconds at most.
constexpr long long kDefaultSpins = 1LL << 23;

// ---- bounded grid barrier ------------------------------------------------
//
// Barrier for kernels launched cooperatively (all blocks co-resident).  One
// 64-bit counter that only grows: thread 0 of each block adds 1 with an
// acquire-release atomic at GPU scope; the value it gets back tells which
// barrier episode it joined (old / blocks), and it waits with acquire loads
// until the counter reaches the end of that episode.  The release/acquire
// pair makes every block's writes before the barrier visible to every block
// after it.  No reset and no generation word: one atomic per block on the
// critical path.  Every wait is bounded: after `limit` polls the block
// records kDevTimeout in *err and returns false; callers must then leave the
// kernel.
constexpr int kBarrierWords = 64;  // [0..1] the counter; the rest unused padding

struct GridBarrier {
    unsigned int* bar;  // kBarrierWords words, zeroed before the launch (8-byte aligned)
    int* err;
    long long limit;
};

__device__ __forceinline__ unsigned ld_volatile_u32(const unsigned* p)
{
    return *reinterpret_cast<const volatile unsigned*>(p);
}
__device__ __forceinline__ int ld_volatile_i32(const int* p)
{
    return *reinterpret_cast<const volatile int*>(p);
}
__device__ __forceinline__ unsigned atom_add_acq_rel_gpu(unsigned* p, unsigned v)
{
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long atom_add_acq_rel_gpu_u64(unsigned long long* p,
                                                                      unsigned long long v)
{
    unsigned long long old;
    asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}
__device__ __forceinline__ unsigned long long ld_acquire_gpu_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p)
{
    return *reinterpret_cast<const volatile unsigned long long*>(p);
}
__device__ __forceinline__ void st_release_gpu_u64(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" : : "l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ bool grid_sync(const GridBarrier& gb)
{
    __shared__ int s_ok;
    if (gridDim.x * gridDim.y * gridDim.z == 1) {  // a one-block grid needs only the block barrier
        __syncthreads();
        return true;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned long long nb = (unsigned long long)gridDim.x * gridDim.y * gridDim.z;
        unsigned long long* ctr = reinterpret_cast<unsigned long long*>(gb.bar);
        unsigned long long old = atom_add_acq_rel_gpu_u64(ctr, 1ull);
        unsigned long long target = (old / nb + 1ull) * nb;
        long long spins = 0;
        while (ld_acquire_gpu_u64(ctr) < target) {
            if (++spins > gb.limit || ((spins & 63) == 0 && ld_volatile_i32(gb.err) != 0)) {
                atomicCAS(gb.err, 0, (int)kDevTimeout);
                ok = 0;
                break;
            }
            if (spins > 20000) __nanosleep(32);
        }
        if (ld_volatile_i32(gb.err) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---- small helpers -----------------------------------------------------

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

inline int bits_for(uint64_t maxval)
{
    int b = 0;
    while (b < 64 && (maxval >> b) != 0) ++b;
    return b == 0 ? 1 : b;
}

// Device properties of the current device (cached per device).
struct DevInfo {
    int device;
    int sms;
    size_t l2_bytes;
    size_t smem_optin;
};
DevInfo dev_info();

// Library-owned stream-ordered memory pool of the current device.  Freed
// blocks stay in the pool (no release threshold), so the many temporary
// buffers of setup and solve are served without remapping device memory.
cudaMemPool_t lib_pool();

// Stream-ordered device buffer (pool allocation / cudaFreeAsync).
template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    cudaStream_t s = nullptr;
    DBuf() = default;
    DBuf(size_t count, cudaStream_t st) { alloc(count, st); }
    void alloc(size_t count, cudaStream_t st)
    {
        release();
        s = st;
        n = count;
        if (count) {
            cudaError_t e = cudaMallocFromPoolAsync((void**)&p, count * sizeof(T), lib_pool(), st);
            if (e != cudaSuccess) {
                p = nullptr;
                (void)cudaGetLastError();
                throw Error{-2, "device allocation of " + std::to_string(count * sizeof(T)) +
                                    " bytes failed: " + cudaGetErrorString(e)};
            }
        }
    }
    void release()
    {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
        n = 0;
    }
    ~DBuf() { release(); }
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr; o.n = 0; }
    DBuf& operator=(DBuf&& o) noexcept
    {
        if (this != &o) { release(); p = o.p; n = o.n; s = o.s; o.p = nullptr; o.n = 0; }
        return *this;
    }
    size_t bytes() const { return n * sizeof(T); }
};

// ---- primitives (primitives.cu) -----------------------------------------

// out[i] = sum_{k<i} in[k] for i in [0, n]; out has n+1 entries (out[n] = total).
void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st);
void exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t st);

// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of the
// key.  keys/vals are sorted in place (scratch allocated internally).
void radix_sort_pairs(uint64_t* keys, uint32_t* vals, int64_t n, int bits, cudaStream_t st);

// A small pinned host buffer of the calling thread (allocated on first use,
// held until the thread exits): device-to-host reads of single values into
// pageable memory would be staged through the driver, which serialises them
// with the other threads' copies.
void* pinned_scratch();

// Read one value back (synchronises the stream).
template <class T>
T read_scalar(const T* dptr, cudaStream_t st)
{
    static_assert(sizeof(T) <= 64, "read_scalar reads small values");
    T* v = static_cast<T*>(pinned_scratch());
    OBK_CUDA(cudaMemcpyAsync(v, dptr, sizeof(T), cudaMemcpyDeviceToHost, st));
    OBK_CUDA(cudaStreamSynchronize(st));
    return *v;
}

// Cooperative launch helper: grid = min(want, co-resident capacity).
int coop_grid(const void* kernel, int block, size_t smem, int64_t want_blocks);

}  // namespace obk

namespace obk {
// Sort (key, value) pairs by key inside each segment [ptr[s], ptr[s+1]).
// Keys within a segment should be distinct for a deterministic result.
void segmented_sort_u32(const int64_t* ptr, int64_t nseg, uint32_t* keys, uint32_t* vals,
                        cudaStream_t st);
// true when the square pattern (sorted, distinct columns per row) lists (c, i)
// for every entry (i, c)
bool pattern_symmetric(int64_t n, const int64_t* rp, const int32_t* ci, int64_t nnz, cudaStream_t st);
// Transpose of a CSR pattern (nrows x ncols, column indices of each row
// distinct): column pointers cptr (ncols + 1) and, per column in ascending
// row order, the row (trow) and the source entry index (tsrc) of each entry.
// A structurally symmetric square pattern sets *symmetric (when given); its
// trow equals ci and is filled only when need_trow.
void transpose_pattern(int64_t nrows, int64_t ncols, const int64_t* rp, const int32_t* ci, int64_t nnz,
                       DBuf<int64_t>& cptr, DBuf<uint32_t>& trow, DBuf<uint32_t>& tsrc, cudaStream_t st,
                       bool* symmetric = nullptr, bool need_trow = true);
}  // namespace obk
