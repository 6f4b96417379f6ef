// capi.cu -- the C ABI declared in include/obk.h: handles, solves, setup
// queries and device plumbing (extension to a square system, permutation of
// the right-hand side, un-permutation of the result).
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/obk.h"
#include "batch.cuh"
#include "common.cuh"
#include "kernels.cuh"
#include "residual.cuh"

namespace obk {

static thread_local std::string g_last_error;
void set_last_error(const std::string& msg) { g_last_error = msg; }

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

cudaMemPool_t lib_pool()
{
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    OBK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) throw Error{-5, "device index out of range"};
    std::lock_guard<std::mutex> lk(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        OBK_CUDA(cudaMemPoolCreate(&pools[dev], &props));
        uint64_t keep = UINT64_MAX;
        OBK_CUDA(cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep));
        // memory freed on one stream is not handed to another stream by
        // making it wait for the first: concurrent requests stay independent
        int no = 0;
        OBK_CUDA(cudaMemPoolSetAttribute(pools[dev], cudaMemPoolReuseAllowInternalDependencies, &no));
    }
    return pools[dev];
}

DevInfo dev_info()
{
    static std::mutex mu;
    static std::vector<DevInfo> cache;
    int dev = 0;
    OBK_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    for (auto& d : cache)
        if (d.device == dev) return d;
    DevInfo d{};
    d.device = dev;
    int v = 0;
    OBK_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
    d.sms = v;
    OBK_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, dev));
    d.l2_bytes = (size_t)v;
    OBK_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    d.smem_optin = (size_t)v;
    cache.push_back(d);
    return d;
}

namespace {

constexpr int kBlock = 256;
inline unsigned grid_for(int64_t n) { return (unsigned)std::min<int64_t>(ceil_div(n, kBlock) + 1, 65535); }

#define GRID_STRIDE(i, n)                                                              \
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); \
         i += (int64_t)gridDim.x * blockDim.x)

__global__ void extend_rowptr(int64_t m, int64_t N, int64_t nnz, int64_t* rp)
{
    GRID_STRIDE(k, N - m) rp[m + 1 + k] = nnz;
}

__global__ void check_rowptr_ends(const int64_t* rp, int64_t m, int64_t nnz, int* bad)
{
    if (threadIdx.x == 0 && blockIdx.x == 0 && (rp[0] != 0 || rp[m] != nnz)) atomicOr(bad, 16);
}

__global__ void check_finite(const double* a, int64_t n, int* bad)
{
    GRID_STRIDE(i, n) if (!isfinite(a[i])) atomicOr(bad, 32);
}

__global__ void values_finite(const double* v, int64_t nnz, int* bad)
{
    GRID_STRIDE(k, nnz) if (!isfinite(v[k])) atomicOr(bad, 8);
}

// The values of a host CSR are first needed by the permutation, after the
// reordering, which reads only the pattern: for a large matrix in pinned host
// memory (a copy from pageable memory is staged by the driver and gains
// nothing) their copy runs on a second stream of the calling thread beside
// the pattern's validation and RCM.  Until the stream that owns the buffer has
// waited for that copy, the buffer must not go back to the pool and the
// caller's host array must stay untouched, so every exit waits.
constexpr int64_t kOverlapValues = int64_t(1) << 20;  // entries

bool pinned_host(const void* p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// the calling thread's copy stream on the current device (created on first
// use, kept for the thread's lifetime)
cudaStream_t copy_stream()
{
    constexpr int kMaxDev = 64;
    thread_local cudaStream_t streams[kMaxDev] = {};
    int dev = 0;
    OBK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDev) throw Error{-5, "device index out of range"};
    if (!streams[dev]) OBK_CUDA(cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking));
    return streams[dev];
}

struct ValueUpload {
    cudaStream_t st2 = nullptr;
    cudaEvent_t ready = nullptr;
    cudaStream_t owner = nullptr;
    bool pending = false;
    void start(double* dst, const double* src, int64_t n, cudaStream_t st)
    {
        owner = st;
        st2 = copy_stream();
        OBK_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
        OBK_CUDA(cudaEventRecord(ready, st));  // dst is allocated in st's order
        OBK_CUDA(cudaStreamWaitEvent(st2, ready, 0));
        pending = true;
        OBK_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, st2));
        OBK_CUDA(cudaEventRecord(ready, st2));
    }
    // later work on the owner stream sees the values
    void join()
    {
        if (!pending) return;
        OBK_CUDA(cudaStreamWaitEvent(owner, ready, 0));
        pending = false;
    }
    ~ValueUpload()
    {
        if (pending) {
            cudaEventSynchronize(ready);
            cudaStreamWaitEvent(owner, ready, 0);
        }
        if (ready) cudaEventDestroy(ready);
    }
};

__global__ void gather_gm(int64_t Ngm, const int32_t* src, const double* f, int64_t m, double* out)
{
    GRID_STRIDE(k, Ngm)
    {
        int32_t o = src[k];
        out[k] = o < m ? f[o] : 0.0;
    }
}

__global__ void permute_x0(int64_t N, const int32_t* perm, const double* x0, int64_t n, double* x)
{
    GRID_STRIDE(k, N)
    {
        int32_t o = perm[k];
        x[k] = (x0 && o < n) ? x0[o] : 0.0;
    }
}

__global__ void unpermute_x(int64_t N, const int32_t* perm, const double* x, int64_t n, double* out)
{
    GRID_STRIDE(k, N)
    {
        int32_t o = perm[k];
        if (o < n) out[o] = x[k];
    }
}

__global__ void compose_src(int64_t Ngm, const int32_t* grp_row, const int32_t* perm, int32_t* src)
{
    GRID_STRIDE(k, Ngm) src[k] = perm[grp_row[k]];
}

__global__ void zero_row_flags(int64_t N, const int32_t* group_of, int32_t* flag)
{
    GRID_STRIDE(k, N) flag[k] = group_of[k] < 0 ? 1 : 0;
}

__global__ void zero_row_list(int64_t N, const int32_t* flag, const int64_t* scan, const int32_t* perm,
                              int32_t* out)
{
    GRID_STRIDE(k, N) if (flag[k]) out[scan[k]] = perm[k];
}

// deterministic sum of squares: fixed grid, fixed per-thread order, ordered final pass
constexpr int kRedBlocks = 256;
__global__ void sumsq_partial(const double* a, const int32_t* idx, int64_t n, int64_t m, double* part)
{
    __shared__ double ws[kBlock / 32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = idx ? idx[i] : i;
        double v = j < m ? a[j] : 0.0;
        s = fma(v, v, s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kBlock / 32; ++k) t += ws[k];
        part[blockIdx.x] = t;
    }
}

__global__ void sumsq_final(const double* part, double* out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kRedBlocks; ++k) t += part[k];
        *out = t;
    }
}

// sum of squares into *out (device), queued on st without waiting
void sum_squares_to(const double* a, const int32_t* idx, int64_t n, int64_t m, double* out, cudaStream_t st)
{
    if (n <= 0) {
        OBK_CUDA(cudaMemsetAsync(out, 0, sizeof(double), st));
        return;
    }
    DBuf<double> part(kRedBlocks, st);
    sumsq_partial<<<kRedBlocks, kBlock, 0, st>>>(a, idx, n, m, part.p);
    OBK_CHECK_LAUNCH();
    sumsq_final<<<1, 32, 0, st>>>(part.p, out);
    OBK_CHECK_LAUNCH();
}


// ---- residual check with per-tile partial sums (residual.cuh) -------------
__global__ void residual_tiles(int64_t m, const int64_t* rp, const int32_t* ci, const double* v, const double* f,
                               const double* x, double* part)
{
    residual_tile_sums(m, rp, ci, v, f, x, part, blockIdx.x);
}

__global__ void residual_final(const double* part, int64_t ntiles, double* out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *out = residual_from_tiles(part, ntiles);
}

bool is_device_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Copy n elements into a device buffer, from host or device memory.
template <class T>
void to_device(T* dst, const T* src, int64_t n, bool src_dev, cudaStream_t st)
{
    if (n <= 0) return;
    OBK_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(T), src_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             st));
}

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t s;
    explicit Timer(cudaStream_t st) : s(st)
    {
        OBK_CUDA(cudaEventCreate(&a));
        OBK_CUDA(cudaEventCreate(&b));
        OBK_CUDA(cudaEventRecord(a, s));
    }
    double stop_ms()
    {
        float ms = 0.f;
        OBK_CUDA(cudaEventRecord(b, s));
        OBK_CUDA(cudaEventSynchronize(b));
        OBK_CUDA(cudaEventElapsedTime(&ms, a, b));
        return ms;
    }
    ~Timer()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

}  // namespace
}  // namespace obk

using namespace obk;

struct obk_handle {
    int device = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int64_t m = 0, n = 0, N = 0, nnz = 0;
    double thr = 0.1;
    DBuf<int32_t> perm;      // N
    DBuf<int32_t> src_gm;    // Ngm: extended original index of each group-major row
    DBuf<int32_t> zero_src;  // extended original indices of all-zero rows
    int64_t n_zero = 0;
    DBuf<int> err;
    SweepLayout L;
    obk_info info{};
    RcmStats rcm{};
    TuneChoice tuned[2];        // per precision, chosen by obk_autotune (sub = 0: not tuned)
    double stage_ms[16] = {};    // obk_create stages (see obk_get_setup_profile)
    int n_stage = 0;
    // A~ in RCM order (rows and columns) for the block form, with its column
    // lists built on the first obk_solve_blocks
    DBuf<int64_t> at_rp;
    DBuf<int32_t> at_ci;
    DBuf<double> at_v;
    bool has_at_cols = false;
    DBuf<int64_t> at_cptr;
    DBuf<int32_t> at_crow;
    DBuf<double> at_cval;
};

namespace {
// Process-wide autotuning table: (device, log2 size class, mean row length
// rounded, log2 bandwidth class after RCM, precision) -> setting.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, TuneChoice> g_tune;

std::tuple<int, int, int, int, int> tune_key(const obk_handle* h, int precision)
{
    int szc = 0;
    while ((int64_t(1) << szc) < h->L.Ngm) ++szc;
    int avg = h->L.Ngm ? (int)((double)h->L.nnz_gm / (double)h->L.Ngm + 0.5) : 0;
    int bwc = bits_for((uint64_t)std::max<int64_t>(h->info.bandwidth_after, 0));
    return {h->device, szc, avg, bwc, precision};
}

// The tuned setting of h (or of its shape), or all zeros (the fixed rules).
TuneChoice tuned_or_rule(const obk_handle* h, int precision)
{
    if (h->tuned[precision].sub) return h->tuned[precision];
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(tune_key(h, precision));
    if (it != g_tune.end()) return it->second;
    return TuneChoice{};
}
}  // namespace

// OBK_API_BEGIN / OBK_API_END (common.cuh) turn exceptions into statuses at the C boundary.

extern "C" {

const char* obk_last_error(void) { return g_last_error.c_str(); }
const char* obk_version(void) { return "obk-gb300 0.1 (sm_103a)"; }
int64_t obk_kernel_launches(void) { return (int64_t)g_launches.load(); }

obk_status obk_create_on_stream(const obk_csr* A, int64_t m, int64_t n, double thr, void* stream,
                                obk_handle** out)
{
    OBK_API_BEGIN
    set_last_error("");
    if (!out) throw Error{-1, "out is NULL"};
    *out = nullptr;
    if (!A || m <= 0 || n <= 0) throw Error{-1, "m and n must be positive and A non-NULL"};
    if (!(thr > 0.0 && thr <= 1.0)) throw Error{-1, "cos_threshold must lie in (0, 1]"};
    if (A->nnz < 0 || (A->nnz > 0 && (!A->col_idx || !A->val)) || !A->row_ptr)
        throw Error{-1, "malformed CSR arguments"};
    if (std::max(m, n) >= (int64_t)INT32_MAX || A->nnz >= (int64_t)UINT32_MAX)
        throw Error{-1, "dimensions exceed the 32-bit index range"};
    obk_handle* h = new obk_handle();
    try {
        OBK_CUDA(cudaGetDevice(&h->device));
        if (stream) {
            h->st = (cudaStream_t)stream;
        } else {
            OBK_CUDA(cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking));
            h->own_stream = true;
        }
        cudaStream_t st = h->st;
        Timer tm(st);
        StageClock clock;
        clock.mark(st);
        h->m = m;
        h->n = n;
        h->N = std::max(m, n);
        h->nnz = A->nnz;
        h->thr = thr;
        int64_t N = h->N, nnz = A->nnz;
        h->err.alloc(1, st);
        OBK_CUDA(cudaMemsetAsync(h->err.p, 0, sizeof(int), st));
        // A on the device with the extended row pointer (Algorithms 5-6); column
        // indices and values already in device memory are read in place (they
        // are only read, and only during this call)
        bool dev = A->device_ptrs != 0;
        DBuf<int64_t> rp(N + 1, st);
        DBuf<int32_t> ci_copy;
        DBuf<double> v_copy;
        to_device(rp.p, A->row_ptr, m + 1, dev, st);
        const int32_t* ci_p = A->col_idx;
        const double* v_p = A->val;
        ValueUpload vup;  // declared after v_copy: ends before it is freed
        if (!dev || nnz == 0) {
            ci_copy.alloc(std::max<int64_t>(nnz, 1), st);
            v_copy.alloc(std::max<int64_t>(nnz, 1), st);
            to_device(ci_copy.p, A->col_idx, nnz, dev, st);
            if (!dev && nnz >= kOverlapValues && pinned_host(A->val)) vup.start(v_copy.p, A->val, nnz, st);
            else to_device(v_copy.p, A->val, nnz, dev, st);
            ci_p = ci_copy.p;
            v_p = v_copy.p;
        }
        DBuf<int> bad(1, st);
        validate_csr(m, n, rp.p, ci_p, vup.pending ? nullptr : v_p, nnz, bad.p, st);
        check_rowptr_ends<<<1, 32, 0, st>>>(rp.p, m, nnz, bad.p);
        OBK_CHECK_LAUNCH();
        int b = read_scalar(bad.p, st);
        if (b) throw Error{-1, "malformed CSR (code " + std::to_string(b) +
                                   ": 1 row_ptr, 2 column range, 4 unsorted/duplicate, 8 non-finite, "
                                   "16 row_ptr ends)"};
        if (N > m) {
            extend_rowptr<<<grid_for(N - m), kBlock, 0, st>>>(m, N, nnz, rp.p);
            OBK_CHECK_LAUNCH();
        }
        clock.mark(st);  // upload, validation, extension
        h->info.bandwidth_before = half_bandwidth(N, rp.p, ci_p, nnz, st);
        clock.mark(st);  // bandwidth of the input
        // Reverse Cuthill-McKee (Section 3.2) and A~ = P A^ P^T (Eq. 3.1)
        h->perm.alloc(N, st);
        rcm_reorder(N, rp.p, ci_p, nnz, h->perm.p, kDefaultSpins, h->err.p, &h->rcm, st, &clock);
        clock.mark(st);  // Cuthill-McKee order, reversed
        if (vup.pending) {  // the values, copied meanwhile, must be finite
            vup.join();
            OBK_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
            values_finite<<<grid_for(nnz), kBlock, 0, st>>>(v_p, nnz, bad.p);
            OBK_CHECK_LAUNCH();
            if (read_scalar(bad.p, st)) throw Error{-1, "malformed CSR (code 8: non-finite value)"};
        }
        DBuf<int32_t> iperm(N, st);
        DBuf<int64_t> rpt(N + 1, st);
        DBuf<int32_t> cit(std::max<int64_t>(nnz, 1), st);
        DBuf<double> vt(std::max<int64_t>(nnz, 1), st);
        permute_csr(N, rp.p, ci_p, v_p, nnz, h->perm.p, iperm.p, rpt.p, cit.p, vt.p, st);
        rp.release();
        ci_copy.release();
        v_copy.release();
        h->info.bandwidth_after = half_bandwidth(N, rpt.p, cit.p, nnz, st);
        clock.mark(st);  // permutation and its bandwidth
        // norms, groups and sweep layout (Section 3.3)
        group_build(N, rpt.p, cit.p, vt.p, nnz, thr, kDefaultSpins, h->err.p, h->L, true, st, &clock);
        h->info.groups = h->L.G;
        h->info.n_conflicts = h->L.n_conflicts;
        h->src_gm.alloc(std::max<int64_t>(h->L.Ngm, 1), st);
        if (h->L.Ngm) {
            compose_src<<<grid_for(h->L.Ngm), kBlock, 0, st>>>(h->L.Ngm, h->L.grp_row.p, h->perm.p, h->src_gm.p);
            OBK_CHECK_LAUNCH();
        }
        h->at_rp = std::move(rpt);
        h->at_ci = std::move(cit);
        h->at_v = std::move(vt);
        DBuf<int32_t> zf(N, st);
        DBuf<int64_t> zs(N + 1, st);
        zero_row_flags<<<grid_for(N), kBlock, 0, st>>>(N, h->L.group_of.p, zf.p);
        OBK_CHECK_LAUNCH();
        exclusive_scan_i32_to_i64(zf.p, zs.p, N, st);
        h->n_zero = read_scalar(zs.p + N, st);
        h->zero_src.alloc(std::max<int64_t>(h->n_zero, 1), st);
        zero_row_list<<<grid_for(N), kBlock, 0, st>>>(N, zf.p, zs.p, h->perm.p, h->zero_src.p);
        OBK_CHECK_LAUNCH();
        clock.mark(st);  // group bookkeeping
        h->n_stage = clock.read(h->stage_ms, 16);
        h->info.setup_ms = tm.stop_ms();
        OBK_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
        obk_destroy(h);
        throw;
    }
    *out = h;
    return OBK_OK;
    OBK_API_END
}

obk_status obk_create(const obk_csr* A, int64_t m, int64_t n, double thr, obk_handle** out)
{
    return obk_create_on_stream(A, m, n, thr, nullptr, out);
}

obk_status obk_solve_ex(obk_handle* h, const obk_opts* opts, const double* f, const double* x0, double tol,
                        int64_t maxit, double* x_out, obk_info* info)
{
    OBK_API_BEGIN
    set_last_error("");
    if (!h || !f || !x_out) throw Error{-1, "handle, f and x_out must be non-NULL"};
    if (!(tol > 0.0) || maxit < 1) throw Error{-1, "tol must be > 0 and maxit >= 1"};
    obk_opts o{};
    if (opts) o = *opts;
    if (o.precision != 0 && o.precision != 1) throw Error{-1, "precision must be 0 or 1"};
    if (o.check_every < -1 || o.inner_sweeps < 0 || o.max_outer < 0 || o.timeout_spins < 0)
        throw Error{-1, "negative option"};
    if (o.pinv_iters < 0) throw Error{-1, "pinv_iters must be >= 0"};
    if (o.sync_mode < 0 || o.sync_mode > 2) throw Error{-1, "sync_mode must be 0, 1 or 2"};
    if (o.staging < 0 || o.staging > 2) throw Error{-1, "staging must be 0, 1 or 2"};
    if (o.block_threads != 0 && o.block_threads != 512 && o.block_threads != 1024)
        throw Error{-1, "block_threads must be 0, 512 or 1024"};
    if (o.reserved != 0) throw Error{-1, "reserved option field must be 0"};
    if (o.rows_per_warp != 0 && o.rows_per_warp != 1 && o.rows_per_warp != 2 && o.rows_per_warp != 4 &&
        o.rows_per_warp != 8 && o.rows_per_warp != 16 && o.rows_per_warp != 32)
        throw Error{-1, "rows_per_warp must be 0, 1, 2, 4, 8, 16 or 32"};
    OBK_CUDA(cudaSetDevice(h->device));
    cudaStream_t st = h->st;
    int64_t m = h->m, n = h->n, N = h->N;
    Timer tm(st);
    bool fdev = is_device_ptr(f), xdev = x0 && is_device_ptr(x0), odev = is_device_ptr(x_out);
    DBuf<double> fd(m, st), x0d, xt(N, st), fgm(std::max<int64_t>(h->L.Ngm, 1), st);
    to_device(fd.p, f, m, fdev, st);
    DBuf<int> bad(1, st);
    OBK_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
    check_finite<<<grid_for(m), kBlock, 0, st>>>(fd.p, m, bad.p);
    OBK_CHECK_LAUNCH();
    if (x0) {
        x0d.alloc(n, st);
        to_device(x0d.p, x0, n, xdev, st);
        check_finite<<<grid_for(n), kBlock, 0, st>>>(x0d.p, n, bad.p);
        OBK_CHECK_LAUNCH();
    }
    // x~0 = P x^0, f in group-major order, ||f||^2 and the all-zero rows' share;
    // the finiteness flag and the two sums come back in one read
    permute_x0<<<grid_for(N), kBlock, 0, st>>>(N, h->perm.p, x0 ? x0d.p : nullptr, n, xt.p);
    OBK_CHECK_LAUNCH();
    if (h->L.Ngm) {
        gather_gm<<<grid_for(h->L.Ngm), kBlock, 0, st>>>(h->L.Ngm, h->src_gm.p, fd.p, m, fgm.p);
        OBK_CHECK_LAUNCH();
    }
    DBuf<double> sums(2, st);
    sum_squares_to(fd.p, nullptr, m, m, sums.p, st);
    sum_squares_to(fd.p, h->zero_src.p, h->n_zero, m, sums.p + 1, st);
    double fnorm2 = 0.0, zero_f2 = 0.0;
    {
        char* hs = static_cast<char*>(pinned_scratch());
        OBK_CUDA(cudaMemcpyAsync(hs, sums.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        OBK_CUDA(cudaMemcpyAsync(hs + 2 * sizeof(double), bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        OBK_CUDA(cudaStreamSynchronize(st));
        int b = 0;
        std::memcpy(&fnorm2, hs, sizeof(double));
        std::memcpy(&zero_f2, hs + sizeof(double), sizeof(double));
        std::memcpy(&b, hs + 2 * sizeof(double), sizeof(int));
        if (b) throw Error{-1, "f or x0 holds NaN or Inf"};
    }
    SolveArgs a;
    a.precision = o.precision;
    a.check_every = o.check_every == 0 ? 1 : o.check_every;
    a.inner_sweeps = o.inner_sweeps;
    a.max_outer = o.max_outer > 0 ? o.max_outer : 100;
    a.stagnation = o.stagnation;
    a.tol = tol;
    a.maxit = maxit;
    a.spin_limit = o.timeout_spins > 0 ? o.timeout_spins : kDefaultSpins;
    TuneChoice tc = tuned_or_rule(h, o.precision);
    a.sub = o.rows_per_warp > 0 ? 32 / o.rows_per_warp : tc.sub;
    if (a.sub == 0) a.sub = choose_sub(h->L.Ngm ? (double)h->L.nnz_gm / (double)h->L.Ngm : 1.0);
    if (a.sub > 1) ensure_gm_csr(h->L, st);  // the sub-warp sweeps read the group-major rows
    a.pinv_iters = o.precision == 0 ? o.pinv_iters : 0;
    a.sync_mode = o.sync_mode != 0 ? o.sync_mode : (tc.sync != 0 ? tc.sync : default_sync_mode(h->L));
    a.staging = o.staging != 0 ? o.staging : (tc.staging != 0 ? tc.staging : 2);
    a.block = o.block_threads != 0 ? o.block_threads : (tc.block != 0 ? tc.block : (a.sync_mode == 2 ? 1024 : 512));
    if (a.pinv_iters > 0 && !h->L.has_gram) build_group_gram(h->L, h->err.p, st);
    SolveResult r = run_solve(h->L, fgm.p, fnorm2, zero_f2, xt.p, a, h->err.p, st);
    // x = P^T x~, then x^(1:n)
    double* xo = x_out;
    DBuf<double> xtmp;
    if (!odev) {
        xtmp.alloc(n, st);
        xo = xtmp.p;
    }
    unpermute_x<<<grid_for(N), kBlock, 0, st>>>(N, h->perm.p, xt.p, n, xo);
    OBK_CHECK_LAUNCH();
    if (!odev) OBK_CUDA(cudaMemcpyAsync(x_out, xo, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    double ms = tm.stop_ms();
    OBK_CUDA(cudaStreamSynchronize(st));
    h->info.sweeps = r.sweeps;
    h->info.rel_res = r.rel_res;
    h->info.solve_ms = ms;
    h->info.outer_iters = r.outer;
    h->info.sweep_ms = r.sweep_ms;
    h->info.status = r.status;
    if (info) *info = h->info;
    return r.status == 0 ? OBK_OK : OBK_NOT_CONVERGED;
    OBK_API_END
}

obk_status obk_solve(obk_handle* h, const double* f, const double* x0, double tol, int64_t maxit, double* x_out,
                     obk_info* info)
{
    return obk_solve_ex(h, nullptr, f, x0, tol, maxit, x_out, info);
}

obk_status obk_solve_blocks(obk_handle* h, obk_block_opts* bo, const double* f, const double* x0, double tol,
                            int64_t maxit, double* x_out, obk_info* info)
{
    OBK_API_BEGIN
    set_last_error("");
    if (!h || !bo || !f || !x_out) throw Error{-1, "handle, options, f and x_out must be non-NULL"};
    if (!(tol > 0.0) || maxit < 1) throw Error{-1, "tol must be > 0 and maxit >= 1"};
    if (bo->k < 1 || bo->k > h->N) throw Error{-1, "k must be in [1, N]"};
    if (bo->inner_max < 0 || bo->thr < 0.0 || bo->thr > 1.0 || bo->inner_tol < 0.0)
        throw Error{-1, "inner_max, thr or inner_tol out of range"};
    OBK_CUDA(cudaSetDevice(h->device));
    cudaStream_t st = h->st;
    int64_t m = h->m, n = h->n, N = h->N;
    Timer tm(st);
    if (!h->has_at_cols) {
        DBuf<int64_t> pos_of;
        build_csc(N, N, h->at_rp.p, h->at_ci.p, h->at_v.p, h->nnz, h->at_cptr, h->at_crow, h->at_cval, pos_of, st);
        h->has_at_cols = true;
    }
    bool fdev = is_device_ptr(f), xdev = x0 && is_device_ptr(x0), odev = is_device_ptr(x_out);
    DBuf<double> fd(m, st), x0d, xt(N, st), ft(N, st);
    to_device(fd.p, f, m, fdev, st);
    DBuf<int> bad(1, st);
    OBK_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
    check_finite<<<grid_for(m), kBlock, 0, st>>>(fd.p, m, bad.p);
    OBK_CHECK_LAUNCH();
    if (x0) {
        x0d.alloc(n, st);
        to_device(x0d.p, x0, n, xdev, st);
        check_finite<<<grid_for(n), kBlock, 0, st>>>(x0d.p, n, bad.p);
        OBK_CHECK_LAUNCH();
    }
    if (read_scalar(bad.p, st)) throw Error{-1, "f or x0 holds NaN or Inf"};
    // f~ = P f^ and x~0 = P x^0 (Eq. 3.1), the extension's appended entries 0
    permute_x0<<<grid_for(N), kBlock, 0, st>>>(N, h->perm.p, fd.p, m, ft.p);
    OBK_CHECK_LAUNCH();
    permute_x0<<<grid_for(N), kBlock, 0, st>>>(N, h->perm.p, x0 ? x0d.p : nullptr, n, xt.p);
    OBK_CHECK_LAUNCH();
    BlockArgs a;
    a.k = bo->k;
    a.thr = bo->thr > 0.0 ? bo->thr : h->thr;
    a.inner_max = bo->inner_max > 0 ? bo->inner_max : 500;
    a.inner_tol = bo->inner_tol > 0.0 ? bo->inner_tol : 1e-13;
    a.tol = tol;
    a.maxit = maxit;
    a.spin_limit = kDefaultSpins;
    BlockResult r = run_blocks(N, h->at_rp.p, h->at_ci.p, h->at_v.p, h->at_cptr.p, h->at_crow.p, h->at_cval.p, ft.p,
                               xt.p, a, h->err.p, st);
    double* xo = x_out;
    DBuf<double> xtmp;
    if (!odev) {
        xtmp.alloc(n, st);
        xo = xtmp.p;
    }
    unpermute_x<<<grid_for(N), kBlock, 0, st>>>(N, h->perm.p, xt.p, n, xo);
    OBK_CHECK_LAUNCH();
    if (!odev) OBK_CUDA(cudaMemcpyAsync(x_out, xo, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    double ms = tm.stop_ms();
    OBK_CUDA(cudaStreamSynchronize(st));
    bo->n_pairs = r.n_pairs;
    bo->n_nclass = r.n_nclass;
    bo->cgls_steps = r.cgls_steps;
    obk_info inf = h->info;
    inf.sweeps = r.iters;
    inf.rel_res = r.rel_res;
    inf.solve_ms = ms;
    inf.outer_iters = 0;
    inf.sweep_ms = 0.0;
    inf.status = r.status;
    if (info) *info = inf;
    return r.status == 0 ? OBK_OK : OBK_NOT_CONVERGED;
    OBK_API_END
}

obk_status obk_select_threshold(const obk_csr* A, int64_t m, int64_t n, const double* f, const double* thr_cand,
                                int32_t n_cand, int32_t probe_sweeps, double tol, double* out_thr, obk_handle** out,
                                obk_thr_probe* probes)
{
    OBK_API_BEGIN
    set_last_error("");
    if (out) *out = nullptr;
    if (!A || !f || !thr_cand || !out_thr || n_cand < 1 || probe_sweeps < 1 || !(tol > 0.0))
        throw Error{-1, "NULL argument, n_cand < 1, probe_sweeps < 1 or tol <= 0"};
    for (int32_t k = 0; k < n_cand; ++k)
        if (!(thr_cand[k] > 0.0 && thr_cand[k] <= 1.0)) throw Error{-1, "every candidate must lie in (0, 1]"};
    obk_handle* best = nullptr;
    double best_ms = 0.0;
    int32_t best_k = -1;
    std::vector<double> x;
    try {
        for (int32_t k = 0; k < n_cand; ++k) {
            obk_handle* h = nullptr;
            obk_status rc = obk_create(A, m, n, thr_cand[k], &h);
            if (rc != OBK_OK) throw Error{(int)rc, obk_last_error()};
            x.assign((size_t)std::max<int64_t>(n, 1), 0.0);
            obk_opts o{};
            o.check_every = probe_sweeps;  // residuals at the start and after the probe
            obk_info info{};
            rc = obk_solve_ex(h, &o, f, nullptr, tol, probe_sweeps, x.data(), &info);
            if (rc != OBK_OK && rc != OBK_NOT_CONVERGED) {
                std::string msg = obk_last_error();
                obk_destroy(h);
                throw Error{(int)rc, msg};
            }
            obk_thr_probe pr{};
            pr.thr = thr_cand[k];
            pr.groups = h->info.groups;
            pr.conflicts = h->info.n_conflicts;
            pr.probe_sweeps = info.sweeps;
            pr.setup_ms = h->info.setup_ms;
            pr.probe_ms = info.solve_ms;
            pr.rel_res = info.rel_res;
            double sweeps = (double)std::max<int64_t>(info.sweeps, 1);
            pr.rate = info.rel_res > 0.0 ? pow(info.rel_res, 1.0 / sweeps) : 0.0;
            if (info.rel_res <= tol) pr.predicted_ms = pr.setup_ms + pr.probe_ms;
            else if (pr.rate > 0.0 && pr.rate < 1.0)
                pr.predicted_ms = pr.setup_ms + pr.probe_ms +
                                  ceil(log(tol / info.rel_res) / log(pr.rate)) * (pr.probe_ms / sweeps);
            else pr.predicted_ms = HUGE_VAL;
            if (probes) probes[k] = pr;
            if (best_k < 0 || pr.predicted_ms < best_ms) {
                if (best) obk_destroy(best);
                best = h;
                best_ms = pr.predicted_ms;
                best_k = k;
            } else {
                obk_destroy(h);
            }
        }
    } catch (...) {
        if (best) obk_destroy(best);
        throw;
    }
    *out_thr = thr_cand[best_k];
    if (out) *out = best;
    else obk_destroy(best);
    set_last_error("");
    return OBK_OK;
    OBK_API_END
}

obk_status obk_grouping_stats(obk_handle* h, obk_gstats* out)
{
    OBK_API_BEGIN
    set_last_error("");
    if (!h || !out) throw Error{-1, "handle or output NULL"};
    OBK_CUDA(cudaSetDevice(h->device));
    obk_gstats r{};
    r.N = h->N;
    int64_t nz = 0;
    uint64_t sum = 0;
    cosine_stats(h->L, &nz, &sum, h->err.p, h->st);
    r.nonzero_entries = nz;
    r.abs_cos_sum = sum;
    double num = (double)h->N * (double)h->N;
    r.zn = num > 0 ? (num - (double)nz) / num : 0.0;
    r.nn = num > 0 ? (double)sum * 0x1p-32 / num : 0.0;
    r.groups = h->L.G;
    r.conflicts = h->L.n_conflicts;
    r.color_rounds = h->L.color_rounds;
    r.min_group_rows = h->L.G ? INT64_MAX : 0;
    for (int64_t g = 0; g < h->L.G; ++g) {
        int64_t c = h->L.h_gptr[g + 1] - h->L.h_gptr[g];
        r.min_group_rows = std::min(r.min_group_rows, c);
        r.max_group_rows = std::max(r.max_group_rows, c);
    }
    *out = r;
    return OBK_OK;
    OBK_API_END
}

}  // extern "C"

namespace obk {
bool batch_eligible(const obk_handle* h)
{
    return h && batch_smem_bytes(h->N, h->L.Ngm) <= batch_smem_limit();
}

void prepare_batch(obk_handle* h)
{
    if (h) ensure_gm_csr(h->L, h->st);
}

void* handle_stream(const obk_handle* h) { return h ? (void*)h->st : nullptr; }
}  // namespace obk

extern "C" {

int64_t obk_batch_max_n(void)
{
    try {
        return (int64_t)(batch_smem_limit() / (3 * sizeof(double)));
    } catch (...) {
        return 0;
    }
}

obk_status obk_solve_batch(obk_handle* const* hs, int32_t count, const obk_opts* opts, const double* const* f,
                           const double* const* x0, double tol, int64_t maxit, double* const* x_out,
                           obk_info* info, obk_status* status)
{
    OBK_API_BEGIN
    set_last_error("");
    if (!hs || count < 0 || !f || !x_out || !status) throw Error{-1, "NULL argument"};
    if (count == 0) return OBK_OK;
    if (!(tol > 0.0) || maxit < 1) throw Error{-1, "tol must be > 0 and maxit >= 1"};
    obk_opts o{};
    if (opts) o = *opts;
    if (o.precision != 0) throw Error{-1, "batched solves run FP64 sweeps (precision 0)"};
    if (o.pinv_iters != 0) throw Error{-1, "batched solves take the simultaneous group step (pinv_iters 0)"};
    if (o.check_every < -1) throw Error{-1, "check_every must be >= -1"};
    int dev = hs[0] ? hs[0]->device : -1;
    OBK_CUDA(cudaSetDevice(dev));
    size_t limit = batch_smem_limit(), smem = 0;
    std::vector<BatchSystem> sys((size_t)count);
    cudaStream_t st = hs[0]->st;
    DBuf<double> res(3 * (size_t)count, st);
    for (int32_t i = 0; i < count; ++i) {
        obk_handle* h = hs[i];
        if (!h || h->device != dev) throw Error{-1, "every handle must be non-NULL and on one device"};
        // the batch kernel reads the group-major rows; they are built on the
        // handle's own stream (their buffers are freed there) and finished
        // before the batch's stream uses them
        if (!h->L.has_gm_csr) {
            ensure_gm_csr(h->L, h->st);
            OBK_CUDA(cudaStreamSynchronize(h->st));
        }
        if (!f[i] || !x_out[i] || !is_device_ptr(f[i]) || !is_device_ptr(x_out[i]) ||
            (x0 && x0[i] && !is_device_ptr(x0[i])))
            throw Error{-1, "f, x0 and x_out of a batch must be device memory"};
        size_t need = batch_smem_bytes(h->N, h->L.Ngm);
        if (need > limit) throw Error{-1, "system " + std::to_string(i) + " needs more shared memory than a block has"};
        smem = std::max(smem, need);
        BatchSystem& d = sys[(size_t)i];
        d.m = h->m; d.n = h->n; d.N = h->N; d.Ngm = h->L.Ngm; d.G = h->L.G; d.n_zero = h->n_zero;
        d.perm = h->perm.p; d.src_gm = h->src_gm.p; d.zero_src = h->zero_src.p;
        d.gptr = h->L.gptr.p; d.gseg_ptr = h->L.gseg_ptr.p; d.grp_rp = h->L.grp_rp.p; d.grp_ci = h->L.grp_ci.p;
        d.grp_v = h->L.grp_v.p; d.grp_inv = h->L.grp_inv.p; d.seg_ptr = h->L.seg_ptr.p; d.seg_col = h->L.seg_col.p;
        d.mir_row = h->L.mir_row.p; d.mir_val = h->L.mir_val.p;
        d.f = f[i]; d.x0 = x0 ? x0[i] : nullptr; d.x_out = x_out[i];
        d.tol = tol; d.stagnation = o.stagnation; d.maxit = maxit;
        d.check_every = o.check_every == 0 ? 1 : o.check_every;
        d.result = res.p + 3 * (size_t)i;
    }
    Timer tm(st);
    DBuf<BatchSystem> dsys((size_t)count, st);
    OBK_CUDA(cudaMemcpyAsync(dsys.p, sys.data(), sys.size() * sizeof(BatchSystem), cudaMemcpyHostToDevice, st));
    launch_batch(dsys.p, count, smem, st);
    std::vector<double> hres(3 * (size_t)count);
    OBK_CUDA(cudaMemcpyAsync(hres.data(), res.p, hres.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    double ms = tm.stop_ms();
    OBK_CUDA(cudaStreamSynchronize(st));
    for (int32_t i = 0; i < count; ++i) {
        status[i] = hres[3 * (size_t)i] == 0.0 ? OBK_OK : OBK_NOT_CONVERGED;
        if (info) {
            info[i] = hs[i]->info;
            info[i].sweeps = (int64_t)hres[3 * (size_t)i + 1];
            info[i].rel_res = hres[3 * (size_t)i + 2];
            info[i].solve_ms = ms;
            info[i].status = status[i];
        }
    }
    return OBK_OK;
    OBK_API_END
}

obk_status obk_autotune(obk_handle* h, int32_t precision, obk_tune* out)
{
    OBK_API_BEGIN
    set_last_error("");
    if (!h || (precision != 0 && precision != 1)) throw Error{-1, "handle NULL or precision not 0/1"};
    OBK_CUDA(cudaSetDevice(h->device));
    obk_tune t{};
    // candidates in the order documented in obk.h
    std::vector<TuneChoice> cand = {{1, 1024, 2, 2}, {1, 1024, 1, 2}, {1, 512, 2, 2}, {1, 512, 1, 2},
                                    {1, 1024, 2, 1}, {1, 512, 2, 1}};
    const double avg = h->L.Ngm ? (double)h->L.nnz_gm / (double)h->L.Ngm : 1.0;
    for (int sub : {2, 4, 8, 16})
        for (int block : {1024, 512}) cand.push_back(TuneChoice{sub, block, 2, 1});
    ensure_gm_csr(h->L, h->st);  // for the sub-warp candidates
    double best = 1e300;
    TuneChoice choice{1, 512, 2, 1};
    int k = 0;
    for (const TuneChoice& c : cand) {
        if (k >= 16) break;
        double ms = 0.0;
        if (!(c.sub > 2 * avg + 2)) {  // more lanes than entries: skip
            ms = time_sweep(h->L, c.sub, precision, c.block, c.staging, c.sync, h->err.p, h->st);
            if (ms > 0.0 && ms < best) { best = ms; choice = c; }
        }
        t.candidate_ms[k++] = ms;
    }
    t.n_candidates = k;
    t.rows_per_warp = 32 / choice.sub;
    t.block_threads = choice.block;
    t.staging = choice.staging;
    t.sync_mode = choice.sync;
    t.sweep_ms = best;
    h->tuned[precision] = choice;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[tune_key(h, precision)] = choice;
    }
    if (out) *out = t;
    return OBK_OK;
    OBK_API_END
}

obk_status obk_get_dims(const obk_handle* h, int64_t* N, int64_t* nnz, int64_t* G)
{
    if (!h) { set_last_error("handle is NULL"); return OBK_ERR_INVALID; }
    if (N) *N = h->N;
    if (nnz) *nnz = h->nnz;
    if (G) *G = h->L.G;
    return OBK_OK;
}

static obk_status copy_out(const obk_handle* h, void* dst, const void* src, size_t bytes)
{
    OBK_API_BEGIN
    if (!h || !dst) throw Error{-1, "NULL argument"};
    OBK_CUDA(cudaSetDevice(h->device));
    bool ddev = is_device_ptr(dst);
    OBK_CUDA(cudaMemcpyAsync(dst, src, bytes, ddev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
    OBK_CUDA(cudaStreamSynchronize(h->st));
    return OBK_OK;
    OBK_API_END
}

obk_status obk_get_perm(const obk_handle* h, int32_t* perm)
{
    if (!h) { set_last_error("handle is NULL"); return OBK_ERR_INVALID; }
    return copy_out(h, perm, h->perm.p, h->N * sizeof(int32_t));
}

obk_status obk_get_groups(const obk_handle* h, int32_t* group_of)
{
    if (!h) { set_last_error("handle is NULL"); return OBK_ERR_INVALID; }
    return copy_out(h, group_of, h->L.group_of.p, h->N * sizeof(int32_t));
}

obk_status obk_get_row_norms(const obk_handle* h, double* nsq)
{
    if (!h) { set_last_error("handle is NULL"); return OBK_ERR_INVALID; }
    return copy_out(h, nsq, h->L.nsq.p, h->N * sizeof(double));
}

int32_t obk_get_setup_profile(const obk_handle* h, double* ms, int32_t cap)
{
    if (!h || !ms || cap <= 0) return 0;
    int n = std::min<int>(h->n_stage, cap);
    for (int i = 0; i < n; ++i) ms[i] = h->stage_ms[i];
    return n;
}

obk_status obk_get_info(const obk_handle* h, obk_info* info)
{
    if (!h || !info) { set_last_error("NULL argument"); return OBK_ERR_INVALID; }
    *info = h->info;
    return OBK_OK;
}

obk_status obk_residual(const obk_csr* A, int64_t m, int64_t n, const double* f, const double* x, double* rel_res)
{
    OBK_API_BEGIN
    set_last_error("");
    if (!A || !f || !x || !rel_res || !A->row_ptr || m <= 0 || n <= 0 || A->nnz < 0 ||
        (A->nnz > 0 && (!A->col_idx || !A->val)))
        throw Error{-1, "NULL pointer or non-positive size"};
    cudaStream_t st;
    OBK_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    try {
        bool adev = A->device_ptrs != 0, fdev = is_device_ptr(f), xdev = is_device_ptr(x);
        int64_t nnz = A->nnz, ntiles = ceil_div(m, kResTile);
        DBuf<int64_t> rp;
        DBuf<int32_t> ci;
        DBuf<double> v, fd, xd, part(2 * ntiles + 1, st);
        const int64_t* prp = A->row_ptr;
        const int32_t* pci = A->col_idx;
        const double* pv = A->val;
        if (!adev) {  // host-resident CSR: check its structure before any device read
            if (A->row_ptr[0] != 0 || A->row_ptr[m] != nnz) throw Error{-1, "row_ptr must run from 0 to nnz"};
            for (int64_t i = 0; i < m; ++i)
                if (A->row_ptr[i + 1] < A->row_ptr[i]) throw Error{-1, "row_ptr is not monotone"};
            for (int64_t e = 0; e < nnz; ++e)
                if (A->col_idx[e] < 0 || (int64_t)A->col_idx[e] >= n)
                    throw Error{-1, "column index out of range at entry " + std::to_string(e)};
            rp.alloc(m + 1, st);
            ci.alloc(std::max<int64_t>(nnz, 1), st);
            v.alloc(std::max<int64_t>(nnz, 1), st);
            to_device(rp.p, A->row_ptr, m + 1, false, st);
            to_device(ci.p, A->col_idx, nnz, false, st);
            to_device(v.p, A->val, nnz, false, st);
            prp = rp.p;
            pci = ci.p;
            pv = v.p;
        }
        const double* pf = f;
        const double* px = x;
        if (!fdev) { fd.alloc(m, st); to_device(fd.p, f, m, false, st); pf = fd.p; }
        if (!xdev) { xd.alloc(n, st); to_device(xd.p, x, n, false, st); px = xd.p; }
        residual_tiles<<<(unsigned)ntiles, kResBlock, 0, st>>>(m, prp, pci, pv, pf, px, part.p);
        OBK_CHECK_LAUNCH();
        residual_final<<<1, 32, 0, st>>>(part.p, ntiles, part.p + 2 * ntiles);
        OBK_CHECK_LAUNCH();
        *rel_res = read_scalar(part.p + 2 * ntiles, st);
    } catch (...) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
        throw;
    }
    OBK_CUDA(cudaStreamSynchronize(st));
    OBK_CUDA(cudaStreamDestroy(st));
    return OBK_OK;
    OBK_API_END
}

void obk_destroy(obk_handle* h)
{
    if (!h) return;
    cudaSetDevice(h->device);
    cudaStream_t st = h->st;
    if (st) cudaStreamSynchronize(st);
    bool own = h->own_stream;
    delete h;  // buffers are freed on st
    if (st) {
        cudaStreamSynchronize(st);
        if (own) cudaStreamDestroy(st);
    }
}

}  // extern "C"
