// server.cu -- request loop with continuous batching (obk_submit / obk_poll).
//
// Requests are queued on the host and admitted while the device memory they
// are estimated to need fits the HBM budget.  Each admitted request is set up
// (obk_create) on one of max_streams worker streams, so requests admitted
// while others run overlap on the device; a request that does not fit yet
// stays PENDING until running ones release their memory.  Large systems are
// then solved on the cooperative grid of their stream; small FP64 systems join
// a ready list that is solved many at a time by obk_solve_batch (one thread
// block per system, x in shared memory), run by whichever worker finds no
// batch in progress.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/obk.h"
#include "batch.cuh"
#include "common.cuh"

namespace {

struct Request {
    uint64_t ticket = 0;
    int64_t m = 0, n = 0;
    double thr = 0.1, tol = 1e-8;
    int64_t maxit = 1000;
    obk_opts opts{};
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    std::vector<double> v, f, x0, x;
    bool has_x0 = false;
    size_t bytes = 0;
    std::atomic<int> state{0};  // 0 queued, 1 running, 2 done
    std::atomic<bool> cancel{false};
    int status = OBK_PENDING;
    obk_info info{};
    std::string err;
    // batched path: prepared system and device copies of f, x0 and x
    obk_handle* h = nullptr;
    obk::DBuf<double> fdev, x0dev, xdev;
};

// Upper estimate of the device bytes a solve needs at its peak (setup).
// HBM a request may need while it is prepared and solved: the handle keeps
// about 100 bytes per entry (group-major rows and column mirror in FP64 and
// FP32, their sliced copies with padding, A~ for the block form) and 80 per
// row; obk_create's transients (sorts, pair tables, conflict lists) add up to
// about as much again at their peak.
size_t footprint(int64_t m, int64_t n, int64_t nnz)
{
    int64_t N = std::max(m, n);
    return (size_t)(nnz * 192 + N * 256 + (64 << 20));
}

}  // namespace

extern "C" size_t obk_request_footprint(int64_t m, int64_t n, int64_t nnz)
{
    return m > 0 && n > 0 && nnz >= 0 ? footprint(m, n, nnz) : 0;
}

struct obk_server {
    size_t budget = 0, in_use = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Request>> queue;
    std::deque<std::shared_ptr<Request>> ready;  // prepared small systems awaiting a batch
    bool batch_running = false;
    std::map<uint64_t, std::shared_ptr<Request>> all;
    uint64_t next_ticket = 1;
    bool stopping = false;
    std::vector<std::thread> workers;
};

// Finish a request: record its result, release its memory and budget.
static void finish(obk_server* s, const std::shared_ptr<Request>& r, int rc)
{
    if (r->h) {
        obk_destroy(r->h);
        r->h = nullptr;
    }
    r->fdev.release();
    r->x0dev.release();
    r->xdev.release();
    if (r->cancel.load() && rc >= 0) rc = OBK_ERR_CANCELLED;
    r->status = rc;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->in_use -= r->bytes;
    }
    r->state.store(2);
    s->cv.notify_all();
}

// Solve the ready small systems in batches (one launch per batch) until the
// ready list is empty; only one worker runs batches at a time.
static void run_batches(obk_server* s)
{
    constexpr size_t kMaxBatch = 2048;
    for (;;) {
        std::vector<std::shared_ptr<Request>> b;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->batch_running || s->ready.empty()) return;
            s->batch_running = true;
            // same tolerance, iteration limit and stopping options in one batch
            const Request& f0 = *s->ready.front();
            for (auto it = s->ready.begin(); it != s->ready.end() && b.size() < kMaxBatch;) {
                const Request& q = **it;
                if (q.tol == f0.tol && q.maxit == f0.maxit && q.opts.check_every == f0.opts.check_every &&
                    q.opts.stagnation == f0.opts.stagnation) {
                    b.push_back(*it);
                    it = s->ready.erase(it);
                } else {
                    ++it;
                }
            }
        }
        std::vector<obk_handle*> hs;
        std::vector<const double*> fs, x0s;
        std::vector<double*> xs;
        for (auto& r : b) {
            hs.push_back(r->h);
            fs.push_back(r->fdev.p);
            x0s.push_back(r->has_x0 ? r->x0dev.p : nullptr);
            xs.push_back(r->xdev.p);
        }
        std::vector<obk_status> st(b.size(), OBK_ERR_CUDA);
        std::vector<obk_info> info(b.size());
        obk_opts o = b[0]->opts;
        obk_status rc = obk_solve_batch(hs.data(), (int32_t)hs.size(), &o, fs.data(), x0s.data(), b[0]->tol,
                                        b[0]->maxit, xs.data(), info.data(), st.data());
        std::string err = rc < 0 ? obk_last_error() : "";
        for (size_t i = 0; i < b.size(); ++i) {
            auto& r = b[i];
            int ri = rc < 0 ? (int)rc : (int)st[i];
            if (ri >= 0) {
                r->x.assign((size_t)r->n, 0.0);
                cudaStream_t hst = static_cast<cudaStream_t>(obk::handle_stream(r->h));
                if (cudaMemcpyAsync(r->x.data(), r->xdev.p, (size_t)r->n * sizeof(double), cudaMemcpyDeviceToHost,
                                    hst) != cudaSuccess ||
                    cudaStreamSynchronize(hst) != cudaSuccess) {
                    ri = OBK_ERR_CUDA;
                    r->err = "copying the result failed";
                }
                r->info = info[i];
            } else {
                r->err = err;
            }
            finish(s, r, ri);
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->batch_running = false;
        }
    }
}

static void worker_loop(obk_server* s)
{
    cudaSetDevice(s->device);
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return;
    for (;;) {
        std::shared_ptr<Request> r;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            for (;;) {
                if (s->stopping && s->queue.empty()) {
                    lk.unlock();
                    run_batches(s);
                    cudaStreamDestroy(st);
                    return;
                }
                // first queued request that fits the remaining budget (arrival order)
                auto it = std::find_if(s->queue.begin(), s->queue.end(), [&](const std::shared_ptr<Request>& q) {
                    return q->cancel.load() || s->in_use + q->bytes <= s->budget;
                });
                if (it != s->queue.end()) {
                    r = *it;
                    s->queue.erase(it);
                    if (!r->cancel.load()) s->in_use += r->bytes;
                    break;
                }
                s->cv.wait(lk);
            }
        }
        if (r->cancel.load()) {
            r->status = OBK_ERR_CANCELLED;
            r->state.store(2);
            continue;
        }
        r->state.store(1);
        obk_csr A{r->rp.data(), r->ci.data(), r->v.data(), (int64_t)r->ci.size(), 0};
        obk_handle* h = nullptr;
        obk_status rc = obk_create_on_stream(&A, r->m, r->n, r->thr, (void*)st, &h);
        if (rc == OBK_OK && r->opts.precision == 0 && r->opts.pinv_iters == 0 && obk::batch_eligible(h) &&
            !r->cancel.load()) {
            // small system: build its group-major rows and stage f (and x0)
            // on the device, on this worker's stream, then join the ready list
            bool ok = true;
            try {
                obk::prepare_batch(h);
                r->fdev.alloc((size_t)r->m, st);
                r->xdev.alloc((size_t)r->n, st);
                ok = cudaMemcpyAsync(r->fdev.p, r->f.data(), (size_t)r->m * sizeof(double), cudaMemcpyHostToDevice,
                                     st) == cudaSuccess;
                if (ok && r->has_x0) {
                    r->x0dev.alloc((size_t)r->n, st);
                    ok = cudaMemcpyAsync(r->x0dev.p, r->x0.data(), (size_t)r->n * sizeof(double),
                                         cudaMemcpyHostToDevice, st) == cudaSuccess;
                }
                ok = ok && cudaStreamSynchronize(st) == cudaSuccess;
            } catch (const obk::Error& e) {
                ok = false;
                r->err = e.msg;
            }
            if (ok) {
                r->h = h;
                {
                    std::lock_guard<std::mutex> lk(s->mu);
                    s->ready.push_back(r);
                }
                run_batches(s);
                continue;
            }
            if (r->err.empty()) r->err = "staging a batched request failed";
            r->h = h;
            finish(s, r, OBK_ERR_CUDA);
            continue;
        }
        if (rc == OBK_OK) {
            r->x.assign((size_t)r->n, 0.0);
            if (r->cancel.load()) rc = OBK_ERR_CANCELLED;
            else
                rc = obk_solve_ex(h, &r->opts, r->f.data(), r->has_x0 ? r->x0.data() : nullptr, r->tol, r->maxit,
                                  r->x.data(), &r->info);
        }
        if (rc < 0) r->err = obk_last_error();
        r->h = h;
        finish(s, r, rc);
        run_batches(s);
    }
}

extern "C" {

obk_status obk_server_create(size_t hbm_budget_bytes, int32_t max_streams, obk_server** out)
{
    if (!out) return OBK_ERR_INVALID;
    *out = nullptr;
    if (max_streams < 0 || max_streams > 256) {
        obk::set_last_error("max_streams must be in [0, 256]");
        return OBK_ERR_INVALID;
    }
    obk_server* s = new (std::nothrow) obk_server();
    if (!s) return OBK_ERR_NOMEM;
    s->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)150 << 30;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        obk::set_last_error("no CUDA device");
        return OBK_ERR_CUDA;
    }
    int nw = max_streams ? max_streams : 8;
    for (int i = 0; i < nw; ++i) s->workers.emplace_back(worker_loop, s);
    *out = s;
    return OBK_OK;
}

obk_status obk_submit(obk_server* s, const obk_csr* A, int64_t m, int64_t n, double thr, const double* f,
                      const double* x0, double tol, int64_t maxit, const obk_opts* opts, uint64_t* ticket)
{
    if (!s || !A || !f || !ticket || m <= 0 || n <= 0 || A->nnz < 0 || !A->row_ptr ||
        (A->nnz > 0 && (!A->col_idx || !A->val))) {
        obk::set_last_error("invalid request arguments");
        return OBK_ERR_INVALID;
    }
    if (!(thr > 0.0 && thr <= 1.0) || !(tol > 0.0) || maxit < 1) {
        obk::set_last_error("thr must be in (0, 1], tol > 0, maxit >= 1");
        return OBK_ERR_INVALID;
    }
    auto r = std::make_shared<Request>();
    r->m = m;
    r->n = n;
    r->thr = thr;
    r->tol = tol;
    r->maxit = maxit;
    if (opts) r->opts = *opts;
    r->bytes = footprint(m, n, A->nnz);
    if (r->bytes > s->budget) {
        obk::set_last_error("request exceeds the server's HBM budget");
        return OBK_ERR_BUDGET;
    }
    try {
        r->rp.resize((size_t)m + 1);
        r->ci.resize((size_t)A->nnz);
        r->v.resize((size_t)A->nnz);
        r->f.resize((size_t)m);
        cudaMemcpyKind k = A->device_ptrs ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
        if (cudaMemcpy(r->rp.data(), A->row_ptr, (m + 1) * sizeof(int64_t), k) != cudaSuccess ||
            (A->nnz && cudaMemcpy(r->ci.data(), A->col_idx, A->nnz * sizeof(int32_t), k) != cudaSuccess) ||
            (A->nnz && cudaMemcpy(r->v.data(), A->val, A->nnz * sizeof(double), k) != cudaSuccess)) {
            obk::set_last_error("copying the request's matrix failed");
            return OBK_ERR_CUDA;
        }
        cudaPointerAttributes pa;
        auto kind_of = [&](const void* p) {
            if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) { (void)cudaGetLastError(); return cudaMemcpyHostToHost; }
            return (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged) ? cudaMemcpyDeviceToHost
                                                                                          : cudaMemcpyHostToHost;
        };
        if (cudaMemcpy(r->f.data(), f, m * sizeof(double), kind_of(f)) != cudaSuccess) return OBK_ERR_CUDA;
        if (x0) {
            r->x0.resize((size_t)n);
            r->has_x0 = true;
            if (cudaMemcpy(r->x0.data(), x0, n * sizeof(double), kind_of(x0)) != cudaSuccess) return OBK_ERR_CUDA;
        }
    } catch (const std::bad_alloc&) {
        return OBK_ERR_NOMEM;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->ticket = s->next_ticket++;
        *ticket = r->ticket;
        s->all[r->ticket] = r;
        s->queue.push_back(r);
    }
    s->cv.notify_all();
    return OBK_OK;
}

obk_status obk_poll(obk_server* s, uint64_t ticket, double* x_out, obk_info* info)
{
    if (!s) return OBK_ERR_INVALID;
    std::shared_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->all.find(ticket);
        if (it == s->all.end()) {
            obk::set_last_error("unknown ticket");
            return OBK_ERR_NOT_FOUND;
        }
        r = it->second;
        if (r->state.load() != 2) return OBK_PENDING;
        s->all.erase(it);
    }
    if (x_out && r->status >= 0 && !r->x.empty()) std::copy(r->x.begin(), r->x.end(), x_out);
    if (info) *info = r->info;
    if (r->status < 0) obk::set_last_error(r->err.empty() ? "request failed" : r->err);
    return (obk_status)r->status;
}

obk_status obk_cancel(obk_server* s, uint64_t ticket)
{
    if (!s) return OBK_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return OBK_ERR_NOT_FOUND;
    it->second->cancel.store(true);
    s->cv.notify_all();
    return OBK_OK;
}

void obk_server_destroy(obk_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv.notify_all();
    for (auto& t : s->workers) t.join();
    delete s;
}

}  // extern "C"
