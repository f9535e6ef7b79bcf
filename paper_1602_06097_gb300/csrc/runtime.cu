// runtime.cu -- many reductions at once: the batch entry point and the
// request server.
//
// Both hand whole reductions (gbla.cu) to a pool of host worker threads,
// each owning a non-blocking CUDA stream on the caller's device, that take
// them from a shared queue.  The reductions' kernels overlap on the device:
// one small reduction leaves most of the GPU idle (short launches, readbacks
// of sizes between phases), so several run side by side.
//
// Batch: every matrix is known up front; workers take them largest first
// (longest-processing-time order) so the tail of the batch is short.
//
// Server: requests arrive over time.  Each is admitted when a worker is free
// and its estimated device footprint fits the memory budget next to the
// requests already running (continuous batching); the queue is served in
// arrival order, and a request that alone exceeds the budget runs when
// nothing else does.  Latency is measured from submit to result ready.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace gbla {
namespace {

struct StreamGuard {
    cudaStream_t s = nullptr;
    int create(int dev) {
        if (cudaSetDevice(dev) != cudaSuccess) return GBLA_E_CUDA;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return GBLA_E_CUDA;
        return GBLA_OK;
    }
    ~StreamGuard() {
        if (s) cudaStreamDestroy(s);
    }
};

int default_workers(int w) { return w > 0 ? (w > 64 ? 64 : w) : 8; }

// One gbla_reduce_batch call as the workers see it.
struct BatchJob {
    int n = 0, nw = 0, dev = 0;
    const int *order = nullptr;   // matrices, largest first
    const gbla_csr_in *in = nullptr;
    const uint32_t *p = nullptr;
    const gbla_options *opt = nullptr;
    gbla_csr_out *outs = nullptr;
    int64_t *ranks = nullptr;
    int *codes = nullptr;
    std::atomic<int> next{0};
};

// Batch workers start on first use and live as long as the process, so each
// keeps its streams, and the per-thread state of the reductions (side stream,
// page-locked readback buffer), from one call to the next instead of
// creating it per call.  Calls are served one at a time; worker w takes part
// in a call that asks for more than w workers.  The pool is never destroyed:
// its threads are detached and wait on its condition variable until the
// process ends.
class BatchPool {
public:
    static BatchPool &get() {
        static BatchPool *pool = new BatchPool();
        return *pool;
    }

    int run(BatchJob &job) {
        std::lock_guard<std::mutex> call(call_mu_);
        {
            std::lock_guard<std::mutex> lk(mu_);
            while (started_ < job.nw) {
                const int w = started_;
                try {
                    std::thread([this, w] { loop(w); }).detach();
                } catch (...) {   // no more threads: run with those already started
                    break;
                }
                ++started_;
            }
            job.nw = std::min(job.nw, started_);
            if (job.nw == 0) return GBLA_E_NOMEM;
            job_ = &job;
            pending_ = job.nw;
            ++gen_;
        }
        cv_job_.notify_all();
        std::unique_lock<std::mutex> lk(mu_);
        cv_done_.wait(lk, [&] { return pending_ == 0; });
        job_ = nullptr;
        return GBLA_OK;
    }

private:
    void loop(int w) {
        std::vector<cudaStream_t> streams;   // one per device, created on first use
        uint64_t seen = 0;
        for (;;) {
            BatchJob *job;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_job_.wait(lk, [&] { return job_ && gen_ != seen && w < job_->nw; });
                seen = gen_;
                job = job_;
            }
            int rc0 = cudaSetDevice(job->dev) == cudaSuccess ? GBLA_OK : GBLA_E_CUDA;
            if (rc0 == GBLA_OK && (int)streams.size() <= job->dev) streams.resize(job->dev + 1, nullptr);
            if (rc0 == GBLA_OK && !streams[job->dev] &&
                cudaStreamCreateWithFlags(&streams[job->dev], cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
                streams[job->dev] = nullptr;
                rc0 = GBLA_E_CUDA;
            }
            for (;;) {
                const int k = job->next.fetch_add(1);
                if (k >= job->n) break;
                const int i = job->order[k];
                if (rc0 != GBLA_OK) { job->codes[i] = rc0; continue; }
                if (job->p[i] >= 65536u || !is_prime(job->p[i])) { job->codes[i] = GBLA_E_INVAL; continue; }
                job->codes[i] = reduce_impl(&job->in[i], job->p[i], job->opt, streams[job->dev], &job->outs[i],
                                            &job->ranks[i], nullptr);
            }
            std::lock_guard<std::mutex> lk(mu_);
            if (--pending_ == 0) cv_done_.notify_all();
        }
    }

    std::mutex call_mu_;   // one batch call at a time
    std::mutex mu_;
    std::condition_variable cv_job_, cv_done_;
    BatchJob *job_ = nullptr;
    uint64_t gen_ = 0;
    int pending_ = 0;
    int started_ = 0;
};

}  // namespace
}  // namespace gbla

using namespace gbla;

// ------------------------------------------------------------------ batch
extern "C" int gbla_reduce_batch(int n, const gbla_csr_in *in, const uint32_t *p, const gbla_options *opt,
                                 int workers, gbla_csr_out *outs, int64_t *ranks, int *codes) {
    if (n < 0 || (n > 0 && (!in || !p || !outs || !ranks || !codes))) return GBLA_E_INVAL;
    for (int i = 0; i < n; ++i) {
        memset(&outs[i], 0, sizeof(outs[i]));
        ranks[i] = 0;
        codes[i] = GBLA_E_INTERNAL;
    }
    if (n == 0) return GBLA_OK;
    BatchJob job;
    if (cudaGetDevice(&job.dev) != cudaSuccess) return GBLA_E_CUDA;
    // largest first
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (double)in[a].nrows * (double)in[a].ncols > (double)in[b].nrows * (double)in[b].ncols;
    });
    job.n = n;
    job.nw = std::min(default_workers(workers), n);
    job.order = order.data();
    job.in = in;
    job.p = p;
    job.opt = opt;
    job.outs = outs;
    job.ranks = ranks;
    job.codes = codes;
    const int rc = BatchPool::get().run(job);
    if (rc != GBLA_OK) return rc;
    for (int i = 0; i < n; ++i)
        if (codes[i] != GBLA_OK) return codes[i];
    return GBLA_OK;
}

// ----------------------------------------------------------------- server
struct gbla_server {
    struct Request {
        int64_t ticket = 0;
        std::vector<int64_t> row_ptr;
        std::vector<int32_t> col;
        std::vector<uint16_t> val;
        gbla_csr_in in{};
        uint32_t p = 0;
        gbla_options opt{};
        size_t est_bytes = 0;
        enum State { QUEUED, RUNNING, DONE, CANCELLED } state = QUEUED;
        gbla_csr_out out{};
        int64_t rank = 0;
        int code = GBLA_OK;
        std::chrono::steady_clock::time_point t_submit, t_start, t_done;
        double dev_t0 = -1.0, dev_t1 = -1.0;   // device timeline (ms since ref)
        int64_t running_at_start = 0;
    };
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::map<int64_t, Request *> reqs;
    std::vector<std::thread> workers;
    std::vector<double> latencies_ms;
    size_t budget = 0, in_use = 0;
    int running = 0;
    int64_t peak_running = 0;
    cudaEvent_t ref = nullptr;   // device time origin of the request timelines
    int64_t next_ticket = 1, submitted = 0, completed = 0, failed = 0, cancelled = 0;
    bool stop = false;
    int dev = 0;

    // Device bytes a reduction of an m x n matrix can need.  The dense path
    // holds the digit planes of A^T, B^T and X (at most 12 bytes per entry of
    // an m x n dense matrix when pivots fill the smaller side) and the
    // uint16 blocks.  The sparse path (the default where the tensor cores
    // apply, see reduce_impl) holds C and D as uint16 and X^T as two digit
    // planes (at most 6 bytes per entry of the m x min(m, n) block C), the
    // compacted sparse operands (at most 24 bytes per input nonzero: a 128-
    // column tile's list entry stores 128 values of four planes) and the
    // echelonisation of D (at most 12 bytes per entry of m x n).
    static size_t estimate(const gbla_csr_in &in, uint32_t p, const gbla_options &opt) {
        const double m = (double)in.nrows, n = (double)in.ncols;
        const double k = std::min(m, n);
        const bool sparse = opt.path != GBLA_PATH_DENSE && p >= 8 && opt.fl_order == GBLA_ORDER_NEW &&
                            (opt.gemm_variant == GBLA_GEMM_AUTO || opt.gemm_variant == GBLA_GEMM_TCGEN05);
        const double work = sparse ? 6.0 * m * k + 24.0 * (double)in.nnz + 12.0 * m * n
                                   : 12.0 * k * n + 6.0 * m * n;
        return (size_t)(8.0 * (m + 1) + 6.0 * (double)in.nnz + work + (64 << 20));
    }

    bool admissible(const Request *r) const {
        return running == 0 || in_use + r->est_bytes <= budget;
    }

    void worker_main() {
        struct ReleaseAtExit {
            ~ReleaseAtExit() { release_thread_resources(); }
        } release_at_exit;   // runs after the stream below is destroyed
        StreamGuard sg;
        const int rc0 = sg.create(dev);
        // events around each reduction on this worker's stream (timeline only)
        cudaEvent_t ev0 = nullptr, ev1 = nullptr;
        if (rc0 == GBLA_OK && ref && (cudaEventCreate(&ev0) != cudaSuccess || cudaEventCreate(&ev1) != cudaSuccess)) {
            cudaGetLastError();
            if (ev0) cudaEventDestroy(ev0);
            ev0 = ev1 = nullptr;
        }
        struct DestroyEvents {
            cudaEvent_t &a, &b;
            ~DestroyEvents() {
                if (a) cudaEventDestroy(a);
                if (b) cudaEventDestroy(b);
            }
        } destroy_events{ev0, ev1};
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            cv_work.wait(lk, [&] { return stop || (!queue.empty() && admissible(queue.front())); });
            if (stop && queue.empty()) return;
            if (queue.empty() || !admissible(queue.front())) continue;
            Request *r = queue.front();
            queue.pop_front();
            r->state = Request::RUNNING;
            in_use += r->est_bytes;
            ++running;
            if (running > peak_running) peak_running = running;
            r->running_at_start = running;
            r->t_start = std::chrono::steady_clock::now();
            lk.unlock();
            int64_t rank = 0;
            gbla_csr_out out{};
            const bool timeline = ev0 && cudaEventRecord(ev0, sg.s) == cudaSuccess;
            const int code = rc0 != GBLA_OK ? rc0 : reduce_impl(&r->in, r->p, &r->opt, sg.s, &out, &rank, nullptr);
            float t0 = -1.f, t1 = -1.f;
            if (timeline && cudaEventRecord(ev1, sg.s) == cudaSuccess && cudaEventSynchronize(ev1) == cudaSuccess &&
                (cudaEventElapsedTime(&t0, ref, ev0) != cudaSuccess || cudaEventElapsedTime(&t1, ref, ev1) != cudaSuccess))
                t0 = t1 = -1.f;
            if (!timeline || t1 < 0.f) cudaGetLastError();
            lk.lock();
            r->dev_t0 = t0;
            r->dev_t1 = t1;
            r->out = out;
            r->rank = rank;
            r->code = code;
            r->t_done = std::chrono::steady_clock::now();
            r->state = Request::DONE;
            in_use -= r->est_bytes;
            --running;
            ++completed;
            if (code != GBLA_OK) ++failed;
            latencies_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
            r->row_ptr.clear(); r->row_ptr.shrink_to_fit();
            r->col.clear(); r->col.shrink_to_fit();
            r->val.clear(); r->val.shrink_to_fit();
            cv_done.notify_all();
            cv_work.notify_all();   // memory was released: queued requests may fit now
        }
    }
};

extern "C" {

int gbla_server_create(size_t mem_budget, int workers, gbla_server **out) {
    if (!out) return GBLA_E_INVAL;
    *out = nullptr;
    auto *s = new (std::nothrow) gbla_server();
    if (!s) return GBLA_E_NOMEM;
    if (cudaGetDevice(&s->dev) != cudaSuccess) {
        delete s;
        return GBLA_E_CUDA;
    }
    if (mem_budget == 0) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return GBLA_E_UNSUPPORTED;
        }
        mem_budget = free_b / 10 * 8;
    }
    s->budget = mem_budget;
    {
        // reference event of the request timelines, recorded and completed here
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreate(&s->ref) == cudaSuccess && cudaEventRecord(s->ref, st) == cudaSuccess &&
            cudaStreamSynchronize(st) == cudaSuccess) {
        } else {
            if (s->ref) cudaEventDestroy(s->ref);
            s->ref = nullptr;
            cudaGetLastError();
        }
        if (st) cudaStreamDestroy(st);
    }
    const int nw = default_workers(workers);
    for (int w = 0; w < nw; ++w) s->workers.emplace_back([s] { s->worker_main(); });
    *out = s;
    return GBLA_OK;
}

int gbla_server_submit(gbla_server *s, const gbla_csr_in *in, uint32_t p, const gbla_options *opt, int64_t *ticket) {
    if (!s || !in || !ticket) return GBLA_E_INVAL;
    if (opt && opt->device_ptrs) return GBLA_E_INVAL;   // the server copies host inputs
    if (p >= 65536u || !is_prime(p)) return GBLA_E_INVAL;
    const int64_t m = in->nrows, nnz = in->nnz;
    if (m < 0 || in->ncols < 0 || nnz < 0 || (m > 0 && !in->row_ptr) || (nnz > 0 && (!in->col || !in->val)))
        return GBLA_E_INVAL;
    auto *r = new (std::nothrow) gbla_server::Request();
    if (!r) return GBLA_E_NOMEM;
    try {
        r->row_ptr.assign(in->row_ptr, in->row_ptr + (m > 0 ? m + 1 : 0));
        r->col.assign(in->col, in->col + nnz);
        r->val.assign(in->val, in->val + nnz);
    } catch (...) {
        delete r;
        return GBLA_E_NOMEM;
    }
    r->in = *in;
    r->in.row_ptr = r->row_ptr.empty() ? nullptr : r->row_ptr.data();
    r->in.col = r->col.empty() ? nullptr : r->col.data();
    r->in.val = r->val.empty() ? nullptr : r->val.data();
    r->p = p;
    if (opt) r->opt = *opt;
    r->opt.device_ptrs = 0;
    r->est_bytes = gbla_server::estimate(*in, p, r->opt);
    r->t_submit = std::chrono::steady_clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    r->ticket = s->next_ticket++;
    s->reqs[r->ticket] = r;
    s->queue.push_back(r);
    ++s->submitted;
    *ticket = r->ticket;
    s->cv_work.notify_one();
    return GBLA_OK;
}

int gbla_server_wait(gbla_server *s, int64_t ticket, double timeout_s, gbla_csr_out *out, int64_t *rank,
                     double *latency_ms) {
    gbla_request_info info;
    const int code = gbla_server_wait_ex(s, ticket, timeout_s, out, rank, latency_ms ? &info : nullptr);
    if (latency_ms && code != GBLA_E_TIMEOUT && code != GBLA_E_INVAL) *latency_ms = info.latency_ms;
    return code;
}

int gbla_server_wait_ex(gbla_server *s, int64_t ticket, double timeout_s, gbla_csr_out *out, int64_t *rank,
                        gbla_request_info *info) {
    if (!s || !out || !rank) return GBLA_E_INVAL;
    memset(out, 0, sizeof(*out));
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return GBLA_E_INVAL;
    gbla_server::Request *r = it->second;
    auto done = [&] {
        return r->state == gbla_server::Request::DONE || r->state == gbla_server::Request::CANCELLED;
    };
    if (timeout_s < 0) {
        s->cv_done.wait(lk, done);
    } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) {
        return GBLA_E_TIMEOUT;   // still queued or running; the ticket stays valid
    }
    int code = r->code;
    if (r->state == gbla_server::Request::CANCELLED) code = GBLA_E_CANCELLED;
    *out = r->out;
    *rank = r->rank;
    if (info) {
        using ms = std::chrono::duration<double, std::milli>;
        info->latency_ms = ms(r->t_done - r->t_submit).count();
        const bool started = r->running_at_start > 0;
        info->queue_ms = started ? ms(r->t_start - r->t_submit).count() : info->latency_ms;
        info->device_start_ms = r->dev_t0;
        info->device_end_ms = r->dev_t1;
        info->running_at_start = r->running_at_start;
    }
    s->reqs.erase(it);
    delete r;
    return code;
}

int gbla_server_poll(gbla_server *s, int64_t ticket, int *state) {
    if (!s || !state) return GBLA_E_INVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return GBLA_E_INVAL;
    switch (it->second->state) {
    case gbla_server::Request::QUEUED: *state = GBLA_REQ_QUEUED; break;
    case gbla_server::Request::RUNNING: *state = GBLA_REQ_RUNNING; break;
    case gbla_server::Request::DONE: *state = GBLA_REQ_DONE; break;
    default: *state = GBLA_REQ_CANCELLED; break;
    }
    return GBLA_OK;
}

int gbla_server_cancel(gbla_server *s, int64_t ticket) {
    if (!s) return GBLA_E_INVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return GBLA_E_INVAL;
    gbla_server::Request *r = it->second;
    if (r->state != gbla_server::Request::QUEUED) return GBLA_E_INVAL;   // running or done
    s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
    r->state = gbla_server::Request::CANCELLED;
    r->t_done = std::chrono::steady_clock::now();
    ++s->cancelled;
    s->cv_done.notify_all();
    return GBLA_OK;
}

int gbla_server_get_stats(gbla_server *s, gbla_server_stats *st) {
    if (!s || !st) return GBLA_E_INVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    memset(st, 0, sizeof(*st));
    st->submitted = s->submitted;
    st->completed = s->completed;
    st->failed = s->failed;
    st->cancelled = s->cancelled;
    st->queued = (int64_t)s->queue.size();
    st->running = s->running;
    st->mem_budget = s->budget;
    st->mem_in_use = s->in_use;
    st->peak_running = s->peak_running;
    if (!s->latencies_ms.empty()) {
        std::vector<double> v = s->latencies_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) {
            const size_t i = (size_t)std::min<double>((double)v.size() - 1, q * (double)(v.size() - 1) + 0.5);
            return v[i];
        };
        st->p50_ms = pct(0.50);
        st->p99_ms = pct(0.99);
        double sum = 0;
        for (double x : v) sum += x;
        st->mean_ms = sum / (double)v.size();
    }
    return GBLA_OK;
}

void gbla_server_destroy(gbla_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        // queued requests are dropped; running ones finish
        for (auto *r : s->queue) {
            r->state = gbla_server::Request::CANCELLED;
            ++s->cancelled;
        }
        s->queue.clear();
        s->stop = true;
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
    for (auto &t : s->workers) t.join();
    for (auto &kv : s->reqs) {
        gbla_free(&kv.second->out);
        delete kv.second;
    }
    if (s->ref) cudaEventDestroy(s->ref);
    delete s;
}

}  // extern "C"
