"""The request server (csrc/runtime.cu) on the CPU: admission, ordering,
cancellation, timeouts, statistics and shutdown.

The server's source, as it stands, is compiled with g++ against stubs (CUDA
stream and memory calls that only answer, a reduce_impl that sleeps in
proportion to the request's rows, records how many requests run at once and
returns a result that identifies the request) and driven under
ThreadSanitizer through these scenarios:

1. 50 requests from two submitting threads: every result is the request's own,
   the statistics count them all, p50 <= p99, nothing left queued, running or
   held against the memory budget;
2. a memory budget below every request's footprint: requests run one at a time
   (a request larger than the budget runs alone);
3. cancellation: a queued request can be cancelled (its wait says so), a
   running one cannot;
4. a wait with a short timeout returns GBLA_E_TIMEOUT and leaves the ticket
   valid for a later wait;
5. destroying a server with requests still queued returns, and every worker
   releases its per-thread resources on exit.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1602_06097_gb300", "csrc", "runtime.cu")
BEGIN = "struct StreamGuard {"

STUBS = r"""
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>
typedef int cudaError_t;
typedef void *cudaStream_t;
const int cudaSuccess = 0, cudaStreamNonBlocking = 1;
#define GBLA_OK 0
#define GBLA_E_INVAL 1
#define GBLA_E_NOMEM 2
#define GBLA_E_CUDA 3
#define GBLA_E_TIMEOUT 4
#define GBLA_E_INTERNAL 5
#define GBLA_E_UNSUPPORTED 6
#define GBLA_E_CANCELLED 7
struct gbla_csr_in { int64_t nrows, ncols, nnz; const int64_t *row_ptr; const int32_t *col; const uint16_t *val; };
struct gbla_csr_out { int64_t nrows, ncols, nnz; int64_t *row_ptr; int32_t *col; uint16_t *val; int on_device; };
struct gbla_options { int want_reduced, gemm_variant, device_ptrs, panel_width, path, leaf_width, kernel_times, fl_order, autotune, echelon; };
#define GBLA_GEMM_AUTO 0
#define GBLA_GEMM_TCGEN05 1
#define GBLA_GEMM_SIMT 2
#define GBLA_PATH_DENSE 1
#define GBLA_ORDER_NEW 0
typedef struct {
    int64_t submitted, completed, failed, cancelled, queued, running;
    double p50_ms, p99_ms, mean_ms;
    size_t mem_budget, mem_in_use;
    int64_t peak_running;
} gbla_server_stats;
typedef struct {
    double latency_ms, queue_ms, device_start_ms, device_end_ms;
    int64_t running_at_start;
} gbla_request_info;
#define GBLA_REQ_QUEUED 0
#define GBLA_REQ_RUNNING 1
#define GBLA_REQ_DONE 2
#define GBLA_REQ_CANCELLED 3
struct gbla_server;
extern "C" int gbla_server_wait_ex(gbla_server *, int64_t, double, gbla_csr_out *, int64_t *, gbla_request_info *);
// events: a host timestamp taken at record time
typedef void *cudaEvent_t;
int cudaEventCreate(cudaEvent_t *e) { *e = new double(0.0); return 0; }
int cudaEventDestroy(cudaEvent_t e) { delete (double *)e; return 0; }
int cudaEventRecord(cudaEvent_t e, cudaStream_t) {
    *(double *)e = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
    return 0;
}
int cudaEventSynchronize(cudaEvent_t) { return 0; }
int cudaEventElapsedTime(float *ms, cudaEvent_t a, cudaEvent_t b) { *ms = (float)(*(double *)b - *(double *)a); return 0; }
int cudaStreamSynchronize(cudaStream_t) { return 0; }
int cudaSetDevice(int) { return 0; }
int cudaGetDevice(int *d) { *d = 0; return 0; }
std::atomic<int> g_streams{0};
int cudaStreamCreateWithFlags(cudaStream_t *s, int) { *s = (void *)(intptr_t)(++g_streams); return 0; }
int cudaStreamDestroy(cudaStream_t) { return 0; }
int cudaMemGetInfo(size_t *f, size_t *t) { *f = (size_t)1 << 30; *t = (size_t)2 << 30; return 0; }
int cudaGetLastError() { return 0; }
extern "C" void gbla_free(gbla_csr_out *o) { if (o) memset(o, 0, sizeof(*o)); }
namespace gbla {
std::atomic<int> g_released{0}, g_running{0}, g_max_running{0};
void release_thread_resources() { ++g_released; }
bool is_prime(uint32_t p) {
    if (p < 2) return false;
    for (uint32_t d = 2; d * d <= p; ++d)
        if (p % d == 0) return false;
    return true;
}
int reduce_impl(const gbla_csr_in *in, uint32_t p, const gbla_options *, cudaStream_t s, gbla_csr_out *out,
                int64_t *rank, void *) {
    if (!s) return 99;
    const int now = ++g_running;
    int prev = g_max_running.load();
    while (now > prev && !g_max_running.compare_exchange_weak(prev, now)) {}
    std::this_thread::sleep_for(std::chrono::microseconds(100 * in->nrows));
    --g_running;
    *rank = in->nrows * 7 + p;
    out->nrows = in->nrows;
    return GBLA_OK;
}
namespace {
"""

DRIVER = r"""
static int fails = 0;
#define CHECK(c) do { if (!(c)) { printf("FAIL line %d: %s\n", __LINE__, #c); ++fails; } } while (0)

struct Req {
    std::vector<int64_t> rp;
    gbla_csr_in in;
    explicit Req(int m) : rp(m + 1, 0) { in = {m, 10, 0, rp.data(), nullptr, nullptr}; }
};

static int64_t submit(gbla_server *s, const Req &r) {
    int64_t t = -1;
    CHECK(gbla_server_submit(s, &r.in, 65521, nullptr, &t) == GBLA_OK);
    return t;
}

static gbla_server_stats stats(gbla_server *s) {
    gbla_server_stats st;
    CHECK(gbla_server_get_stats(s, &st) == GBLA_OK);
    return st;
}

int main() {
    // 1. results and statistics, two submitting threads
    {
        gbla_server *s = nullptr;
        CHECK(gbla_server_create(0, 4, &s) == GBLA_OK);
        std::vector<Req> reqs;
        for (int i = 0; i < 50; ++i) reqs.emplace_back(1 + i % 17);
        std::vector<int64_t> tickets(50);
        std::thread a([&] { for (int i = 0; i < 50; i += 2) tickets[i] = submit(s, reqs[i]); });
        std::thread b([&] { for (int i = 1; i < 50; i += 2) tickets[i] = submit(s, reqs[i]); });
        a.join();
        b.join();
        for (int i = 0; i < 50; ++i) {
            gbla_csr_out o;
            int64_t rank = 0;
            double ms = 0;
            CHECK(gbla_server_wait(s, tickets[i], -1.0, &o, &rank, &ms) == GBLA_OK);
            CHECK(rank == reqs[i].in.nrows * 7 + 65521 && o.nrows == reqs[i].in.nrows && ms >= 0);
        }
        const gbla_server_stats st = stats(s);
        CHECK(st.submitted == 50 && st.completed == 50 && st.failed == 0 && st.cancelled == 0);
        CHECK(st.peak_running >= 2 && st.peak_running <= 4);
        CHECK(st.queued == 0 && st.running == 0 && st.mem_in_use == 0);
        CHECK(st.p50_ms > 0 && st.p50_ms <= st.p99_ms);
        gbla_server_destroy(s);
    }
    // 2. a budget below every footprint: one request at a time
    {
        g_max_running = 0;
        gbla_server *s = nullptr;
        CHECK(gbla_server_create(1, 4, &s) == GBLA_OK);
        std::vector<Req> reqs;
        for (int i = 0; i < 12; ++i) reqs.emplace_back(20);
        std::vector<int64_t> t;
        for (auto &r : reqs) t.push_back(submit(s, r));
        for (auto x : t) {
            gbla_csr_out o;
            int64_t rank;
            CHECK(gbla_server_wait(s, x, -1.0, &o, &rank, nullptr) == GBLA_OK);
        }
        CHECK(g_max_running.load() == 1);
        gbla_server_destroy(s);
    }
    // 3. cancel a queued request, not a running one; 4. wait with a timeout
    {
        gbla_server *s = nullptr;
        CHECK(gbla_server_create(0, 1, &s) == GBLA_OK);
        Req big(1000), small(3);
        const int64_t t0 = submit(s, big);
        const int64_t t1 = submit(s, small), t2 = submit(s, small);
        for (int i = 0; i < 2000 && stats(s).running == 0; ++i) std::this_thread::sleep_for(std::chrono::milliseconds(1));
        CHECK(stats(s).running == 1);
        int state = -1;
        CHECK(gbla_server_poll(s, t0, &state) == GBLA_OK && state == GBLA_REQ_RUNNING);
        CHECK(gbla_server_poll(s, t1, &state) == GBLA_OK && state == GBLA_REQ_QUEUED);
        CHECK(gbla_server_cancel(s, t0) == GBLA_E_INVAL);        // running
        CHECK(gbla_server_cancel(s, t2) == GBLA_OK);             // queued
        CHECK(gbla_server_poll(s, t2, &state) == GBLA_OK && state == GBLA_REQ_CANCELLED);
        gbla_csr_out o;
        int64_t rank;
        CHECK(gbla_server_wait(s, t0, 0.001, &o, &rank, nullptr) == GBLA_E_TIMEOUT);
        gbla_request_info info;
        CHECK(gbla_server_wait_ex(s, t0, -1.0, &o, &rank, &info) == GBLA_OK && rank == 1000 * 7 + 65521);
        CHECK(info.running_at_start == 1 && info.queue_ms >= 0 && info.latency_ms >= info.queue_ms);
        CHECK(info.device_start_ms >= 0 && info.device_end_ms >= info.device_start_ms + 50);   // slept 100 ms
        CHECK(gbla_server_poll(s, t0, &state) == GBLA_E_INVAL);  // consumed
        for (int i = 0; i < 2000; ++i) {
            CHECK(gbla_server_poll(s, t1, &state) == GBLA_OK);
            if (state == GBLA_REQ_DONE) break;
            std::this_thread::sleep_for(std::chrono::milliseconds(1));
        }
        CHECK(state == GBLA_REQ_DONE);
        CHECK(gbla_server_wait(s, t1, -1.0, &o, &rank, nullptr) == GBLA_OK && rank == 3 * 7 + 65521);
        CHECK(gbla_server_wait(s, t2, -1.0, &o, &rank, nullptr) == GBLA_E_CANCELLED);
        CHECK(gbla_server_wait(s, t2, -1.0, &o, &rank, nullptr) == GBLA_E_INVAL);   // ticket consumed
        const gbla_server_stats st = stats(s);
        CHECK(st.completed == 2 && st.cancelled == 1);
        gbla_server_destroy(s);
    }
    // invalid requests are refused at submit
    {
        gbla_server *s = nullptr;
        CHECK(gbla_server_create(0, 2, &s) == GBLA_OK);
        Req r(4);
        int64_t t;
        CHECK(gbla_server_submit(s, &r.in, 65520, nullptr, &t) == GBLA_E_INVAL);   // not prime
        gbla_options dev{0, 0, 1, 0};
        CHECK(gbla_server_submit(s, &r.in, 65521, &dev, &t) == GBLA_E_INVAL);     // device pointers
        gbla_server_destroy(s);
    }
    // 5. destroy with requests still queued
    const int released0 = g_released.load();
    {
        gbla_server *s = nullptr;
        CHECK(gbla_server_create(0, 3, &s) == GBLA_OK);
        Req big(200), small(2);
        submit(s, big);
        for (int i = 0; i < 20; ++i) submit(s, small);
        gbla_server_destroy(s);
    }
    CHECK(g_released.load() - released0 == 3);
    printf("fails %d\n", fails);
    return fails != 0;
}
"""


def test_server_under_thread_sanitizer(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    src = open(SRC).read()
    a = src.find(BEGIN)
    assert a >= 0, "server section not found in runtime.cu"
    cpp = tmp_path / "server.cpp"
    cpp.write_text(STUBS + src[a:] + DRIVER)
    exe = tmp_path / "server"
    r = subprocess.run([gxx, "-O1", "-g", "-std=c++17", "-pthread", "-fsanitize=thread", str(cpp), "-o", str(exe)],
                       capture_output=True, text=True, timeout=300)
    if r.returncode != 0 and "sanitize" in r.stderr:
        pytest.skip("ThreadSanitizer not available: " + r.stderr[-200:])
    assert r.returncode == 0, r.stderr[-3000:]
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    out = run.stdout + run.stderr
    assert "WARNING: ThreadSanitizer" not in out, out[-3000:]
    assert run.returncode == 0 and "fails 0" in out, out[-3000:]
