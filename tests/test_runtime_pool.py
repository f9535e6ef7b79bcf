"""The batch entry point's worker pool (csrc/runtime.cu) on the CPU.

The pool's code -- gbla_reduce_batch and the process-wide workers it hands
matrices to -- is taken from the source as it stands and compiled with g++
against stubs: CUDA stream calls that only count, and a reduce_impl that
records which matrix it was given.  Four caller threads then make thousands
of batch calls with random sizes and worker counts (0 = the default, and more
workers than matrices), under ThreadSanitizer.  Every matrix must be reduced
exactly once with its own result, invalid primes must come back as
GBLA_E_INVAL, the streams must be created once per worker rather than per
call, and the sanitizer must report nothing.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1602_06097_gb300", "csrc", "runtime.cu")
BEGIN = "int default_workers(int w)"
END = "// ----------------------------------------------------------------- server"

STUBS = r"""
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <random>
#include <thread>
#include <vector>
typedef int cudaError_t;
typedef void *cudaStream_t;
const int cudaSuccess = 0, cudaStreamNonBlocking = 1;
#define GBLA_OK 0
#define GBLA_E_INVAL 1
#define GBLA_E_NOMEM 2
#define GBLA_E_CUDA 3
#define GBLA_E_INTERNAL 5
struct gbla_csr_in { int64_t nrows, ncols, nnz; const int64_t *row_ptr; const int32_t *col; const uint16_t *val; };
struct gbla_csr_out { int64_t nrows, ncols, nnz; int64_t *row_ptr; int32_t *col; uint16_t *val; int on_device; };
struct gbla_options { int want_reduced, gemm_variant, device_ptrs, panel_width, path, leaf_width, kernel_times, fl_order, autotune, echelon; };
static thread_local int cur_dev = 0;
int cudaSetDevice(int d) { cur_dev = d; return 0; }
int cudaGetDevice(int *d) { *d = cur_dev; return 0; }
std::atomic<int> g_streams{0};
int cudaStreamCreateWithFlags(cudaStream_t *s, int) { *s = (void *)(intptr_t)(++g_streams); return 0; }
int cudaGetLastError() { return 0; }
namespace gbla {
bool is_prime(uint32_t p) {
    if (p < 2) return false;
    for (uint32_t d = 2; d * d <= p; ++d)
        if (p % d == 0) return false;
    return true;
}
std::atomic<long> g_calls{0};
int reduce_impl(const gbla_csr_in *in, uint32_t p, const gbla_options *, cudaStream_t s, gbla_csr_out *out,
                int64_t *rank, void *) {
    if (!s) return 99;
    ++g_calls;
    *rank = in->nrows * 7 + p;    // a result that identifies the matrix
    out->nrows = in->nrows;
    if (in->nrows % 5 == 0) std::this_thread::sleep_for(std::chrono::microseconds(50));
    return GBLA_OK;
}
namespace {
"""

DRIVER = r"""
int main() {
    std::vector<std::thread> callers;
    std::atomic<long> bad{0}, calls{0}, items{0};
    for (int t = 0; t < 4; ++t)
        callers.emplace_back([&, t] {
            std::mt19937 rng(t + 1);
            for (int it = 0; it < 800; ++it) {
                const int n = rng() % 40, workers = rng() % 12;
                std::vector<gbla_csr_in> in(n);
                std::vector<uint32_t> p(n);
                std::vector<gbla_csr_out> outs(n);
                std::vector<int64_t> ranks(n);
                std::vector<int> codes(n);
                for (int i = 0; i < n; ++i) {
                    in[i] = {(int64_t)(rng() % 1000 + 1), (int64_t)(rng() % 1000 + 1), 0, nullptr, nullptr, nullptr};
                    p[i] = (rng() % 7 == 0) ? 65520u : 65521u;
                }
                const int rc = gbla_reduce_batch(n, in.data(), p.data(), nullptr, workers, outs.data(), ranks.data(),
                                                 codes.data());
                bool any_bad = false;
                for (int i = 0; i < n; ++i) {
                    if (p[i] == 65520u) {
                        any_bad = true;
                        if (codes[i] != GBLA_E_INVAL) ++bad;
                    } else {
                        ++items;
                        if (codes[i] != GBLA_OK || ranks[i] != in[i].nrows * 7 + 65521 || outs[i].nrows != in[i].nrows)
                            ++bad;
                    }
                }
                if (any_bad ? rc == GBLA_OK : rc != GBLA_OK) ++bad;
                ++calls;
            }
        });
    for (auto &c : callers) c.join();
    printf("calls %ld items %ld reduced %ld bad %ld streams %d\n", calls.load(), items.load(), gbla::g_calls.load(),
           bad.load(), g_streams.load());
    return bad.load() != 0;
}
"""


def test_batch_pool_under_thread_sanitizer(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    src = open(SRC).read()
    a, b = src.find(BEGIN), src.find(END)
    assert 0 <= a < b, "pool section not found in runtime.cu"
    cpp = tmp_path / "pool.cpp"
    cpp.write_text(STUBS + src[a:b] + DRIVER)
    exe = tmp_path / "pool"
    r = subprocess.run([gxx, "-O1", "-g", "-std=c++17", "-pthread", "-fsanitize=thread", str(cpp), "-o", str(exe)],
                       capture_output=True, text=True, timeout=300)
    if r.returncode != 0 and "sanitize" in r.stderr:
        pytest.skip("ThreadSanitizer not available: " + r.stderr[-200:])
    assert r.returncode == 0, r.stderr[-3000:]
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    out = run.stdout + run.stderr
    assert "WARNING: ThreadSanitizer" not in out, out[-3000:]
    assert run.returncode == 0, out[-3000:]
    fields = dict(zip(out.split()[0::2], out.split()[1::2]))
    assert fields["bad"] == "0"
    assert fields["items"] == fields["reduced"]            # every valid matrix reduced exactly once
    assert int(fields["streams"]) <= 11                     # one stream per worker, not per call
