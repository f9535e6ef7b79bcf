"""The page-locked result cache (host_alloc / host_release in csrc/gbla.cu) on
the CPU.

Its source, as it stands, is compiled with g++ against a pinning stub that
counts page-locks and releases (and can be made to fail), then checked:
a released block is handed to a later request of 1 to 2 times its rounded
size and to no other; above the cap (GBLA_HOST_CACHE_MB) the oldest cached
blocks are released, but never while a reduction is in flight; a block that
could not be pinned comes from malloc and is freed, not cached; four threads
allocating and releasing at once keep the books balanced under
ThreadSanitizer.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1602_06097_gb300", "csrc", "gbla.cu")

STUBS = r"""
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <random>
#include <thread>
#include <utility>
#include <vector>
typedef int cudaError_t;
const int cudaSuccess = 0, cudaHostAllocDefault = 0;
std::atomic<long> g_pins{0}, g_unpins{0};
std::atomic<bool> g_pin_fails{false};
cudaError_t cudaHostAlloc(void **p, size_t bytes, int) {
    if (g_pin_fails) return 2;
    *p = malloc(bytes);
    ++g_pins;
    return cudaSuccess;
}
cudaError_t cudaFreeHost(void *p) { free(p); ++g_unpins; return cudaSuccess; }
cudaError_t cudaGetLastError() { return cudaSuccess; }
inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
namespace gbla {
bool inject_alloc_fault() { return false; }
namespace {
"""

DRIVER = r"""
static int fails = 0;
#define CHECK(c) do { if (!(c)) { printf("FAIL line %d: %s\n", __LINE__, #c); ++fails; } } while (0)
const size_t MB = 1 << 20;

int main() {
    using namespace gbla;
    HostCache &c = host_cache();
    CHECK(c.cap == 10 * MB);                                // GBLA_HOST_CACHE_MB=10
    // reuse within [want, 2 want] of the rounded request (2 MiB granules)
    void *a = host_alloc(3 * MB);                            // 4 MiB pinned
    CHECK(g_pins == 1);
    host_release(a);
    CHECK(c.cached == 4 * MB);
    void *b = host_alloc(3 * MB + 5);                        // same 4 MiB block
    CHECK(b == a && g_pins == 1 && c.cached == 0);
    host_release(b);
    void *d = host_alloc(1 * MB);                            // want 2 MiB: 4 MiB is within 2x
    CHECK(d == a && g_pins == 1);
    host_release(d);
    void *e = host_alloc(MB / 2);                            // want 2 MiB: 4 MiB still within 2x
    CHECK(e == a);
    void *f = host_alloc(MB / 2);                            // nothing cached: a new pin
    CHECK(f != a && g_pins == 2);
    host_release(e);
    host_release(f);
    void *big = host_alloc(20 * MB);                         // 20 MiB: no cached block fits
    CHECK(g_pins == 3);
    host_release(big);                                       // cached 4 + 2 + 20 > 10: evict oldest first
    CHECK(c.cached <= 10 * MB || c.free_blocks.empty());
    CHECK(g_unpins >= 2);
    // no eviction while a reduction is in flight
    const long unpins0 = g_unpins;
    g_active_reductions = 1;
    std::vector<void *> held;
    for (int i = 0; i < 4; ++i) held.push_back(host_alloc(6 * MB));
    for (void *p : held) host_release(p);
    CHECK(g_unpins == unpins0 && c.cached > 10 * MB);
    g_active_reductions = 0;
    void *x = host_alloc(6 * MB);
    host_release(x);                                         // now the excess goes
    CHECK(c.cached <= 10 * MB && g_unpins > unpins0);
    // unpinnable: malloc, freed on release, never cached
    g_pin_fails = true;
    const size_t cached0 = c.cached;
    void *m = host_alloc(64 * MB);
    CHECK(m != nullptr);
    host_release(m);
    CHECK(c.cached == cached0);
    g_pin_fails = false;
    // four threads
    std::vector<std::thread> th;
    for (int t = 0; t < 4; ++t)
        th.emplace_back([t] {
            std::mt19937 rng(t + 7);
            std::vector<void *> mine;
            for (int i = 0; i < 2000; ++i) {
                if (mine.size() < 3 && (rng() & 1)) mine.push_back(host_alloc((rng() % 6 + 1) * MB));
                else if (!mine.empty()) { host_release(mine.back()); mine.pop_back(); }
            }
            for (void *p : mine) host_release(p);
        });
    for (auto &t : th) t.join();
    size_t cached_bytes = 0;
    for (auto &blk : c.free_blocks) cached_bytes += blk.second;
    CHECK(c.live.empty() && cached_bytes == c.cached && c.cached <= 10 * MB);
    CHECK(g_pins - g_unpins == (long)c.free_blocks.size());
    printf("fails %d pins %ld unpins %ld\n", fails, g_pins.load(), g_unpins.load());
    return fails != 0;
}
"""


def region(src, begin, end):
    a = src.find(begin)
    b = src.find(end, a)
    assert 0 <= a < b, f"section {begin!r} not found"
    return src[a:b]


def test_host_cache(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    src = open(SRC).read()
    body = (region(src, "struct HostCache {", "\n}  // namespace") + "\n}  // namespace\n"
            + "static std::atomic<int> g_active_reductions{0};\n"
            + region(src, "void *host_alloc(size_t bytes) {", "int planes_alloc(") + "}  // namespace gbla\n")
    cpp = tmp_path / "cache.cpp"
    cpp.write_text(STUBS + body + DRIVER)
    exe = tmp_path / "cache"
    r = subprocess.run([gxx, "-O1", "-g", "-std=c++17", "-pthread", "-fsanitize=thread", str(cpp), "-o", str(exe)],
                       capture_output=True, text=True, timeout=300)
    if r.returncode != 0 and "sanitize" in r.stderr:
        pytest.skip("ThreadSanitizer not available: " + r.stderr[-200:])
    assert r.returncode == 0, r.stderr[-3000:]
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300,
                         env=dict(os.environ, GBLA_HOST_CACHE_MB="10"))
    out = run.stdout + run.stderr
    assert "WARNING: ThreadSanitizer" not in out, out[-3000:]
    assert run.returncode == 0 and "fails 0" in out, out[-3000:]
