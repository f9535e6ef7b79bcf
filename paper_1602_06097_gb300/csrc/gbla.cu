// gbla.cu -- C ABI entry points and the host orchestration of one reduction.
//
// One call runs the whole Faugere-Lachartre reduction (GBLA paper Sec. 4.1,
// new order of Sec. 4.3) on the caller's stream:
//   step 1  pivot analysis and split (split.cu)
//   step 2' X = C * A^-1 by the blocked multiline solve (solve.cu)
//   step 3' D <- D - X * B, exact tensor-core product (modgemm.cu)
//   step 4  reduced echelon form of D' (solve.cu)
//   (RREF)  Y = A^-1 * B, Y <- Y - Y[:, P_D] * RREF(D')   (second FL pass)
//   step 5  output in the input column order, rows by pivot column.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "internal.cuh"
#include "solve.cuh"
#include "split.cuh"

namespace gbla {

static thread_local char g_last_err[512];
thread_local long long g_launches = 0;
thread_local long long g_pair_launches = 0;

void set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
    snprintf(g_last_err, sizeof(g_last_err), "%s (%s) at %s:%d: %s", cudaGetErrorName(e), what, file, line,
             cudaGetErrorString(e));
}

// ------------------------------------------------------------- memory
static std::once_flag g_pool_once;

static void setup_pool() {
    std::call_once(g_pool_once, [] {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = ~0ull;   // keep freed blocks for reuse by later calls
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    });
}

// Host-side fault injection: every device and host allocation of the library
// counts against one process-wide counter; once armed with n (the environment
// switch GBLA_FAULT_ALLOC_AFTER=n at the first allocation, or
// gbla_selftest_fail_alloc_after), the allocation that follows the next n
// fails once, as if the memory were exhausted.  Tests use it to drive every
// error path of a reduction and check that it releases what it holds.
static std::atomic<long long> g_fault_at{-1};   // allocation index that fails
static std::atomic<long long> g_alloc_count{0};
static std::once_flag g_fault_env_once;

bool inject_alloc_fault() {
    std::call_once(g_fault_env_once, [] {
        const char *e = getenv("GBLA_FAULT_ALLOC_AFTER");
        if (e && atoll(e) >= 0) g_fault_at = atoll(e);
    });
    const long long at = g_fault_at.load();
    const long long i = g_alloc_count.fetch_add(1);
    if (at < 0 || i != at) return false;
    long long expect = at;
    g_fault_at.compare_exchange_strong(expect, -1);   // one shot
    return true;
}

cudaError_t out_malloc(void **ptr, size_t bytes) {
    *ptr = nullptr;
    if (inject_alloc_fault()) return cudaErrorMemoryAllocation;
    return cudaMalloc(ptr, bytes);
}

int dalloc(void **ptr, size_t bytes, cudaStream_t s) {
    *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    if (inject_alloc_fault()) {
        set_last_cuda_error(cudaErrorMemoryAllocation, "injected allocation fault", __FILE__, __LINE__);
        return GBLA_E_NOMEM;
    }
    cudaError_t e = cudaMallocAsync(ptr, bytes, s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e, "cudaMallocAsync", __FILE__, __LINE__);
        cudaGetLastError();
        *ptr = nullptr;
        return GBLA_E_NOMEM;
    }
    return GBLA_OK;
}

void dfree(void *ptr, cudaStream_t s) {
    if (ptr) cudaFreeAsync(ptr, s);
}

// Host results live in page-locked memory so that the device-to-host copy runs
// at full link speed.  Pinning is expensive (the pages are locked one by one),
// so released blocks are cached and handed to later results of a similar size
// (a block of 1 to 2 times the rounded request); at most GBLA_HOST_CACHE_MB
// (default 8192) megabytes stay cached, the oldest evicted first.  Blocks that
// cannot be pinned fall back to malloc.
namespace {
struct HostCache {
    std::mutex mu;
    std::vector<std::pair<void *, size_t>> free_blocks;  // cached, unused
    std::vector<std::pair<void *, size_t>> live;         // handed out, pinned
    size_t cached = 0;
    size_t cap = 0;
};
HostCache &host_cache() {
    static HostCache *c = [] {
        auto *h = new HostCache();
        const char *e = getenv("GBLA_HOST_CACHE_MB");
        const long long mb = e ? atoll(e) : 8192;
        h->cap = (size_t)(mb > 0 ? mb : 0) << 20;
        return h;
    }();
    return *c;
}
}  // namespace

static std::atomic<int> g_active_reductions{0};

// Readbacks of sizes, indices and status words go through a page-locked
// buffer per host thread: a device-to-host copy into pageable memory is staged
// by the driver and was measured to block for 20 s while another thread's
// reduction ran (two batch workers); into page-locked memory it does not.
struct Scratch {
    void *p = nullptr;
    size_t cap = 0;
};
static thread_local Scratch g_scratch;

int readback(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return GBLA_OK;
    if (g_scratch.cap < bytes) {
        size_t want = (size_t)1 << 20;
        while (want < bytes) want <<= 1;
        void *np = nullptr;
        if (cudaHostAlloc(&np, want, cudaHostAllocDefault) == cudaSuccess) {
            // freeing page-locked memory waits for an idle device: the
            // outgrown buffer is kept while other reductions are in flight
            if (g_scratch.p && g_active_reductions.load() <= 1) cudaFreeHost(g_scratch.p);
            g_scratch.p = np;
            g_scratch.cap = want;
        } else {
            cudaGetLastError();
        }
    }
    if (g_scratch.cap >= bytes) {
        GBLA_CUDA_TRY(cudaMemcpyAsync(g_scratch.p, src, bytes, cudaMemcpyDeviceToHost, s));
        GBLA_CUDA_TRY(cudaStreamSynchronize(s));
        memcpy(dst, g_scratch.p, bytes);
    } else {   // no page-locked memory: copy directly
        GBLA_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
        GBLA_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return GBLA_OK;
}

struct ActiveReduction {
    ActiveReduction() { ++g_active_reductions; }
    ~ActiveReduction() { --g_active_reductions; }
};

// Reductions on different streams run their device work concurrently (the
// batch workers and the server's requests overlap on the GPU).  With
// GBLA_SERIALIZE=1 in the environment a process-wide lock makes them follow
// one another instead (kept for diagnosis: an earlier version of the library
// stalled for tens of seconds with overlapping reductions; the current one,
// traced around every host synchronisation and allocation, does not).
static std::mutex g_device_mu;
static bool serialize_reductions() {
    static const bool v = [] {
        const char *e = getenv("GBLA_SERIALIZE");
        return e && atoi(e) != 0;
    }();
    return v;
}

void *host_alloc(size_t bytes) {
    if (inject_alloc_fault()) return nullptr;
    if (bytes == 0) bytes = 16;
    const size_t want = round_up((int64_t)bytes, 1 << 21);
    HostCache &c = host_cache();
    {
        std::lock_guard<std::mutex> lk(c.mu);
        size_t best = (size_t)-1;
        for (size_t i = 0; i < c.free_blocks.size(); ++i) {
            const size_t sz = c.free_blocks[i].second;
            if (sz >= want && sz <= 2 * want && (best == (size_t)-1 || sz < c.free_blocks[best].second)) best = i;
        }
        if (best != (size_t)-1) {
            auto blk = c.free_blocks[best];
            c.free_blocks.erase(c.free_blocks.begin() + (long)best);
            c.cached -= blk.second;
            c.live.push_back(blk);
            return blk.first;
        }
    }
    void *ptr = nullptr;
    if (cudaHostAlloc(&ptr, want, cudaHostAllocDefault) == cudaSuccess) {
        std::lock_guard<std::mutex> lk(c.mu);
        c.live.emplace_back(ptr, want);
        return ptr;
    }
    cudaGetLastError();
    return malloc(bytes);
}

void host_release(void *ptr) {
    if (!ptr) return;
    HostCache &c = host_cache();
    std::vector<void *> drop;
    {
        std::lock_guard<std::mutex> lk(c.mu);
        size_t i = 0;
        while (i < c.live.size() && c.live[i].first != ptr) ++i;
        if (i == c.live.size()) {   // a malloc fallback block
            free(ptr);
            return;
        }
        auto blk = c.live[i];
        c.live.erase(c.live.begin() + (long)i);
        c.free_blocks.push_back(blk);
        c.cached += blk.second;
        // evict the oldest; freeing page-locked memory also waits for an idle
        // device, so not while reductions are in flight
        while (c.cached > c.cap && !c.free_blocks.empty() && g_active_reductions.load() == 0) {
            drop.push_back(c.free_blocks.front().first);
            c.cached -= c.free_blocks.front().second;
            c.free_blocks.erase(c.free_blocks.begin());
        }
    }
    for (void *d : drop) cudaFreeHost(d);
}

int planes_alloc(Planes *pl, int64_t rows, int64_t k, int nplanes, cudaStream_t s) {
    pl->rows = round_up(rows > 0 ? rows : 1, 128);
    pl->kp = round_up(k > 0 ? k : 1, 128);
    pl->nplanes = nplanes;
    pl->ptr = nullptr;
    return dalloc(reinterpret_cast<void **>(&pl->ptr), pl->plane_elems() * (size_t)nplanes * sizeof(__nv_bfloat16), s);
}

void planes_free(Planes *pl, cudaStream_t s) {
    dfree(pl->ptr, s);
    pl->ptr = nullptr;
}

static int planes_zero(const Planes &pl, cudaStream_t s) {
    if (!pl.ptr) return GBLA_OK;
    GBLA_CUDA_TRY(cudaMemsetAsync(pl.ptr, 0, pl.plane_elems() * (size_t)pl.nplanes * sizeof(__nv_bfloat16), s));
    return GBLA_OK;
}

bool is_prime(uint32_t p) {
    if (p < 2) return false;
    for (uint32_t d = 2; d * d <= p; ++d)
        if (p % d == 0) return false;
    return true;
}

int check_device() {
    int dev = 0, major = 0, minor = 0, n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        return GBLA_E_UNSUPPORTED;
    }
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) return GBLA_E_UNSUPPORTED;   // built for sm_103a only
    setup_pool();
    return GBLA_OK;
}

int map_dev_err(uint32_t e) {
    if (e & DEV_ERR_TIMEOUT) return GBLA_E_TIMEOUT;
    if (e & DEV_ERR_INVAL) return GBLA_E_INVAL;
    if (e & DEV_ERR_INTERNAL) return GBLA_E_INTERNAL;
    return GBLA_OK;
}

// ------------------------------------------------------- output assembly
__global__ void mark_pivot_cols_kernel(int64_t npiv, const int32_t *__restrict__ pivcol_orig, int64_t *outflag) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < npiv) outflag[pivcol_orig[k]] = 1;
}

__global__ void mark_bottom_cols_kernel(int64_t rank_d, const int32_t *__restrict__ pcol,
                                        const int32_t *__restrict__ npcol_orig, int64_t *outflag) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < rank_d) outflag[npcol_orig[pcol[k]]] = 1;
}

__device__ __forceinline__ int64_t warp_count_nz(const uint16_t *row, int64_t n, int lane) {
    int64_t c = 0;
    for (int64_t i = lane; i < n; i += 32) c += row[i] != 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    return c;
}

// counts of the top rows: echelon form = input row length; RREF = 1 + nnz(Y row)
__global__ void top_counts_kernel(int64_t npiv, const int32_t *__restrict__ piv_row, const int32_t *__restrict__ pivcol_orig,
                                  const int64_t *__restrict__ row_ptr, const uint16_t *__restrict__ Y, int64_t ldy,
                                  int64_t n_d, const int64_t *__restrict__ outpos, int64_t *cnt) {
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= npiv) return;
    int64_t c;
    if (Y) c = 1 + warp_count_nz(Y + k * ldy, n_d, lane);
    else c = row_ptr[piv_row[k] + 1] - row_ptr[piv_row[k]];
    if (lane == 0) cnt[outpos[pivcol_orig[k]]] = c;
}

__global__ void bottom_counts_kernel(int64_t rank_d, const int32_t *__restrict__ prow, const int32_t *__restrict__ pcol,
                                     const int32_t *__restrict__ npcol_orig, const uint16_t *__restrict__ D, int64_t ldd,
                                     int64_t n_d, const int64_t *__restrict__ outpos, int64_t *cnt) {
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= rank_d) return;
    const int64_t c = warp_count_nz(D + (prow ? (int64_t)prow[k] : k) * ldd, n_d, lane);
    if (lane == 0) cnt[outpos[npcol_orig[pcol[k]]]] = c;
}

// Compact the nonzeros of a dense row (columns = permuted non-pivot indices,
// increasing input columns) into (col, val) at out_off.
__device__ __forceinline__ void warp_compact(const uint16_t *row, int64_t n, const int32_t *__restrict__ npcol_orig,
                                             int32_t *ocol, uint16_t *oval, int64_t out_off, int lane) {
    int64_t off = out_off;
    for (int64_t base = 0; base < n; base += 32) {
        const int64_t i = base + lane;
        const uint16_t v = (i < n) ? row[i] : 0;
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, v != 0);
        if (v) {
            const int64_t pos = off + __popc(bal & ((1u << lane) - 1u));
            ocol[pos] = npcol_orig[i];
            oval[pos] = v;
        }
        off += __popc(bal);
    }
}

__global__ void top_fill_kernel(int64_t npiv, const int32_t *__restrict__ piv_row, const int32_t *__restrict__ pivcol_orig,
                                const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                const uint16_t *__restrict__ val, const uint32_t *__restrict__ inv_lead,
                                const uint16_t *__restrict__ Y, int64_t ldy, int64_t n_d,
                                const int32_t *__restrict__ npcol_orig, const int64_t *__restrict__ outpos,
                                const int64_t *__restrict__ orp, int32_t *ocol, uint16_t *oval, ModP mp) {
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= npiv) return;
    const int64_t off = orp[outpos[pivcol_orig[k]]];
    if (Y) {
        if (lane == 0) {
            ocol[off] = pivcol_orig[k];
            oval[off] = 1;
        }
        warp_compact(Y + k * ldy, n_d, npcol_orig, ocol, oval, off + 1, lane);
    } else {
        const int64_t r = piv_row[k];
        const int64_t b = row_ptr[r], e = row_ptr[r + 1];
        const uint32_t inv = inv_lead[k];
        for (int64_t i = b + lane; i < e; i += 32) {
            ocol[off + (i - b)] = col[i];
            oval[off + (i - b)] = (uint16_t)mulmod(val[i], inv, mp);
        }
    }
}

__global__ void bottom_fill_kernel(int64_t rank_d, const int32_t *__restrict__ prow, const int32_t *__restrict__ pcol,
                                   const int32_t *__restrict__ npcol_orig, const uint16_t *__restrict__ D, int64_t ldd,
                                   int64_t n_d, const int64_t *__restrict__ outpos, const int64_t *__restrict__ orp,
                                   int32_t *ocol, uint16_t *oval) {
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= rank_d) return;
    const int64_t off = orp[outpos[npcol_orig[pcol[k]]]];
    warp_compact(D + (prow ? (int64_t)prow[k] : k) * ldd, n_d, npcol_orig, ocol, oval, off, lane);
}

// Bottom rows from the reduced rows' non-pivot part Rnp (row k = RREF row k of
// D'): the row is the pivot entry (pcol[k], 1) followed by the nonzeros of
// Rnp[k] in column order (its entries left of the lead are zero).  A warp per
// row; a lane loads 8 residues at a time (rows of Rnp are 128-byte aligned).
__device__ __forceinline__ void load8_np(const uint16_t *row, int64_t i0, int64_t nnp, uint16_t (&v)[8]) {
    if (i0 + 8 <= nnp) {
        const uint4 x = __ldg(reinterpret_cast<const uint4 *>(row + i0));
        const uint32_t u[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = (uint16_t)(u[e >> 1] >> ((e & 1) * 16));
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = i0 + e < nnp ? row[i0 + e] : (uint16_t)0;
    }
}

__global__ void bottom_counts_np_kernel(int64_t rank_d, const int32_t *__restrict__ pcol,
                                        const int32_t *__restrict__ npcol_orig, const uint16_t *__restrict__ Rnp,
                                        int64_t ldnp, int64_t nnp, const int64_t *__restrict__ outpos, int64_t *cnt) {
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= rank_d) return;
    const uint16_t *row = Rnp + k * ldnp;
    int64_t c = 0;
    for (int64_t i0 = (int64_t)lane * 8; i0 < nnp; i0 += 256) {
        uint16_t v[8];
        load8_np(row, i0, nnp, v);
#pragma unroll
        for (int e = 0; e < 8; ++e) c += v[e] != 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    if (lane == 0) cnt[outpos[npcol_orig[pcol[k]]]] = 1 + c;
}

// Input column of each non-pivot column of D': ocolmap[i] = npcol_orig[npc[i]].
__global__ void np_colmap_kernel(int64_t nnp, const int32_t *__restrict__ npc, const int32_t *__restrict__ npcol_orig,
                                 int32_t *__restrict__ ocolmap) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nnp) ocolmap[i] = npcol_orig[npc[i]];
}

__global__ void bottom_fill_np_kernel(int64_t rank_d, const int32_t *__restrict__ pcol,
                                      const int32_t *__restrict__ npcol_orig, const uint16_t *__restrict__ Rnp,
                                      int64_t ldnp, const int32_t *__restrict__ ocolmap, int64_t nnp,
                                      const int64_t *__restrict__ outpos, const int64_t *__restrict__ orp,
                                      int32_t *ocol, uint16_t *oval) {
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= rank_d) return;
    const int32_t pc = npcol_orig[pcol[k]];
    const int64_t off = orp[outpos[pc]];
    if (lane == 0) {
        ocol[off] = pc;
        oval[off] = 1;
    }
    warp_compact(Rnp + k * ldnp, nnp, ocolmap, ocol, oval, off + 1, lane);
}

__global__ void transpose_u16_kernel(const uint16_t *__restrict__ src, int64_t lds, int64_t rows, int64_t cols,
                                     uint16_t *__restrict__ dst, int64_t ldd) {
    __shared__ uint16_t t[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        t[i][threadIdx.x] = (r < rows && c < cols) ? src[r * lds + c] : 0;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < rows) dst[c * ldd + r] = t[threadIdx.x][i];
    }
}

// ------------------------------------------------------------ one call
// Phase markers for profilers (NVTX ranges "gbla.<phase>"; no cost without
// an attached tool).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

struct Timer {
    cudaEvent_t ev[8];
    int n = 0;
    bool on = false;
    void init(bool enable) {
        on = enable;
        if (on)
            for (auto &e : ev) cudaEventCreate(&e);
    }
    void mark(cudaStream_t s) {   // events 0..6 mark the phases; 7 is recorded inside the echelon
        if (on && n < 7) cudaEventRecord(ev[n++], s);
    }
    double ms(int a, int b) {
        float t = 0;
        if (!on || b >= n) return 0;
        cudaEventElapsedTime(&t, ev[a], ev[b]);
        return t;
    }
    ~Timer() {
        if (on)
            for (auto &e : ev) cudaEventDestroy(e);
    }
};

// GBLA_LOG=1 in the environment: one line per reduction on stderr with the
// planner's choices (path, order, product variant, leaf width), the block
// shapes, the compacted list sizes and the phase times.
static bool log_enabled() {
    static const bool v = [] {
        const char *e = getenv("GBLA_LOG");
        return e && atoi(e) != 0;
    }();
    return v;
}

// A second stream (and a fork/join event pair) per host thread, for work of
// one reduction that can overlap its main stream.
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    int dev = -1;
    bool get() {
        int d = 0;
        if (cudaGetDevice(&d) != cudaSuccess) return false;
        if (s && dev == d) return true;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            s = nullptr;
            return false;
        }
        dev = d;
        return true;
    }
};
static thread_local SideStream g_side;

void release_thread_resources() {
    if (g_side.s) {
        cudaStreamDestroy(g_side.s);
        cudaEventDestroy(g_side.fork);
        cudaEventDestroy(g_side.join);
        g_side = SideStream{};
    }
    // freeing page-locked memory waits for an idle device: left allocated
    // while reductions of other threads are in flight
    if (g_scratch.p && g_active_reductions.load() == 0) {
        cudaFreeHost(g_scratch.p);
        g_scratch = Scratch{};
    }
}

// Column width of the tensor-core leaf solves of C*A^-1: env GBLA_TRSM_LEAF
// (128, 256, 512 or 1024), else 0 = chosen per matrix (trsm_leaf_for).
static int trsm_leaf_width() {
    static const int v = [] {
        const char *e = getenv("GBLA_TRSM_LEAF");
        const int x = e ? atoi(e) : 0;
        return (x == 128 || x == 256 || x == 512 || x == 1024) ? x : 0;
    }();
    return v;
}

// Wider leaves mean fewer, larger products and two fewer levels of small block
// updates, for a little more product work and larger diagonal-block inverses:
// 1024 columns once there are enough pivots to fill them, else 512.  An
// explicit option wins over the environment.
static int trsm_leaf_for(int64_t npiv, int opt_leaf) {
    if (opt_leaf == 128 || opt_leaf == 256 || opt_leaf == 512 || opt_leaf == 1024) return opt_leaf;
    const int v = trsm_leaf_width();
    return v > 0 ? v : (npiv >= 4096 ? 1024 : 512);
}

// Row width of the leaves of the back-substitution of the echelon form (env
// GBLA_BACK_LEAF overrides: 128, 256, 512 or 1024).
static int back_leaf_width() {
    static const int v = [] {
        const char *e = getenv("GBLA_BACK_LEAF");
        const int x = e ? atoi(e) : 0;
        return (x == 128 || x == 256 || x == 512 || x == 1024) ? x : 512;
    }();
    return v;
}

// ------------------------------------------------------------ autotuner
// With gbla_options.autotune the choices a caller leaves open are made per
// shape bucket (rows, columns and density rounded to powers of two) by
// measurement.  The candidates differ only in how the same exact result is
// computed: the sparse path with leaves of 512 or 1024 columns, with raster
// groups of 4 or 8 row tiles in the gathered product, and (for matrices of at
// most 20,000 rows) the dense path.  The first calls of a bucket claim the
// candidates one by one as trials; a call that finds every candidate claimed
// but not all timed runs the default; once all are timed (event-timed whole
// reduction, a failed trial counts as infinitely slow) every later call runs
// the fastest.
namespace {
struct TuneCand {
    int path, leaf, group_m;
};
struct TuneBucket {
    std::vector<TuneCand> cands;
    std::vector<double> ms;
    int claimed = 0, timed = 0, best = -1;
};
std::mutex g_tune_mu;
std::map<uint64_t, TuneBucket> g_tune;

uint64_t tune_key(int64_t m, int64_t n, int64_t nnz, bool free_path, bool free_leaf) {
    auto lg = [](double x) { return (uint64_t)std::ceil(std::log2(x < 1.0 ? 1.0 : x)); };
    const double dens = (double)nnz / ((double)(m > 0 ? m : 1) * (double)(n > 0 ? n : 1));
    return lg((double)m) | lg((double)n) << 8 | lg(1.0 / (dens > 1e-12 ? dens : 1e-12)) << 16 |
           (uint64_t)free_path << 24 | (uint64_t)free_leaf << 25;
}

struct TuneTicket {
    uint64_t key = 0;
    int idx = -1;   // candidate run (-1: none)
    int state = 0;  // gbla_stats.tune_state
    TuneCand cand{GBLA_PATH_AUTO, 0, 0};
};

TuneTicket tune_pick(int64_t m, int64_t n, int64_t nnz, bool free_path, bool free_leaf) {
    TuneTicket t;
    t.key = tune_key(m, n, nnz, free_path, free_leaf);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TuneBucket &b = g_tune[t.key];
    if (b.cands.empty()) {
        const int path0 = free_path ? GBLA_PATH_SPARSE : GBLA_PATH_AUTO;
        const int gm0 = gather_group_m_default();
        for (int leaf : {512, 1024})
            for (int gm : {gm0, 2 * gm0}) {
                if (!free_leaf && leaf != 512) continue;
                b.cands.push_back({path0, free_leaf ? leaf : 0, gm});
            }
        if (free_path && m <= 20000) b.cands.push_back({GBLA_PATH_DENSE, 0, 0});
        b.ms.assign(b.cands.size(), -1.0);
    }
    if (b.best >= 0) {
        t.idx = b.best;
        t.state = 2;
    } else if (b.claimed < (int)b.cands.size()) {
        t.idx = b.claimed++;
        t.state = 1;
    } else {
        t.state = 3;   // trials in flight: the default
        return t;
    }
    t.cand = b.cands[(size_t)t.idx];
    return t;
}

void tune_report(const TuneTicket &t, double ms) {
    if (t.state != 1) return;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TuneBucket &b = g_tune[t.key];
    if (b.ms[(size_t)t.idx] >= 0.0) return;
    b.ms[(size_t)t.idx] = ms;
    if (++b.timed == (int)b.cands.size()) {
        b.best = 0;
        for (size_t i = 1; i < b.ms.size(); ++i)
            if (b.ms[i] < b.ms[(size_t)b.best]) b.best = (int)i;
    }
}

// Sets the gathered product's raster group for this thread while in scope.
struct GroupOverride {
    int prev;
    explicit GroupOverride(int v) : prev(g_gather_group_m_override) {
        if (v > 0) g_gather_group_m_override = v;
    }
    ~GroupOverride() { g_gather_group_m_override = prev; }
};
}  // namespace

int reduce_impl(const gbla_csr_in *in, uint32_t p, const gbla_options *opt, cudaStream_t s, gbla_csr_out *out,
                int64_t *rank_out, gbla_stats *stats) {
    const int want_reduced = opt ? opt->want_reduced : 0;
    const int variant = opt ? opt->gemm_variant : GBLA_GEMM_AUTO;
    const int device_ptrs = opt ? opt->device_ptrs : 0;
    const int path_req = opt ? opt->path : GBLA_PATH_AUTO;
    const bool ktimes = opt && opt->kernel_times && stats;
    const int leaf_req = opt ? opt->leaf_width : 0;
    const bool autotune = opt && opt->autotune;
    const int echelon_opt = opt ? opt->echelon : GBLA_ECHELON_AUTO;
    if (variant < 0 || variant > GBLA_GEMM_U8) return GBLA_E_INVAL;
    if (path_req < GBLA_PATH_AUTO || path_req > GBLA_PATH_SPARSE) return GBLA_E_INVAL;
    // FP64 and U8 name the pipe of the Schur update on the dense path; every
    // other product of the reduction runs on the tcgen05 tensor cores.
    const bool alt_schur = variant == GBLA_GEMM_FP64 || variant == GBLA_GEMM_U8;
    // Order of the FL steps: the new order (Sec. 4.3: X = C A^-1, then
    // D <- D - X B) or the original one (Sec. 4.1 steps 2-3: B <- A^-1 B
    // first, then D <- D - C B), which saves the solve with C when the
    // reduced form needs A^-1 B anyway.  The original order runs on the dense
    // path.
    const int order_opt = opt ? opt->fl_order : GBLA_ORDER_NEW;
    if (order_opt != GBLA_ORDER_NEW && order_opt != GBLA_ORDER_TRSM_FIRST) return GBLA_E_INVAL;
    const bool trsm_first = order_opt == GBLA_ORDER_TRSM_FIRST;
    const int pvariant = alt_schur ? GBLA_GEMM_TCGEN05 : variant;
    if (leaf_req != 0 && leaf_req != 128 && leaf_req != 256 && leaf_req != 512 && leaf_req != 1024)
        return GBLA_E_INVAL;
    if (echelon_opt < GBLA_ECHELON_AUTO || echelon_opt > GBLA_ECHELON_SGE) return GBLA_E_INVAL;
    const int64_t m = in->nrows, n = in->ncols, nnz = in->nnz;
    if (m < 0 || n < 0 || nnz < 0 || m >= (1ll << 31) || n >= (1ll << 31)) return GBLA_E_INVAL;
    if (m > 0 && !in->row_ptr) return GBLA_E_INVAL;
    if (nnz > 0 && (!in->col || !in->val)) return GBLA_E_INVAL;
    GBLA_TRY(check_device());
    std::unique_lock<std::mutex> device_lock(g_device_mu, std::defer_lock);
    if (serialize_reductions()) device_lock.lock();
    const ActiveReduction active;
    const ModP mp = make_modp(p);
    // diagonal blocks of the triangular solve on the tensor cores too
    const bool tc_leaves =
        pvariant == GBLA_GEMM_TCGEN05 || (pvariant == GBLA_GEMM_AUTO && p >= 8 && tc_supported());
    // The sparse path keeps A and B sparse and runs C*A^-1 and the Schur
    // update as K-compacted tensor-core products; it needs the tensor-core
    // variant.  The dense path materialises A and B (and serves p < 8 and the
    // exact SIMT variant).
    const bool tc_ok = pvariant != GBLA_GEMM_SIMT && p >= 8 && tc_supported();
    if (path_req == GBLA_PATH_SPARSE && (!tc_ok || alt_schur || trsm_first)) return GBLA_E_UNSUPPORTED;
    if (alt_schur && !tc_ok) return GBLA_E_UNSUPPORTED;
    // choices left open, made by the autotuner where it applies
    TuneTicket tune;
    if (autotune && tc_ok && !alt_schur && !trsm_first && (path_req == GBLA_PATH_AUTO || leaf_req == 0))
        tune = tune_pick(m, n, nnz, path_req == GBLA_PATH_AUTO, leaf_req == 0);
    const int path_opt = (tune.idx >= 0 && path_req == GBLA_PATH_AUTO) ? tune.cand.path : path_req;
    const int leaf_opt = (tune.idx >= 0 && leaf_req == 0) ? tune.cand.leaf : leaf_req;
    const GroupOverride group_override(tune.idx >= 0 ? tune.cand.group_m : 0);
    const bool sparse = tc_ok && path_opt != GBLA_PATH_DENSE && !alt_schur && !trsm_first;
    int tc_leaf_w = 512;
    GemmCounters ctr;
    const long long launches0 = g_launches, pair_launches0 = g_pair_launches;
    Timer tm;
    const bool log_on = log_enabled();
    tm.init(stats != nullptr || log_on || tune.state == 1);
    tm.mark(s);

    // Everything below allocates from the stream-ordered pool; `cleanup`
    // releases it on every path.
    int rc = GBLA_OK;
    uint32_t *err = nullptr;
    unsigned long long *exec_ctr = nullptr;   // executed list entries x row tiles of the Schur launch
    unsigned long long *tc_work = nullptr;    // dense product tile work (kernel timing)
    KernelTimeTotals kt;
    int64_t *d_rp = nullptr;
    int32_t *d_col = nullptr;
    uint16_t *d_val = nullptr;
    PivotInfo pi;
    Multiline ml;
    Planes At{}, Arow{}, Bt{}, Xp{}, Xq{}, RdT{}, XpdT{}, Zt{}, Ct{}, XT{}, Cp{}, Yb{}, Zr{}, CtL{};
    bool need_zr = false;   // the solve with B takes tensor-core leaves
    double d_density = -1.0;
    int sge_done = 0;
    Compact SA, SB;
    uint16_t *Adiag = nullptr;
    uint16_t *C16 = nullptr, *D16 = nullptr, *Bt16 = nullptr, *Y16 = nullptr, *R16 = nullptr;
    EchelonD::NonPivot np_d;   // the reduced rows of D' at its non-pivot columns (output without R16)
    int32_t *np_ocol = nullptr;   // input column of each of them
    uint16_t *A16 = nullptr, *B16 = nullptr;
    int32_t *is_piv_row = nullptr, *prow = nullptr, *pcol = nullptr;
    int64_t *outflag = nullptr, *outpos = nullptr, *cnt = nullptr, *orp = nullptr;
    int32_t *ocol = nullptr;
    uint16_t *oval = nullptr;
    int64_t rank_d = 0, npiv = 0, m_cd = 0, n_d = 0, rank = 0, onnz = 0;
    int64_t ldc = 0, ldd = 0, ldbt = 0;
    DevCSR dc;
    std::vector<int32_t> lead_h;
    double schur_ops = 0;
    bool side_pending = false;   // work on g_side.s not yet joined into s

#define STEP(expr)                 \
    do {                           \
        rc = (expr);               \
        if (rc != GBLA_OK) goto cleanup; \
    } while (0)
#define CSTEP(expr)                                               \
    do {                                                          \
        cudaError_t _e = (expr);                                  \
        if (_e != cudaSuccess) {                                  \
            set_last_cuda_error(_e, #expr, __FILE__, __LINE__);   \
            rc = _e == cudaErrorMemoryAllocation ? GBLA_E_NOMEM : GBLA_E_CUDA; \
            goto cleanup;                                         \
        }                                                         \
    } while (0)

    STEP(dalloc_t(&err, 4, s));
    CSTEP(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
    if (ktimes) {
        STEP(dalloc_t(&tc_work, 1, s));
        CSTEP(cudaMemsetAsync(tc_work, 0, sizeof(unsigned long long), s));
        kernel_times_begin(tc_work);
    }
    if (device_ptrs) {
        dc.row_ptr = in->row_ptr;
        dc.col = in->col;
        dc.val = in->val;
    } else {
        STEP(dalloc_t(&d_rp, (size_t)m + 1, s));
        STEP(dalloc_t(&d_col, (size_t)nnz + 1, s));
        STEP(dalloc_t(&d_val, (size_t)nnz + 1, s));
        if (m > 0) CSTEP(cudaMemcpyAsync(d_rp, in->row_ptr, sizeof(int64_t) * (size_t)(m + 1), cudaMemcpyHostToDevice, s));
        if (nnz > 0) {
            // two copy streams: the values and the first quarter of the
            // columns on the side stream, the rest of the columns here
            const int64_t c0 = g_side.get() ? nnz / 4 : 0;
            if (c0 > 0) {
                CSTEP(cudaEventRecord(g_side.fork, s));
                CSTEP(cudaStreamWaitEvent(g_side.s, g_side.fork, 0));
                side_pending = true;
                CSTEP(cudaMemcpyAsync(d_val, in->val, sizeof(uint16_t) * (size_t)nnz, cudaMemcpyHostToDevice, g_side.s));
                CSTEP(cudaMemcpyAsync(d_col, in->col, sizeof(int32_t) * (size_t)c0, cudaMemcpyHostToDevice, g_side.s));
                CSTEP(cudaEventRecord(g_side.join, g_side.s));
            } else {
                CSTEP(cudaMemcpyAsync(d_val, in->val, sizeof(uint16_t) * (size_t)nnz, cudaMemcpyHostToDevice, s));
            }
            CSTEP(cudaMemcpyAsync(d_col + c0, in->col + c0, sizeof(int32_t) * (size_t)(nnz - c0), cudaMemcpyHostToDevice,
                                  s));
            if (side_pending) {
                CSTEP(cudaStreamWaitEvent(s, g_side.join, 0));
                side_pending = false;
            }
        }
        dc.row_ptr = d_rp;
        dc.col = d_col;
        dc.val = d_val;
    }
    dc.m = m;
    dc.n = n;
    dc.nnz = nnz;

    // ---- step 1: pivots and split
    nvtxRangePushA("gbla.split");
    rc = pivot_analysis(dc, mp, &pi, err, s);
    nvtxRangePop();
    if (rc != GBLA_OK) goto cleanup;
    npiv = pi.npiv;
    tc_leaf_w = trsm_leaf_for(npiv, leaf_opt);
    m_cd = pi.m_cd;
    n_d = pi.n_d;
    ldc = round_up(npiv > 0 ? npiv : 1, 64);
    ldd = round_up(n_d > 0 ? n_d : 1, 64);
    ldbt = ldc;
    {
        // dense uint16 blocks: C, D (other rows); A, B (pivot rows, normalised)
        // on the dense path, and for the second pass of the reduced form
        const bool dense_ab = !sparse || (want_reduced && npiv > 0 && n_d > 0);
        if (dense_ab) {
            STEP(dalloc_t(&A16, (size_t)(npiv > 0 ? npiv : 1) * (size_t)ldc, s));
            STEP(dalloc_t(&B16, (size_t)(npiv > 0 ? npiv : 1) * (size_t)ldd, s));
        }
        STEP(dalloc_t(&C16, (size_t)(m_cd > 0 ? m_cd : 1) * (size_t)ldc, s));
        STEP(dalloc_t(&D16, (size_t)(m_cd > 0 ? m_cd : 1) * (size_t)ldd, s));
        if (npiv > 0 && dense_ab) {
            CSTEP(cudaMemsetAsync(A16, 0, sizeof(uint16_t) * (size_t)npiv * (size_t)ldc, s));
            CSTEP(cudaMemsetAsync(B16, 0, sizeof(uint16_t) * (size_t)npiv * (size_t)ldd, s));
        }
        if (m_cd > 0) {
            CSTEP(cudaMemsetAsync(C16, 0, sizeof(uint16_t) * (size_t)m_cd * (size_t)ldc, s));
            CSTEP(cudaMemsetAsync(D16, 0, sizeof(uint16_t) * (size_t)m_cd * (size_t)ldd, s));
        }
    }
    STEP(split_scatter(dc, pi, A16, ldc, B16, ldd, C16, ldc, D16, ldd, mp, s));
    // the solve with B (A^-1 B) also takes tensor-core leaves: Z_J as B-operand planes
    need_zr = tc_leaves && (want_reduced || trsm_first) && npiv > 0 && n_d > 0;
    if (need_zr && ((sparse && m_cd > 0) || !sparse)) STEP(planes_alloc(&Zr, round_up(npiv, tc_leaf_w), tc_leaf_w, 4, s));
    if (sparse && m_cd > 0 && npiv > 0) {
        // pivot rows as sparse operands, then the inverses of A's diagonal
        // blocks from their dense copies (on the side stream: the main stream
        // goes on with the second pass's conversions, if any)
        STEP(dalloc_t(&Adiag, (size_t)round_up(npiv, tc_leaf_w) * (size_t)tc_leaf_w, s));
        STEP(sparse_build(dc, pi, tc_leaf_w, Adiag, &SA, &SB, mp, s));
        STEP(planes_alloc(&Zt, round_up(npiv, tc_leaf_w), tc_leaf_w, 4, s));
        if (g_side.get()) {
            CSTEP(cudaEventRecord(g_side.fork, s));
            CSTEP(cudaStreamWaitEvent(g_side.s, g_side.fork, 0));
            side_pending = true;
            rc = upper_leaf_inverses_diag(Adiag, npiv, tc_leaf_w, Zt, mp, err, g_side.s, Zr.ptr ? &Zr : nullptr);
            CSTEP(cudaEventRecord(g_side.join, g_side.s));
            STEP(rc);
        } else {
            STEP(upper_leaf_inverses_diag(Adiag, npiv, tc_leaf_w, Zt, mp, err, s, Zr.ptr ? &Zr : nullptr));
        }
    }
    if (!sparse && npiv > 0 && tc_leaves && ((!trsm_first && m_cd > 0) || need_zr)) {
        // inverses of A's diagonal blocks for the tensor-core leaf solves, on
        // the side stream while the main stream converts A and B
        STEP(planes_alloc(&Zt, round_up(npiv, tc_leaf_w), tc_leaf_w, 4, s));
        if (g_side.get()) {
            CSTEP(cudaEventRecord(g_side.fork, s));
            CSTEP(cudaStreamWaitEvent(g_side.s, g_side.fork, 0));
            side_pending = true;
            rc = upper_leaf_inverses(A16, ldc, npiv, tc_leaf_w, Zt, mp, err, g_side.s, Zr.ptr ? &Zr : nullptr);
            CSTEP(cudaEventRecord(g_side.join, g_side.s));
            STEP(rc);
        } else {
            STEP(upper_leaf_inverses(A16, ldc, npiv, tc_leaf_w, Zt, mp, err, s, Zr.ptr ? &Zr : nullptr));
        }
    }
    // digit planes of the operands the dense products read
    if (!sparse && !trsm_first && m_cd > 0 && npiv > 0) {
        // A^T: B-operand of C <- C - X*A.  The triangular solve reads it only
        // below its diagonal blocks (column of A after row of A), so tiles
        // entirely above the diagonal are not converted.
        STEP(planes_alloc(&At, npiv, npiv, 4, s));
        STEP(to_planes(At, npiv, npiv, A16, ldc, 0, true, nullptr, nullptr, mp, s, nullptr, true));
    }
    if (!sparse && !trsm_first && m_cd > 0 && n_d > 0 && npiv > 0) {
        STEP(planes_alloc(&Bt, n_d, npiv, 4, s));    // B^T: B-operand of D <- D - X*B
        STEP(to_planes(Bt, n_d, npiv, B16, ldd, 0, true, nullptr, nullptr, mp, s));
    }
    if ((want_reduced || trsm_first) && npiv > 0 && n_d > 0) {
        STEP(planes_alloc(&Arow, npiv, npiv, 4, s)); // A: B-operand of the solve with B
        STEP(to_planes(Arow, npiv, npiv, A16, ldc, 0, false, nullptr, nullptr, mp, s));
        STEP(dalloc_t(&Bt16, (size_t)n_d * (size_t)ldbt, s));
        dim3 grid((unsigned)((n_d + 31) / 32), (unsigned)((npiv + 31) / 32));
        transpose_u16_kernel<<<grid, dim3(32, 8), 0, s>>>(B16, ldd, npiv, n_d, Bt16, ldbt);
        CSTEP(launch_check());
    }
    if (side_pending) {
        CSTEP(cudaStreamWaitEvent(s, g_side.join, 0));
        side_pending = false;
    }
    dfree(A16, s);
    dfree(B16, s);
    A16 = B16 = nullptr;
    dfree(Adiag, s);   // the side stream's work is joined into s above
    Adiag = nullptr;
    // the 2-multiline form of A drives the sparse leaf solves: those of the
    // first pass unless they run on the tensor cores, those of the second
    if ((!sparse && !tc_leaves) || ((want_reduced || trsm_first) && !Zr.ptr)) STEP(multiline_build(dc, pi, &ml, mp, s));
    tm.mark(s);  // 1

    // ---- new order: X = C A^-1, then D <- D - X B
    if (sparse && m_cd > 0 && npiv > 0) {
        // X^T as A-operand planes (rows = pivots, K = rows of C), zero where
        // no leaf writes (the staircase left of each row's lead)
        STEP(planes_alloc(&XT, npiv, m_cd, 2, s));
        STEP(planes_zero(XT, s));
        STEP(planes_alloc(&Ct, m_cd, tc_leaf_w, 4, s));
        lead_h.resize((size_t)m_cd);
        STEP(readback(lead_h.data(), pi.cd_lead, sizeof(int32_t) * (size_t)m_cd, s));
        TrsmSparse T{m_cd, npiv, C16, ldc, &SA, &Zt, &Ct, &XT, tc_leaf_w, &mp, err, s, &ctr, pi.cd_lead, &lead_h};
        NvtxRange r("gbla.trsm");
        STEP(trsm_sparse(T));
    } else if (trsm_first) {
        // original order: Y = A^-1 B as the lower solve Y^T A^T = B^T (in place
        // in Bt16), before the Schur update
        if (npiv > 0 && n_d > 0) {
            STEP(planes_alloc(&Xq, n_d, npiv, 2, s));
            STEP(planes_zero(Xq, s));
            if (Zr.ptr && !CtL.ptr) STEP(planes_alloc(&CtL, n_d, tc_leaf_w, 2, s));
            TrsmLower T{n_d, npiv, Bt16, ldbt, &ml, &Xq, &Arow, &mp, pvariant, err, s, &ctr,
                        Zr.ptr ? &Zr : nullptr, Zr.ptr ? &CtL : nullptr, Zr.ptr ? tc_leaf_w : 0};
            NvtxRange r("gbla.trsm");
            STEP(trsm_lower(T));
        }
    } else if (m_cd > 0 && npiv > 0) {
        STEP(planes_alloc(&Xp, m_cd, npiv, 2, s));
        STEP(planes_zero(Xp, s));
        lead_h.resize((size_t)m_cd);
        STEP(readback(lead_h.data(), pi.cd_lead, sizeof(int32_t) * (size_t)m_cd, s));
        if (tc_leaves) STEP(planes_alloc(&Ct, m_cd, tc_leaf_w, 2, s));
        TrsmUpper T{m_cd, npiv, C16, ldc, &ml, &Xp, &At, &mp, pvariant, err, s, &ctr, pi.cd_lead, &lead_h,
                    tc_leaves ? &Zt : nullptr, tc_leaves ? &Ct : nullptr, tc_leaf_w};
        NvtxRange r("gbla.trsm");
        STEP(trsm_upper(T));
    }
    tm.mark(s);  // 2
    if (sparse && m_cd > 0 && npiv > 0 && n_d > 0) {
        NvtxRange r("gbla.schur");
        if (stats) {
            STEP(dalloc_t(&exec_ctr, 1, s));
            CSTEP(cudaMemsetAsync(exec_ctr, 0, sizeof(unsigned long long), s));
        }
        STEP(modgemm_gather(SB, 0, XT, npiv, D16, ldd, m_cd, n_d, -1, pi.cd_lead, mp, err, s, &ctr, exec_ctr));
    } else if (trsm_first && m_cd > 0 && npiv > 0 && n_d > 0) {
        // D <- D - C Y: C's rows are zero left of their leads like X's
        NvtxRange r("gbla.schur");
        lead_h.resize((size_t)m_cd);
        STEP(readback(lead_h.data(), pi.cd_lead, sizeof(int32_t) * (size_t)m_cd, s));
        STEP(planes_alloc(&Cp, m_cd, npiv, 2, s));
        STEP(to_planes(Cp, m_cd, npiv, C16, ldc, 0, false, nullptr, nullptr, mp, s));
        STEP(planes_alloc(&Yb, n_d, npiv, 4, s));
        STEP(to_planes(Yb, n_d, npiv, Bt16, ldbt, 0, false, nullptr, nullptr, mp, s));
        STEP(modgemm(Cp, 0, 0, Yb, 0, 0, D16, ldd, m_cd, n_d, npiv, -1, mp, variant, err, s, &ctr, nullptr,
                     pi.cd_lead, lead_h.data()));
        schur_ops = ctr.last_ops;
        planes_free(&Cp, s);
        planes_free(&Yb, s);
    } else if (m_cd > 0 && npiv > 0 && n_d > 0) {
        NvtxRange r("gbla.schur");
        STEP(modgemm(Xp, 0, 0, Bt, 0, 0, D16, ldd, m_cd, n_d, npiv, -1, mp, variant, err, s, &ctr, nullptr,
                     pi.cd_lead, lead_h.data()));
        schur_ops = ctr.last_ops;
    }
    tm.mark(s);  // 3

    // ---- step 4: RREF of D'
    STEP(dalloc_t(&is_piv_row, (size_t)m_cd + 1, s));
    STEP(dalloc_t(&prow, (size_t)m_cd + 1, s));
    STEP(dalloc_t(&pcol, (size_t)m_cd + 1, s));
    {
        EchelonD E{m_cd, n_d, D16, ldd, is_piv_row, prow, pcol, &R16, &mp, pvariant, err, s, &ctr,
                   tm.on ? tm.ev[7] : nullptr, back_leaf_width(),
                   echelon_opt == GBLA_ECHELON_SGE ? 1 : (echelon_opt == GBLA_ECHELON_AUTO ? 2 : 0),
                   &d_density, &sge_done};
        // the second FL pass reads the dense rows; the output alone does not
        if (!want_reduced) E.np_out = &np_d;
        NvtxRange r("gbla.echelon");
        STEP(echelon_d(E, &rank_d));
    }
    tm.mark(s);  // 4

    // ---- second FL pass: Y = A^-1 B, then clear the columns P_D of Y
    if (want_reduced && npiv > 0 && n_d > 0) {
        if (!trsm_first) {
            STEP(planes_alloc(&Xq, n_d, npiv, 2, s));
            STEP(planes_zero(Xq, s));
            if (Zr.ptr && !CtL.ptr) STEP(planes_alloc(&CtL, n_d, tc_leaf_w, 2, s));
            TrsmLower T{n_d, npiv, Bt16, ldbt, &ml, &Xq, &Arow, &mp, pvariant, err, s, &ctr,
                        Zr.ptr ? &Zr : nullptr, Zr.ptr ? &CtL : nullptr, Zr.ptr ? tc_leaf_w : 0};
            STEP(trsm_lower(T));
        }
        if (rank_d > 0) {
            // Y^T[c][j] -= sum_k RREF(D')[k][c] * Y^T[P_D[k]][j]
            STEP(planes_alloc(&RdT, n_d, rank_d, 2, s));
            STEP(planes_alloc(&XpdT, npiv, rank_d, 4, s));
            STEP(to_planes(RdT, n_d, rank_d, R16, ldd, 0, true, nullptr, nullptr, mp, s));
            STEP(to_planes(XpdT, npiv, rank_d, Bt16, ldbt, 0, true, pcol, nullptr, mp, s));
            STEP(modgemm(RdT, 0, 0, XpdT, 0, 0, Bt16, ldbt, n_d, npiv, rank_d, -1, mp, pvariant, err, s, &ctr));
        }
        STEP(dalloc_t(&Y16, (size_t)npiv * (size_t)ldd, s));
        dim3 grid((unsigned)((npiv + 31) / 32), (unsigned)((n_d + 31) / 32));
        transpose_u16_kernel<<<grid, dim3(32, 8), 0, s>>>(Bt16, ldbt, n_d, npiv, Y16, ldd);
        CSTEP(launch_check());
    } else if (want_reduced && npiv > 0) {
        // no B block: the top rows are unit vectors
        STEP(dalloc_t(&Y16, (size_t)npiv * (size_t)ldd, s));
        CSTEP(cudaMemsetAsync(Y16, 0, sizeof(uint16_t) * (size_t)npiv * (size_t)ldd, s));
    }
    tm.mark(s);  // 5

    // ---- step 5: output in input column order, rows sorted by pivot column
    rank = npiv + rank_d;
    STEP(dalloc_t(&outflag, (size_t)n + 1, s));
    STEP(dalloc_t(&outpos, (size_t)n + 1, s));
    STEP(dalloc_t(&cnt, (size_t)rank + 1, s));
    STEP(dalloc_t(&orp, (size_t)rank + 2, s));
    CSTEP(cudaMemsetAsync(outflag, 0, sizeof(int64_t) * (size_t)(n + 1), s));
    if (npiv > 0) {
        mark_pivot_cols_kernel<<<(unsigned)((npiv + 255) / 256), 256, 0, s>>>(npiv, pi.pivcol_orig, outflag);
        CSTEP(launch_check());
    }
    if (rank_d > 0) {
        mark_bottom_cols_kernel<<<(unsigned)((rank_d + 255) / 256), 256, 0, s>>>(rank_d, pcol, pi.npcol_orig, outflag);
        CSTEP(launch_check());
    }
    STEP(scan_i64(outflag, outpos, n, nullptr, s));
    if (npiv > 0) {
        top_counts_kernel<<<(unsigned)((npiv * 32 + 255) / 256), 256, 0, s>>>(npiv, pi.piv_row, pi.pivcol_orig,
                                                                            dc.row_ptr, Y16, ldd, n_d, outpos, cnt);
        CSTEP(launch_check());
    }
    if (rank_d > 0 && R16) {
        bottom_counts_kernel<<<(unsigned)((rank_d * 32 + 255) / 256), 256, 0, s>>>(rank_d, nullptr, pcol, pi.npcol_orig,
                                                                                  R16, ldd, n_d, outpos, cnt);
        CSTEP(launch_check());
    } else if (rank_d > 0) {
        bottom_counts_np_kernel<<<(unsigned)((rank_d * 32 + 255) / 256), 256, 0, s>>>(
            rank_d, pcol, pi.npcol_orig, np_d.Rnp, np_d.ldnp, np_d.nnp, outpos, cnt);
        CSTEP(launch_check());
    }
    STEP(scan_i64(cnt, orp, rank, orp + rank, s));
    STEP(readback(&onnz, orp + rank, sizeof(int64_t), s));
    STEP(dalloc_t(&ocol, (size_t)onnz + 1, s));
    STEP(dalloc_t(&oval, (size_t)onnz + 1, s));
    if (npiv > 0) {
        top_fill_kernel<<<(unsigned)((npiv * 32 + 255) / 256), 256, 0, s>>>(
            npiv, pi.piv_row, pi.pivcol_orig, dc.row_ptr, dc.col, dc.val, pi.inv_lead, Y16, ldd, n_d, pi.npcol_orig,
            outpos, orp, ocol, oval, mp);
        CSTEP(launch_check());
    }
    if (rank_d > 0 && R16) {
        bottom_fill_kernel<<<(unsigned)((rank_d * 32 + 255) / 256), 256, 0, s>>>(
            rank_d, nullptr, pcol, pi.npcol_orig, R16, ldd, n_d, outpos, orp, ocol, oval);
        CSTEP(launch_check());
    } else if (rank_d > 0) {
        STEP(dalloc_t(&np_ocol, (size_t)(np_d.nnp > 0 ? np_d.nnp : 1), s));
        if (np_d.nnp > 0) {
            np_colmap_kernel<<<(unsigned)((np_d.nnp + 255) / 256), 256, 0, s>>>(np_d.nnp, np_d.npc, pi.npcol_orig,
                                                                               np_ocol);
            CSTEP(launch_check());
        }
        bottom_fill_np_kernel<<<(unsigned)((rank_d * 32 + 255) / 256), 256, 0, s>>>(
            rank_d, pcol, pi.npcol_orig, np_d.Rnp, np_d.ldnp, np_ocol, np_d.nnp, outpos, orp, ocol, oval);
        CSTEP(launch_check());
    }
    {
        // results leave the pool: device results in plain device memory,
        // host results in cached page-locked memory
        out->nrows = rank;
        out->ncols = n;
        out->nnz = onnz;
        if (device_ptrs) {
            out->on_device = 1;
            CSTEP(out_malloc((void **)&out->row_ptr, sizeof(int64_t) * (size_t)(rank + 1)));
            CSTEP(out_malloc((void **)&out->col, sizeof(int32_t) * (size_t)(onnz + 1)));
            CSTEP(out_malloc((void **)&out->val, sizeof(uint16_t) * (size_t)(onnz + 1)));
            CSTEP(cudaMemcpyAsync(out->row_ptr, orp, sizeof(int64_t) * (size_t)(rank + 1), cudaMemcpyDeviceToDevice, s));
            if (onnz > 0) {
                CSTEP(cudaMemcpyAsync(out->col, ocol, sizeof(int32_t) * (size_t)onnz, cudaMemcpyDeviceToDevice, s));
                CSTEP(cudaMemcpyAsync(out->val, oval, sizeof(uint16_t) * (size_t)onnz, cudaMemcpyDeviceToDevice, s));
            }
        } else {
            out->on_device = 0;
            out->row_ptr = (int64_t *)host_alloc(sizeof(int64_t) * (size_t)(rank + 1));
            out->col = (int32_t *)host_alloc(sizeof(int32_t) * (size_t)(onnz + 1));
            out->val = (uint16_t *)host_alloc(sizeof(uint16_t) * (size_t)(onnz + 1));
            if (!out->row_ptr || !out->col || !out->val) { rc = GBLA_E_NOMEM; goto cleanup; }
            CSTEP(cudaMemcpyAsync(out->row_ptr, orp, sizeof(int64_t) * (size_t)(rank + 1), cudaMemcpyDeviceToHost, s));
            if (onnz > 0) {
                // two copy streams, as for the input
                const int64_t c0 = g_side.get() ? onnz / 4 : 0;
                if (c0 > 0) {
                    CSTEP(cudaEventRecord(g_side.fork, s));
                    CSTEP(cudaStreamWaitEvent(g_side.s, g_side.fork, 0));
                    side_pending = true;
                    CSTEP(cudaMemcpyAsync(out->val, oval, sizeof(uint16_t) * (size_t)onnz, cudaMemcpyDeviceToHost,
                                          g_side.s));
                    CSTEP(cudaMemcpyAsync(out->col, ocol, sizeof(int32_t) * (size_t)c0, cudaMemcpyDeviceToHost,
                                          g_side.s));
                    CSTEP(cudaEventRecord(g_side.join, g_side.s));
                } else {
                    CSTEP(cudaMemcpyAsync(out->val, oval, sizeof(uint16_t) * (size_t)onnz, cudaMemcpyDeviceToHost, s));
                }
                CSTEP(cudaMemcpyAsync(out->col + c0, ocol + c0, sizeof(int32_t) * (size_t)(onnz - c0),
                                      cudaMemcpyDeviceToHost, s));
                if (side_pending) {
                    CSTEP(cudaStreamWaitEvent(s, g_side.join, 0));
                    side_pending = false;
                }
            }
        }
    }
    tm.mark(s);  // 6
    CSTEP(cudaStreamSynchronize(s));
    {
        uint32_t herr = 0;
        STEP(readback(&herr, err, sizeof(herr), s));
        rc = map_dev_err(herr);
    }
    if (rc == GBLA_OK) {
        *rank_out = rank;
        if (stats) {
            stats->npiv = npiv;
            stats->m_cd = m_cd;
            stats->n_d = n_d;
            stats->rank_d = rank_d;
            stats->ms_split = tm.ms(0, 1);
            stats->ms_trsm = tm.ms(1, 2);
            stats->ms_schur = tm.ms(2, 3);
            stats->ms_echelon = tm.ms(3, 4);
            if (tm.on && tm.n >= 5) {   // event 7: start of the backward pass of the echelon
                float t = 0;
                if (cudaEventQuery(tm.ev[7]) == cudaSuccess && cudaEventElapsedTime(&t, tm.ev[7], tm.ev[4]) == cudaSuccess)
                    stats->ms_echelon_back = t;
                cudaGetLastError();
            }
            stats->ms_backsub = tm.ms(4, 5);
            stats->ms_output = tm.ms(5, 6);
            stats->ms_total = tm.ms(0, 6);
            stats->mod_ops = ctr.mod_ops;
            stats->launches = g_launches - launches0;
            stats->tc_pair_launches = g_pair_launches - pair_launches0;
            stats->gather_group_m = sparse ? (g_gather_group_m_override ? g_gather_group_m_override
                                                                        : gather_group_m_default())
                                           : 0;
            stats->tune_state = tune.state;
            stats->echelon_method = sge_done ? GBLA_ECHELON_SGE : GBLA_ECHELON_PANELS;
            stats->d_density = d_density;
            stats->schur_mod_ops = schur_ops;
            stats->path = sparse ? GBLA_PATH_SPARSE : GBLA_PATH_DENSE;
            stats->list_a = SA.total;
            stats->list_b = SB.total;
            stats->leaf_width = tc_leaf_w;
            if (exec_ctr) {
                unsigned long long e = 0;
                if (readback(&e, exec_ctr, sizeof(e), s) == GBLA_OK) stats->schur_exec_mod_ops = (double)e * 128.0 * 128.0;
            }
            if (ktimes) {
                kernel_times_end(&kt);
                stats->tc_launches = kt.launches[0];
                stats->gather_launches = kt.launches[1];
                stats->tc_ms = kt.ms[0];
                stats->gather_ms = kt.ms[1];
                unsigned long long w = 0;
                if (readback(&w, tc_work, sizeof(w), s) == GBLA_OK) stats->tc_mod_ops = (double)w;
            }
        }
    }

cleanup:
    if (tune.state == 1) tune_report(tune, rc == GBLA_OK ? tm.ms(0, 6) : 1e30);
    if (log_on) {
        fprintf(stderr,
                "gbla: m=%lld n=%lld nnz=%lld p=%u path=%s order=%s variant=%d reduced=%d leaf=%d npiv=%lld "
                "m_cd=%lld n_d=%lld list_a=%lld list_b=%lld rank_d=%lld rc=%d ms split=%.3f trsm=%.3f schur=%.3f "
                "echelon=%.3f backsub=%.3f output=%.3f total=%.3f\n",
                (long long)m, (long long)n, (long long)nnz, p, sparse ? "sparse" : "dense",
                trsm_first ? "trsm_first" : "new", variant, want_reduced, tc_leaf_w, (long long)npiv, (long long)m_cd,
                (long long)n_d, (long long)SA.total, (long long)SB.total, (long long)rank_d, rc,
                rc == GBLA_OK ? tm.ms(0, 1) : 0.0, rc == GBLA_OK ? tm.ms(1, 2) : 0.0, rc == GBLA_OK ? tm.ms(2, 3) : 0.0,
                rc == GBLA_OK ? tm.ms(3, 4) : 0.0, rc == GBLA_OK ? tm.ms(4, 5) : 0.0, rc == GBLA_OK ? tm.ms(5, 6) : 0.0,
                rc == GBLA_OK ? tm.ms(0, 6) : 0.0);
    }
    if (ktimes && rc != GBLA_OK) kernel_times_end(&kt);
    if (side_pending) {   // nothing the side stream uses may be freed before it is done
        cudaStreamSynchronize(g_side.s);
        cudaGetLastError();
    }
    dfree(err, s);
    dfree(exec_ctr, s);
    dfree(tc_work, s);
    dfree(d_rp, s);
    dfree(d_col, s);
    dfree(d_val, s);
    pivot_free(&pi, s);
    multiline_free(&ml, s);
    planes_free(&At, s);
    planes_free(&Arow, s);
    planes_free(&Zt, s);
    planes_free(&Ct, s);
    planes_free(&Bt, s);
    planes_free(&Xp, s);
    planes_free(&Xq, s);
    planes_free(&RdT, s);
    planes_free(&XpdT, s);
    planes_free(&XT, s);
    planes_free(&Cp, s);
    planes_free(&Yb, s);
    planes_free(&Zr, s);
    planes_free(&CtL, s);
    compact_free(&SA, s);
    compact_free(&SB, s);
    dfree(Adiag, s);
    dfree(A16, s);
    dfree(B16, s);
    dfree(C16, s);
    dfree(D16, s);
    dfree(Bt16, s);
    dfree(Y16, s);
    dfree(R16, s);
    dfree(np_d.Rnp, s);
    dfree(np_d.npc, s);
    dfree(np_ocol, s);
    dfree(is_piv_row, s);
    dfree(prow, s);
    dfree(pcol, s);
    dfree(outflag, s);
    dfree(outpos, s);
    dfree(cnt, s);
    dfree(orp, s);
    dfree(ocol, s);
    dfree(oval, s);
    if (rc != GBLA_OK) {
        cudaStreamSynchronize(s);
        cudaGetLastError();
        gbla_free(out);
    }
#undef STEP
#undef CSTEP
    return rc;
}

__global__ void piv_row_out_kernel(int64_t n, const unsigned long long *__restrict__ best, int64_t *out) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) out[c] = best[c] == ~0ull ? -1 : (int64_t)(best[c] & 0xFFFFFFFFull);
}

}  // namespace gbla

// ==================================================================== ABI
using namespace gbla;

extern "C" {

int gbla_version(void) { return 100; }

int gbla_selftest_fail_alloc_after(int64_t n) {
    inject_alloc_fault();   // reads the environment switch once, before it is overridden
    g_alloc_count = 0;
    g_fault_at = n < 0 ? -1 : (long long)n;
    return GBLA_OK;
}

int gbla_device_bytes_in_use(int64_t *bytes) {
    if (!bytes) return GBLA_E_INVAL;
    *bytes = 0;
    GBLA_TRY(check_device());
    GBLA_CUDA_TRY(cudaDeviceSynchronize());
    int dev = 0;
    cudaMemPool_t pool;
    uint64_t used = 0;
    GBLA_CUDA_TRY(cudaGetDevice(&dev));
    GBLA_CUDA_TRY(cudaDeviceGetDefaultMemPool(&pool, dev));
    GBLA_CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
    *bytes = (int64_t)used;
    return GBLA_OK;
}

const char *gbla_strerror(int code) {
    switch (code) {
        case GBLA_OK: return "ok";
        case GBLA_E_INVAL: return "invalid argument or malformed matrix";
        case GBLA_E_NOMEM: return "out of memory";
        case GBLA_E_CUDA: return "CUDA error";
        case GBLA_E_TIMEOUT: return "a bounded device wait expired";
        case GBLA_E_INTERNAL: return "internal error";
        case GBLA_E_UNSUPPORTED: return "unsupported device or option";
        case GBLA_E_CANCELLED: return "request cancelled";
        default: return "unknown error";
    }
}

void gbla_free(gbla_csr_out *out) {
    if (!out) return;
    if (out->on_device) {
        if (out->row_ptr) cudaFree(out->row_ptr);
        if (out->col) cudaFree(out->col);
        if (out->val) cudaFree(out->val);
    } else {
        gbla::host_release(out->row_ptr);
        gbla::host_release(out->col);
        gbla::host_release(out->val);
    }
    memset(out, 0, sizeof(*out));
}

int gbla_reduce_ex(const gbla_csr_in *in, uint32_t p, const gbla_options *opt, void *stream, gbla_csr_out *out,
                   int64_t *rank, gbla_stats *stats) {
    if (!in || !out || !rank || p >= 65536u || !is_prime(p)) {
        if (out) memset(out, 0, sizeof(*out));
        return GBLA_E_INVAL;
    }
    memset(out, 0, sizeof(*out));
    if (stats) memset(stats, 0, sizeof(*stats));
    return reduce_impl(in, p, opt, (cudaStream_t)stream, out, rank, stats);
}

int gbla_reduce(const gbla_csr_in *in, uint32_t p, int want_reduced, gbla_csr_out *out, int64_t *rank) {
    gbla_options o;
    memset(&o, 0, sizeof(o));
    o.want_reduced = want_reduced;
    return gbla_reduce_ex(in, p, &o, nullptr, out, rank, nullptr);
}

int gbla_modmatmul(int64_t M, int64_t N, int64_t K, const uint16_t *A, int64_t lda, const uint16_t *B, int64_t ldb,
                   uint16_t *C, int64_t ldc, uint32_t p, int sign, int variant, void *stream) {
    if (M < 0 || N < 0 || K < 0 || p >= 65536u || !is_prime(p) || (sign != 1 && sign != -1)) return GBLA_E_INVAL;
    if (variant < 0 || variant > GBLA_GEMM_U8) return GBLA_E_INVAL;
    if (M == 0 || N == 0 || K == 0) return GBLA_OK;
    if (!A || !B || !C || lda < K || ldb < N || ldc < N) return GBLA_E_INVAL;
    GBLA_TRY(check_device());
    cudaStream_t s = (cudaStream_t)stream;
    const ModP mp = make_modp(p);
    Planes Ap{}, Bp{};
    uint32_t *err = nullptr;
    int rc = GBLA_OK;
    if ((rc = dalloc_t(&err, 4, s)) == GBLA_OK && (rc = planes_alloc(&Ap, M, K, 2, s)) == GBLA_OK &&
        (rc = planes_alloc(&Bp, N, K, 4, s)) == GBLA_OK) {
        cudaMemsetAsync(err, 0, 4, s);
        rc = to_planes(Ap, M, K, A, lda, 0, false, nullptr, nullptr, mp, s);
        if (rc == GBLA_OK) rc = to_planes(Bp, N, K, B, ldb, 0, true, nullptr, nullptr, mp, s);
        if (rc == GBLA_OK) rc = modgemm(Ap, 0, 0, Bp, 0, 0, C, ldc, M, N, K, sign, mp, variant, err, s, nullptr);
        if (cudaStreamSynchronize(s) != cudaSuccess) rc = GBLA_E_CUDA;
        uint32_t herr = 0;
        if (rc == GBLA_OK && readback(&herr, err, 4, s) == GBLA_OK) rc = map_dev_err(herr);
    }
    planes_free(&Ap, s);
    planes_free(&Bp, s);
    dfree(err, s);
    cudaStreamSynchronize(s);
    return rc;
}

int gbla_modmatmul32(int64_t M, int64_t N, int64_t K, const uint32_t *A, int64_t lda, const uint32_t *B,
                     int64_t ldb, uint32_t *C, int64_t ldc, uint32_t p, int sign, void *stream) {
    if (M < 0 || N < 0 || K < 0 || p < 3 || p >= (1u << 31) || !is_prime(p) || (sign != 1 && sign != -1))
        return GBLA_E_INVAL;
    if (M == 0 || N == 0 || K == 0) return GBLA_OK;
    if (!A || !B || !C || lda < K || ldb < N || ldc < N) return GBLA_E_INVAL;
    GBLA_TRY(check_device());
    return modmatmul32(M, N, K, A, lda, B, ldb, C, ldc, p, sign, (cudaStream_t)stream);
}

int gbla_pipe_peak(int variant, double *tops, void *stream) {
    if (!tops || (variant != GBLA_GEMM_FP64 && variant != GBLA_GEMM_U8)) return GBLA_E_INVAL;
    GBLA_TRY(check_device());
    return pipe_peak(variant, tops, (cudaStream_t)stream);
}

int gbla_spmm(int64_t M, int64_t N, int64_t K, const uint16_t *X, int64_t ldx, const gbla_csr_in *S_dev,
              const int32_t *x_lead, uint16_t *C, int64_t ldc, uint32_t p, int sign, void *stream) {
    if (M < 0 || N < 0 || K < 0 || !S_dev || p >= 65536u || !is_prime(p) || (sign != 1 && sign != -1))
        return GBLA_E_INVAL;
    if (S_dev->nrows != K || S_dev->ncols != N || S_dev->nnz < 0) return GBLA_E_INVAL;
    if (M == 0 || N == 0 || K == 0) return GBLA_OK;
    if (!X || !C || ldx < K || ldc < N || !S_dev->row_ptr || (S_dev->nnz > 0 && (!S_dev->col || !S_dev->val)))
        return GBLA_E_INVAL;
    GBLA_TRY(check_device());
    if (!tc_supported() || p < 8) return GBLA_E_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    const ModP mp = make_modp(p);
    DevCSR S;
    S.m = K;
    S.n = N;
    S.nnz = S_dev->nnz;
    S.row_ptr = S_dev->row_ptr;
    S.col = S_dev->col;
    S.val = S_dev->val;
    Compact SB;
    Planes XT{};
    uint32_t *err = nullptr;
    int rc = dalloc_t(&err, 4, s);
    if (rc == GBLA_OK && cudaMemsetAsync(err, 0, 4, s) != cudaSuccess) rc = GBLA_E_CUDA;
    if (rc == GBLA_OK) rc = compact_from_csr(S, &SB, mp, err, s);
    if (rc == GBLA_OK) rc = planes_alloc(&XT, K, M, 2, s);
    if (rc == GBLA_OK) rc = planes_zero(XT, s);
    if (rc == GBLA_OK) rc = to_planes(XT, K, M, X, ldx, 0, true, nullptr, nullptr, mp, s);
    if (rc == GBLA_OK) rc = modgemm_gather(SB, 0, XT, K, C, ldc, M, N, sign, x_lead, mp, err, s, nullptr);
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == GBLA_OK) rc = GBLA_E_CUDA;
    uint32_t herr = 0;
    if (rc == GBLA_OK && readback(&herr, err, 4, s) == GBLA_OK) rc = map_dev_err(herr);
    compact_free(&SB, s);
    planes_free(&XT, s);
    dfree(err, s);
    cudaStreamSynchronize(s);
    return rc;
}

int gbla_selftest_wait_timeout(void *stream) {
    GBLA_TRY(check_device());
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *err = nullptr;
    int rc = dalloc_t(&err, 4, s);
    if (rc == GBLA_OK && cudaMemsetAsync(err, 0, 4, s) != cudaSuccess) rc = GBLA_E_CUDA;
    if (rc == GBLA_OK) rc = modgemm_withheld_loads(err, s);
    uint32_t herr = 0;
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = GBLA_E_CUDA;
    if (rc == GBLA_OK && readback(&herr, err, 4, s) != GBLA_OK) rc = GBLA_E_CUDA;
    dfree(err, s);
    cudaStreamSynchronize(s);
    if (rc != GBLA_OK) return rc;
    return map_dev_err(herr);
}

int gbla_pivots(const gbla_csr_in *in_dev, uint32_t p, int64_t *piv_row_dev, int64_t *npiv, void *stream) {
    if (!in_dev || !piv_row_dev || !npiv || p >= 65536u || !is_prime(p)) return GBLA_E_INVAL;
    if (in_dev->nrows < 0 || in_dev->ncols < 0 || in_dev->nnz < 0) return GBLA_E_INVAL;
    GBLA_TRY(check_device());
    cudaStream_t s = (cudaStream_t)stream;
    const ModP mp = make_modp(p);
    DevCSR dc;
    dc.m = in_dev->nrows;
    dc.n = in_dev->ncols;
    dc.nnz = in_dev->nnz;
    dc.row_ptr = in_dev->row_ptr;
    dc.col = in_dev->col;
    dc.val = in_dev->val;
    PivotInfo pi;
    uint32_t *err = nullptr;
    int rc = dalloc_t(&err, 4, s);
    if (rc == GBLA_OK && cudaMemsetAsync(err, 0, 4, s) != cudaSuccess) rc = GBLA_E_CUDA;
    if (rc == GBLA_OK) rc = pivot_analysis(dc, mp, &pi, err, s);
    if (rc == GBLA_OK && dc.n > 0) {
        piv_row_out_kernel<<<(unsigned)((dc.n + 255) / 256), 256, 0, s>>>(dc.n, pi.best, piv_row_dev);
        if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
    }
    if (rc == GBLA_OK) *npiv = pi.npiv;
    pivot_free(&pi, s);
    dfree(err, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == GBLA_OK) rc = GBLA_E_CUDA;
    return rc;
}

int gbla_multiline(const gbla_csr_in *pairs_host, int64_t *ml_ptr, int32_t *ml_pos, uint16_t *ml_val, void *stream) {
    if (!pairs_host || !ml_ptr || pairs_host->nrows < 0 || pairs_host->nnz < 0) return GBLA_E_INVAL;
    GBLA_TRY(check_device());
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t m = pairs_host->nrows, nnz = pairs_host->nnz;
    const int64_t npairs = (m + 1) / 2;
    int64_t *rp = nullptr, *mp_ = nullptr;
    int32_t *col = nullptr, *pos = nullptr;
    uint16_t *val = nullptr, *mv = nullptr;
    int64_t total = 0;
    int rc = GBLA_OK;
    if ((rc = dalloc_t(&rp, (size_t)m + 1, s)) || (rc = dalloc_t(&col, (size_t)nnz + 1, s)) ||
        (rc = dalloc_t(&val, (size_t)nnz + 1, s)) || (rc = dalloc_t(&mp_, (size_t)npairs + 2, s)) ||
        (rc = dalloc_t(&pos, (size_t)nnz + 1, s)) || (rc = dalloc_t(&mv, (size_t)2 * nnz + 2, s))) {
    } else {
        cudaMemcpyAsync(rp, pairs_host->row_ptr, sizeof(int64_t) * (size_t)(m + 1), cudaMemcpyHostToDevice, s);
        if (nnz) {
            cudaMemcpyAsync(col, pairs_host->col, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(val, pairs_host->val, sizeof(uint16_t) * (size_t)nnz, cudaMemcpyHostToDevice, s);
        }
        rc = multiline_pairs(m, rp, col, val, mp_, pos, mv, &total, s);
        if (rc == GBLA_OK) {
            cudaMemcpyAsync(ml_ptr, mp_, sizeof(int64_t) * (size_t)(npairs + 1), cudaMemcpyDeviceToHost, s);
            if (total) {
                cudaMemcpyAsync(ml_pos, pos, sizeof(int32_t) * (size_t)total, cudaMemcpyDeviceToHost, s);
                cudaMemcpyAsync(ml_val, mv, sizeof(uint16_t) * (size_t)(2 * total), cudaMemcpyDeviceToHost, s);
            }
            if (cudaStreamSynchronize(s) != cudaSuccess) rc = GBLA_E_CUDA;
        }
    }
    dfree(rp, s);
    dfree(col, s);
    dfree(val, s);
    dfree(mp_, s);
    dfree(pos, s);
    dfree(mv, s);
    cudaStreamSynchronize(s);
    return rc;
}

}  // extern "C"
