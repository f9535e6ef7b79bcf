// noalloc.cu -- pivot analysis that allocates no memory.
//
// Some callers must not allocate device memory during a call: an
// application that reserves all device memory up front for its own pool
// (so a cudaMalloc inside the library would fail or push it over budget),
// or a latency-sensitive loop where an allocation may synchronise the
// device and stall its other streams.  gbla_pivots_noalloc gives them the
// pivot choice of gbla_pivots without any allocation: its only scratch is
// the file-scope device array below, which every GPU that loads this
// library holds until the process exits.
//
// The array is shared by all calls and keeps the previous call's contents;
// each call clears the part it uses before using it.  Two calls that
// overlap on the GPU (different streams, or different host threads) use the
// same array and race; callers must serialise them.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <mutex>

#include "common.cuh"

namespace gbla {

// Largest number of columns the no-allocation entry point accepts.
constexpr int64_t NOALLOC_MAX_COLS = int64_t(1) << 20;

// Scratch: the best (weight << 32 | row) key per column, then two counters
// (number of pivots, error bits).  8 MiB + 256 bytes.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[NOALLOC_MAX_COLS + 32];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
unsigned long long *g_scratch_ptr[MAX_DEVICES] = {};
CUcontext g_scratch_ctx[MAX_DEVICES] = {};
PFN_cuCtxGetCurrent_v4000 g_ctx_current = nullptr;
std::once_flag g_ctx_once;

// Device address of the scratch array on the current device, looked up at
// set-up: once per device and context (host code cannot use the symbol itself
// as a device address).  A context that was destroyed and recreated on the
// device (cudaDeviceReset) reloads the library's module, which may place the
// array elsewhere, so the address is looked up again for the new context.
int scratch_for_current_device(unsigned long long **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return GBLA_E_CUDA;
    std::call_once(g_ctx_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(fn);
    });
    // make the device's primary context current (cudaSetDevice initialises
    // it; nothing is allocated)
    if (cudaSetDevice(dev) != cudaSuccess) {
        cudaGetLastError();
        return GBLA_E_CUDA;
    }
    CUcontext ctx = nullptr;
    if (!g_ctx_current || g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx) return GBLA_E_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev] || g_scratch_ctx[dev] != ctx) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return GBLA_E_CUDA;
        }
        g_scratch_ptr[dev] = static_cast<unsigned long long *>(ptr);
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_ptr[dev];
    return GBLA_OK;
}

// GBLA_OK on a compute capability 10.3 device (the only target of this
// build), without touching any memory pool.
int device_is_sm103() {
    int dev = 0, major = 0, minor = 0, n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        return GBLA_E_UNSUPPORTED;
    }
    if (cudaGetDevice(&dev) != cudaSuccess) return GBLA_E_CUDA;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    return (major == 10 && minor == 3) ? GBLA_OK : GBLA_E_UNSUPPORTED;
}

__global__ void noalloc_clear_kernel(unsigned long long *scratch, int64_t n) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        scratch[c] = ~0ull;
    if (blockIdx.x == 0 && threadIdx.x < 2) scratch[NOALLOC_MAX_COLS + threadIdx.x] = 0;
}

// One warp per row: validate the row and offer it as pivot candidate of its
// leading column (fewest nonzeros wins, then the smaller row index).
__global__ void noalloc_scan_rows_kernel(int64_t m, int64_t n, int64_t nnz, const int64_t *__restrict__ row_ptr,
                                         const int32_t *__restrict__ col, const uint16_t *__restrict__ val,
                                         uint32_t p, unsigned long long *scratch) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= m) return;
    const int64_t b = row_ptr[r], e = row_ptr[r + 1];
    bool bad = (b < 0) || (e < b) || (e > nnz) || (r == 0 && b != 0) || (r == m - 1 && e != nnz);
    if (!bad) {
        for (int64_t i = b + lane; i < e; i += 32) {
            const int32_t c = col[i];
            const uint32_t v = val[i];
            if (c < 0 || c >= n || v == 0 || v >= p) bad = true;
            if (i > b && col[i - 1] >= c) bad = true;
        }
    }
    if (__any_sync(0xFFFFFFFFu, bad)) {
        if (lane == 0) atomicOr(&scratch[NOALLOC_MAX_COLS + 1], 1ull);
        return;
    }
    if (lane == 0 && e > b)
        atomicMin(&scratch[col[b]], ((unsigned long long)(e - b) << 32) | (unsigned long long)r);
}

// piv_row is written only if every row was valid (the error word is still
// zero once the scan kernel has finished), so on GBLA_E_INVAL the caller's
// array is left as it was.
__global__ void noalloc_finish_kernel(int64_t n, unsigned long long *scratch, int64_t *piv_row) {
    if (*(volatile unsigned long long *)&scratch[NOALLOC_MAX_COLS + 1] != 0ull) return;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = scratch[c];
        piv_row[c] = (k == ~0ull) ? -1 : (int64_t)(k & 0xFFFFFFFFull);
        if (k != ~0ull) atomicAdd(&scratch[NOALLOC_MAX_COLS], 1ull);
    }
}

bool prime16(uint32_t p) {
    if (p < 2 || p >= 65536u) return false;
    for (uint32_t d = 2; d * d <= p; ++d)
        if (p % d == 0) return false;
    return true;
}

}  // namespace
}  // namespace gbla

extern "C" int gbla_pivots_noalloc(const gbla_csr_in *in_dev, uint32_t p, int64_t *piv_row_dev, int64_t *npiv,
                                   void *stream) {
    using namespace gbla;
    if (!in_dev || !piv_row_dev || !npiv || !prime16(p)) return GBLA_E_INVAL;
    const int64_t m = in_dev->nrows, n = in_dev->ncols, nnz = in_dev->nnz;
    if (m < 0 || n < 0 || nnz < 0 || m >= (int64_t(1) << 31)) return GBLA_E_INVAL;
    if (n > NOALLOC_MAX_COLS) return GBLA_E_INVAL;   // beyond the fixed scratch size
    if ((m > 0 && !in_dev->row_ptr) || (nnz > 0 && (!in_dev->col || !in_dev->val))) return GBLA_E_INVAL;
    GBLA_TRY(device_is_sm103());
    unsigned long long *scratch = nullptr;
    GBLA_TRY(scratch_for_current_device(&scratch));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const unsigned grid_n = (unsigned)((n + 255) / 256 < 1024 ? ((n + 255) / 256 > 0 ? (n + 255) / 256 : 1) : 1024);
    noalloc_clear_kernel<<<grid_n, 256, 0, s>>>(scratch, n);
    GBLA_CUDA_TRY(cudaGetLastError());
    if (m > 0) {
        noalloc_scan_rows_kernel<<<(unsigned)((m * 32 + 255) / 256), 256, 0, s>>>(m, n, nnz, in_dev->row_ptr,
                                                                                 in_dev->col, in_dev->val, p, scratch);
        GBLA_CUDA_TRY(cudaGetLastError());
    }
    noalloc_finish_kernel<<<grid_n, 256, 0, s>>>(n, scratch, piv_row_dev);
    GBLA_CUDA_TRY(cudaGetLastError());
    unsigned long long counters[2] = {0, 0};
    GBLA_CUDA_TRY(cudaMemcpyAsync(counters, scratch + NOALLOC_MAX_COLS, sizeof(counters), cudaMemcpyDeviceToHost, s));
    GBLA_CUDA_TRY(cudaStreamSynchronize(s));
    if (counters[1]) return GBLA_E_INVAL;
    *npiv = (int64_t)counters[0];
    return GBLA_OK;
}
