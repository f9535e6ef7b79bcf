// sge.cu -- structured Gaussian elimination of the Schur complement D' with
// sparse pivot rows: the parallel SGE of the paper (Alg. 3 and its parallel
// form, Sec. 5.1) as a persistent GPU kernel, an alternative forward pass of
// the echelon step for a D' that stays sparse.
//
// Every warp takes the next row of D' (a global counter) and works on it in
// place (rows of D16 only ever receive row operations, so the row space never
// changes):
//   1. find the row's leading column c (a ballot over 32 columns at a time);
//   2. if c has no pivot yet, claim it (atomic compare-and-swap on
//      pivot_of_col[c]), normalise the row to a leading 1, copy its nonzeros
//      into the sparse pivot pool and publish the pivot; the row is done;
//   3. if c is being claimed by another warp, wait for its pivot (bounded);
//   4. else subtract row[c] times the pivot row (its sparse entries, one per
//      lane) and go on from column c + 1.
// A zero row is done.  The claimed columns play the role of the paper's
// shared pivot list; a row waiting on a column being claimed is its waiting
// list; rows are fetched in index order.
//
// The result is an echelon form: every pivot row is normalised and zero left
// of its lead, the pivot rows span the rows of D'.  Which row becomes the pivot
// of a column depends on timing, but the reduced echelon form computed from it
// afterwards does not.  If the pivot pool fills up, the pass stops between row
// operations and the caller continues with the dense panel method on the
// partly reduced rows.  Every wait is bounded (about a second of clock64); on
// expiry the kernel records DEV_ERR_TIMEOUT and returns.
#include <algorithm>

#include "common.cuh"
#include "internal.cuh"
#include "solve.cuh"

namespace gbla {
namespace {

constexpr int SGE_WARPS = 4;
constexpr int32_t COL_FREE = -1, COL_CLAIMING = -2, COL_FAILED = -3;
constexpr long long SGE_WAIT_CYCLES = 2000000000ll;   // ~1 s at 2 GHz

struct SgeState {
    int32_t *pivot_of_col;   // [n]: COL_FREE, COL_CLAIMING, COL_FAILED or a pivot index
    int64_t *piv_row;        // [m]: D row of pivot k
    int64_t *piv_off;        // [m]: its first entry in the pool
    int32_t *piv_len;        // [m]: its entries
    int32_t *pool_col;       // [cap]
    uint16_t *pool_val;      // [cap]
    int64_t cap;
    unsigned long long *counters;   // [0] next row, [1] pivots, [2] pool entries used, [3] overflow
};

__device__ __forceinline__ int32_t ld_volatile(const int32_t *p) { return *(const volatile int32_t *)p; }

__global__ void __launch_bounds__(32 * SGE_WARPS) sge_kernel(uint16_t *D, int64_t ldd, int64_t m, int64_t n,
                                                            SgeState st, ModP mp, uint32_t *err)
{
    const int lane = threadIdx.x & 31;
    const uint32_t P = mp.p;
    for (;;) {
        unsigned long long r_ = 0;
        if (lane == 0) r_ = atomicAdd(&st.counters[0], 1ull);
        const int64_t r = (int64_t)__shfl_sync(0xffffffffu, r_, 0);
        if (r >= m) return;
        if (*(volatile unsigned long long *)&st.counters[3] || *(volatile uint32_t *)err) return;
        uint16_t *row = D + r * ldd;
        int64_t pos = 0;
        for (;;) {
            // 1. leading column at or after pos
            int64_t lead = n;
            for (int64_t c0 = pos; c0 < n; c0 += 32) {
                const int64_t c = c0 + lane;
                const uint32_t b = __ballot_sync(0xffffffffu, c < n && row[c] != 0);
                if (b) {
                    lead = c0 + __ffs(b) - 1;
                    break;
                }
            }
            if (lead >= n) break;   // zero row
            // 2./3. the column's pivot: claim it, wait for it, or use it
            int32_t k = 0;
            if (lane == 0) {
                k = ld_volatile(&st.pivot_of_col[lead]);
                if (k == COL_FREE) {
                    const int32_t old = atomicCAS(&st.pivot_of_col[lead], COL_FREE, COL_CLAIMING);
                    k = old == COL_FREE ? -100 : old;
                }
                if (k == COL_CLAIMING) {
                    const long long t0 = clock64();
                    do {
                        __nanosleep(64);
                        k = ld_volatile(&st.pivot_of_col[lead]);
                    } while (k == COL_CLAIMING && clock64() - t0 < SGE_WAIT_CYCLES);
                    if (k == COL_CLAIMING) {
                        dev_fail(err, DEV_ERR_TIMEOUT);
                        k = COL_FAILED;
                    }
                }
            }
            k = __shfl_sync(0xffffffffu, k, 0);
            if (k == COL_FAILED) return;
            if (k == -100) {
                // normalise to a leading 1, count the entries, copy them to the pool
                const uint32_t inv = invmod(row[lead], mp);
                int64_t cnt = 0;
                for (int64_t c0 = lead; c0 < n; c0 += 32) {
                    const int64_t c = c0 + lane;
                    uint32_t v = c < n ? row[c] : 0u;
                    if (v) {
                        v = mulmod(v, inv, mp);
                        row[c] = (uint16_t)v;
                    }
                    cnt += __popc(__ballot_sync(0xffffffffu, v != 0));
                }
                unsigned long long off_ = 0;
                if (lane == 0) off_ = atomicAdd(&st.counters[2], (unsigned long long)cnt);
                const int64_t off = (int64_t)__shfl_sync(0xffffffffu, off_, 0);
                if (off + cnt > st.cap) {
                    if (lane == 0) {
                        atomicExch((unsigned long long *)&st.counters[3], 1ull);
                        atomicExch(&st.pivot_of_col[lead], COL_FAILED);
                    }
                    return;
                }
                int64_t at = off;
                for (int64_t c0 = lead; c0 < n; c0 += 32) {
                    const int64_t c = c0 + lane;
                    const uint32_t v = c < n ? row[c] : 0u;
                    const uint32_t b = __ballot_sync(0xffffffffu, v != 0);
                    if (v) {
                        const int64_t idx = at + __popc(b & ((1u << lane) - 1u));
                        st.pool_col[idx] = (int32_t)c;
                        st.pool_val[idx] = (uint16_t)v;
                    }
                    at += __popc(b);
                }
                __syncwarp();
                if (lane == 0) {
                    const int32_t kk = (int32_t)atomicAdd(&st.counters[1], 1ull);
                    st.piv_row[kk] = r;
                    st.piv_off[kk] = off;
                    st.piv_len[kk] = (int32_t)cnt;
                    __threadfence();
                    atomicExch(&st.pivot_of_col[lead], kk);
                }
                break;   // the row is a pivot
            }
            // 4. row -= row[lead] * pivot k (the pivot's entry at lead is 1)
            __threadfence();
            const uint32_t f = row[lead];
            const int64_t poff = __ldcg(&st.piv_off[k]);
            const int32_t plen = __ldcg(&st.piv_len[k]);
            const uint32_t nf = P - f;
            for (int32_t e = lane; e < plen; e += 32) {
                const int32_t c = __ldcg(&st.pool_col[poff + e]);
                const uint32_t v = __ldcg(&st.pool_val[poff + e]);
                uint32_t x = row[c] + mulmod(nf, v, mp);
                if (x >= P) x -= P;
                row[c] = (uint16_t)x;
            }
            __syncwarp();
            pos = lead + 1;
        }
    }
}

// nonzeros of every stride-th row of D
__global__ void sge_count_kernel(const uint16_t *__restrict__ D, int64_t ldd, int64_t m, int64_t n, int64_t stride,
                                 unsigned long long *nnz)
{
    unsigned long long c = 0;
    for (int64_t r = (int64_t)blockIdx.x * stride; r < m; r += (int64_t)gridDim.x * stride)
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) c += D[r * ldd + j] != 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(nnz, c);
}

__global__ void sge_flags_kernel(const int32_t *__restrict__ pivot_of_col, int64_t n, int64_t *flag)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) flag[c] = pivot_of_col[c] >= 0 ? 1 : 0;
}

// pivots in ascending column order: pcol[i], prow[i] (the D row it lives in)
__global__ void sge_collect_kernel(const int32_t *__restrict__ pivot_of_col, const int64_t *__restrict__ pos,
                                   const int64_t *__restrict__ piv_row, int64_t n, int32_t *prow, int32_t *pcol)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int32_t k = pivot_of_col[c];
    if (k < 0) return;
    pcol[pos[c]] = (int32_t)c;
    prow[pos[c]] = (int32_t)piv_row[k];
}

}  // namespace

int dprime_density(const EchelonD &E, double *density)
{
    *density = 0.0;
    const int64_t m = E.m, n = E.n;
    cudaStream_t s = E.s;
    if (m <= 0 || n <= 0) return GBLA_OK;
    DevTemp<unsigned long long> nnz_dev(s);
    GBLA_TRY(nnz_dev.alloc(1));
    GBLA_CUDA_TRY(cudaMemsetAsync(nnz_dev, 0, sizeof(unsigned long long), s));
    // a sample of at most 4,096 evenly spaced rows
    const int64_t stride = m > 4096 ? m / 4096 : 1;
    const int64_t rows = (m + stride - 1) / stride;
    sge_count_kernel<<<device_sm_count() * 8, 256, 0, s>>>(E.D16, E.ldd, m, n, stride, nnz_dev);
    GBLA_CUDA_TRY(launch_check());
    unsigned long long nnz = 0;
    GBLA_TRY(readback(&nnz, nnz_dev, sizeof(nnz), s));
    *density = (double)nnz / ((double)rows * (double)n);
    return GBLA_OK;
}

int sge_forward(const EchelonD &E, double density, int64_t *rank, bool *overflow)
{
    *rank = 0;
    *overflow = false;
    const int64_t m = E.m, n = E.n;
    cudaStream_t s = E.s;
    if (m <= 0 || n <= 0) return GBLA_OK;
    DevTemp<unsigned long long> counters(s);
    DevTemp<int32_t> pivot_of_col(s), piv_len(s), pool_col(s);
    DevTemp<int64_t> piv_row(s), piv_off(s), flag(s);
    DevTemp<uint16_t> pool_val(s);
    // pool for the pivot rows: room for four times the nonzeros of D' (fill-in)
    // plus a band, never more than the dense block
    const double nnz = density * (double)m * (double)n;
    const int64_t cap = std::min<int64_t>(m * n, (int64_t)(4.0 * nnz) + 64 * n + 1024);
    GBLA_TRY(counters.alloc(4));
    GBLA_TRY(pivot_of_col.alloc((size_t)n));
    GBLA_TRY(piv_row.alloc((size_t)m));
    GBLA_TRY(piv_off.alloc((size_t)m));
    GBLA_TRY(piv_len.alloc((size_t)m));
    GBLA_TRY(pool_col.alloc((size_t)cap));
    GBLA_TRY(pool_val.alloc((size_t)cap));
    GBLA_CUDA_TRY(cudaMemsetAsync(counters, 0, 4 * sizeof(unsigned long long), s));
    GBLA_CUDA_TRY(cudaMemsetAsync(pivot_of_col, 0xFF, sizeof(int32_t) * (size_t)n, s));   // COL_FREE
    SgeState st{pivot_of_col, piv_row, piv_off, piv_len, pool_col, pool_val, cap, counters};
    const int grid = device_sm_count() * 8;
    sge_kernel<<<grid, 32 * SGE_WARPS, 0, s>>>(E.D16, E.ldd, m, n, st, *E.mp, E.err);
    GBLA_CUDA_TRY(launch_check());
    unsigned long long cnt[4] = {0, 0, 0, 0};
    GBLA_TRY(readback(cnt, counters, sizeof(cnt), s));
    uint32_t herr = 0;
    GBLA_TRY(readback(&herr, E.err, sizeof(herr), s));
    if (herr) return map_dev_err(herr);
    if (cnt[3]) {
        *overflow = true;
        return GBLA_OK;
    }
    GBLA_TRY(flag.alloc((size_t)n + 1));
    sge_flags_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pivot_of_col, n, flag);
    GBLA_CUDA_TRY(launch_check());
    GBLA_TRY(scan_i64(flag, flag, n, nullptr, s));
    sge_collect_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pivot_of_col, flag, piv_row, n, E.prow, E.pcol);
    GBLA_CUDA_TRY(launch_check());
    *rank = (int64_t)cnt[1];
    return GBLA_OK;
}

}  // namespace gbla
