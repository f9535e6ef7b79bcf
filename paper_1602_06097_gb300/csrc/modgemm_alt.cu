// modgemm_alt.cu -- the Schur update's alternative exact products on the
// legacy warp-level tensor-core instructions, and microbenchmarks of their
// pipes.
//
// Both compute C <- (C + sign * A * B^T) mod p (the Schur update
// D <- D - X*B of the new order, Sec. 4.3) from the same digit-plane operand
// sets as the tcgen05 product: an A set holds the balanced digits (hi, lo) of
// each residue, s = 256*hi + lo with |s| <= (p-1)/2.
//
// FP64 (DMMA, mma.sync m8n8k4 f64).  Each operand is the balanced residue s as
// a double.  |s_a * s_b| <= 32760^2 < 2^30, so any sum of at most 2^23 such
// products is an integer below 2^53 in magnitude and fp64 accumulation is
// exact in every order (delayed reduction: one reduction mod p per k-block of
// 2^23).
//
// U8 (IMMA, mma.sync m16n8k32 u8 x u8 -> s32).  Each operand is the
// unbalanced residue u in [0, p) split into its bytes u = 256*uh + ul, so
//     a*b = 65536*(ah*bh) + 256*(ah*bl + al*bh) + al*bl
// and three s32 accumulators (hh, mid, ll) hold the sums.  mid adds two
// products of at most 255^2 per k, so over a k-block of 2^14 it stays below
// 2 * 255^2 * 2^14 = 2,130,739,200 < 2^31: exact, never wrapping.
//
// Kernel shape (both): 64 x 64 output tiles, 4 warps of 32 x 32, K staged in
// 32-wide chunks through a double-buffered shared-memory tile; the next
// chunk's global loads are in flight while the current one is multiplied.
// At the end of each k-block the thread's accumulators are reduced mod p and
// added into C (its own elements only), then cleared.
#include <stdio.h>

#include <mutex>

#include "common.cuh"
#include "internal.cuh"

namespace gbla {
namespace alt {

constexpr int BM = 64, BN = 64, BK = 32, THREADS = 128;
constexpr int64_t F64_KBLOCK = (int64_t)1 << 23;   // 2^23 * 32760^2 < 2^53
constexpr int64_t U8_KBLOCK = (int64_t)1 << 14;    // 2 * 255^2 * 2^14 < 2^31
constexpr int F64_LD = BK + 4;                      // doubles per shared row (bank spread)
constexpr int U8_LD = 48;                           // bytes per shared row (bank spread)
constexpr int F64_SMEM = 2 * 2 * BM * F64_LD * 8;   // 2 buffers x (A, B) tiles

// Eight balanced residues of one operand row at chunk offset k8 (a multiple of
// 8): digits from planes 0 and 1, zero outside the logical K range.
__device__ __forceinline__ void load8(const Planes &P, int64_t row, bool row_ok, int64_t k_abs, int64_t k_rel,
                                      int64_t K, int (&s)[8]) {
#pragma unroll
    for (int e = 0; e < 8; ++e) s[e] = 0;
    if (!row_ok || k_rel >= K || k_abs >= P.kp || row >= P.rows) return;
    const uint4 h = *reinterpret_cast<const uint4 *>(P.at(0, row, k_abs));
    const uint4 l = *reinterpret_cast<const uint4 *>(P.at(1, row, k_abs));
    const uint32_t hw[4] = {h.x, h.y, h.z, h.w}, lw[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const uint32_t hb = (e & 1) ? (hw[e >> 1] & 0xFFFF0000u) : (hw[e >> 1] << 16);
        const uint32_t lb = (e & 1) ? (lw[e >> 1] & 0xFFFF0000u) : (lw[e >> 1] << 16);
        const int v = 256 * __float2int_rz(__uint_as_float(hb)) + __float2int_rz(__uint_as_float(lb));
        s[e] = (k_rel + e < K) ? v : 0;
    }
}

// C[row, col] <- (C + sign * v) mod p, v in [0, p); row through c_rows.
__device__ __forceinline__ void add_into_c(uint16_t *C, int64_t ldc, const int32_t *c_rows, int64_t m, int64_t n,
                                           int64_t M, int64_t N, uint32_t v, int sign, uint32_t p) {
    if (m >= M || n >= N) return;
    const int64_t r = c_rows ? (int64_t)c_rows[m] : m;
    if (r < 0) return;
    uint32_t cur = C[r * ldc + n];
    uint32_t o = sign > 0 ? cur + v : cur + (p - v);
    if (o >= p) o -= p;
    C[r * ldc + n] = (uint16_t)o;
}

// First K index (relative, a multiple of BK) a row tile must read: its first
// row's lead when leads ascend.
__device__ __forceinline__ int64_t tile_kstart(const int32_t *row_lead, int64_t m0, int64_t a_k0, int64_t K) {
    if (!row_lead) return 0;
    int64_t z = (int64_t)row_lead[m0] - a_k0;
    if (z < 0) z = 0;
    if (z > K) z = K;
    return z / BK * BK;
}

__device__ __forceinline__ void dmma(double &c0, double &c1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c0), "+d"(c1)
                 : "d"(a), "d"(b));
}

__device__ __forceinline__ void imma(int (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// ------------------------------------------------------------ FP64 (DMMA)
// Fragment layout of m8n8k4 (g = lane / 4, t = lane % 4): A element (g, t),
// B element (k = t, n = g), accumulator elements (g, 2t) and (g, 2t + 1).
__global__ void __launch_bounds__(THREADS) modgemm_f64_kernel(Planes A, int64_t a_row0, int64_t a_k0, Planes B,
                                                              int64_t b_row0, int64_t b_k0, uint16_t *C, int64_t ldc,
                                                              const int32_t *__restrict__ c_rows,
                                                              const int32_t *__restrict__ row_lead, int64_t M,
                                                              int64_t N, int64_t K, int sign, ModP mp)
{
    extern __shared__ __align__(16) double f64_smem[];
    double *As = f64_smem;                      // [2][BM][F64_LD]
    double *Bs = f64_smem + 2 * BM * F64_LD;    // [2][BN][F64_LD]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3, wm = warp >> 1, wn = warp & 1;
    const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
    const int64_t ks = tile_kstart(row_lead, m0, a_k0, K);

    double acc[4][4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

    auto drain = [&]() {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    long long v = __double2ll_rn(acc[i][j][e]) % (long long)mp.p;
                    if (v < 0) v += mp.p;
                    add_into_c(C, ldc, c_rows, m0 + wm * 32 + i * 8 + g, n0 + wn * 32 + j * 8 + 2 * t + e, M, N,
                               (uint32_t)v, sign, mp.p);
                    acc[i][j][e] = 0.0;
                }
    };

    int ra[2][8], rb[2][8];
    auto fetch = [&](int64_t kk) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int it = tid + h * THREADS, row = it >> 2, k8 = (it & 3) * 8;
            load8(A, a_row0 + m0 + row, m0 + row < M, a_k0 + kk + k8, kk + k8, K, ra[h]);
            load8(B, b_row0 + n0 + row, n0 + row < N, b_k0 + kk + k8, kk + k8, K, rb[h]);
        }
    };
    auto stash = [&](int buf) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int it = tid + h * THREADS, row = it >> 2, k8 = (it & 3) * 8;
            double *a = As + (size_t)(buf * BM + row) * F64_LD + k8;
            double *b = Bs + (size_t)(buf * BN + row) * F64_LD + k8;
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
                *reinterpret_cast<double2 *>(a + e) = make_double2((double)ra[h][e], (double)ra[h][e + 1]);
                *reinterpret_cast<double2 *>(b + e) = make_double2((double)rb[h][e], (double)rb[h][e + 1]);
            }
        }
    };

    if (ks < K) fetch(ks);
    int buf = 0, steps = 0;   // K steps since the last drain
    for (int64_t kk = ks; kk < K; kk += BK) {
        stash(buf);
        __syncthreads();
        if (kk + BK < K) fetch(kk + BK);
        const double *a_s = As + (size_t)(buf * BM + wm * 32 + g) * F64_LD + t;
        const double *b_s = Bs + (size_t)(buf * BN + wn * 32 + g) * F64_LD + t;
#pragma unroll
        for (int k4 = 0; k4 < BK; k4 += 4) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = a_s[i * 8 * F64_LD + k4];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = b_s[j * 8 * F64_LD + k4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) dmma(acc[i][j][0], acc[i][j][1], a[i], b[j]);
        }
        if (++steps == F64_KBLOCK / BK && kk + BK < K) {
            drain();
            steps = 0;
        }
        buf ^= 1;
    }
    drain();
}

// ------------------------------------------------------------ U8 (IMMA)
// Fragment layout of m16n8k32 with 8-bit operands (g = lane / 4, t = lane % 4):
// A registers 0..3 hold rows g, g+8, g, g+8 at columns 4t..4t+3 (registers 0,
// 1) and 16+4t.. (registers 2, 3), the lower column in the lower byte; B
// registers 0, 1 hold column g at rows 4t..4t+3 and 16+4t..; accumulator
// registers 0..3 hold (g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1).
struct U8Smem {
    uint8_t ah[2][BM * U8_LD], al[2][BM * U8_LD], bh[2][BN * U8_LD], bl[2][BN * U8_LD];
};

__device__ __forceinline__ uint32_t lds32(const uint8_t *p) { return *reinterpret_cast<const uint32_t *>(p); }

__global__ void __launch_bounds__(THREADS) modgemm_u8_kernel(Planes A, int64_t a_row0, int64_t a_k0, Planes B,
                                                             int64_t b_row0, int64_t b_k0, uint16_t *C, int64_t ldc,
                                                             const int32_t *__restrict__ c_rows,
                                                             const int32_t *__restrict__ row_lead, int64_t M,
                                                             int64_t N, int64_t K, int sign, ModP mp)
{
    __shared__ __align__(16) U8Smem sm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3, wm = warp >> 1, wn = warp & 1;
    const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
    const int64_t ks = tile_kstart(row_lead, m0, a_k0, K);
    const int P = (int)mp.p;

    int hh[2][4][4], mid[2][4][4], ll[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) hh[i][j][e] = mid[i][j][e] = ll[i][j][e] = 0;

    auto drain = [&]() {
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const uint64_t v = ((uint64_t)(uint32_t)hh[i][j][e] << 16) +
                                       ((uint64_t)(uint32_t)mid[i][j][e] << 8) + (uint64_t)(uint32_t)ll[i][j][e];
                    add_into_c(C, ldc, c_rows, m0 + wm * 32 + i * 16 + g + (e >> 1) * 8,
                               n0 + wn * 32 + j * 8 + 2 * t + (e & 1), M, N, mod64(v, mp), sign, mp.p);
                    hh[i][j][e] = mid[i][j][e] = ll[i][j][e] = 0;
                }
    };

    int ra[2][8], rb[2][8];
    auto fetch = [&](int64_t kk) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int it = tid + h * THREADS, row = it >> 2, k8 = (it & 3) * 8;
            load8(A, a_row0 + m0 + row, m0 + row < M, a_k0 + kk + k8, kk + k8, K, ra[h]);
            load8(B, b_row0 + n0 + row, n0 + row < N, b_k0 + kk + k8, kk + k8, K, rb[h]);
        }
    };
    // bytes of the unbalanced residues, 8 per row segment
    auto split_store = [&](const int (&s)[8], uint8_t *hi, uint8_t *lo) {
        uint32_t h[2] = {0, 0}, l[2] = {0, 0};
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const uint32_t u = (uint32_t)(s[e] < 0 ? s[e] + P : s[e]);
            h[e >> 2] |= (u >> 8) << (8 * (e & 3));
            l[e >> 2] |= (u & 0xFFu) << (8 * (e & 3));
        }
        *reinterpret_cast<uint2 *>(hi) = make_uint2(h[0], h[1]);
        *reinterpret_cast<uint2 *>(lo) = make_uint2(l[0], l[1]);
    };
    auto stash = [&](int buf) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int it = tid + h * THREADS, row = it >> 2, k8 = (it & 3) * 8;
            split_store(ra[h], &sm.ah[buf][row * U8_LD + k8], &sm.al[buf][row * U8_LD + k8]);
            split_store(rb[h], &sm.bh[buf][row * U8_LD + k8], &sm.bl[buf][row * U8_LD + k8]);
        }
    };

    if (ks < K) fetch(ks);
    int buf = 0, steps = 0;   // K steps since the last drain
    for (int64_t kk = ks; kk < K; kk += BK) {
        stash(buf);
        __syncthreads();
        if (kk + BK < K) fetch(kk + BK);
        uint32_t fah[2][4], fal[2][4], fbh[4][2], fbl[4][2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int r = (wm * 32 + i * 16 + g) * U8_LD + 4 * t;
            const int r8 = r + 8 * U8_LD;
            fah[i][0] = lds32(&sm.ah[buf][r]);      fah[i][1] = lds32(&sm.ah[buf][r8]);
            fah[i][2] = lds32(&sm.ah[buf][r + 16]); fah[i][3] = lds32(&sm.ah[buf][r8 + 16]);
            fal[i][0] = lds32(&sm.al[buf][r]);      fal[i][1] = lds32(&sm.al[buf][r8]);
            fal[i][2] = lds32(&sm.al[buf][r + 16]); fal[i][3] = lds32(&sm.al[buf][r8 + 16]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = (wn * 32 + j * 8 + g) * U8_LD + 4 * t;
            fbh[j][0] = lds32(&sm.bh[buf][c]); fbh[j][1] = lds32(&sm.bh[buf][c + 16]);
            fbl[j][0] = lds32(&sm.bl[buf][c]); fbl[j][1] = lds32(&sm.bl[buf][c + 16]);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                imma(hh[i][j], fah[i], fbh[j]);
                imma(mid[i][j], fah[i], fbl[j]);
                imma(mid[i][j], fal[i], fbh[j]);
                imma(ll[i][j], fal[i], fbl[j]);
            }
        if (++steps == U8_KBLOCK / BK && kk + BK < K) {
            drain();
            steps = 0;
        }
        buf ^= 1;
    }
    drain();
}

// ------------------------------------------------ pipe microbenchmarks
// Eight independent accumulator chains per warp, operands in registers: the
// issue rate of the instruction alone.  The sums are stored so that nothing
// is dead.
constexpr int PEAK_CHAINS = 8;

__global__ void __launch_bounds__(256) pipe_f64_kernel(int iters, double *out) {
    double c[PEAK_CHAINS][2];
#pragma unroll
    for (int u = 0; u < PEAK_CHAINS; ++u) c[u][0] = c[u][1] = 0.0;
    const double a = 1.0 + threadIdx.x * 0x1p-20, b = 1.0 - blockIdx.x * 0x1p-24;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int u = 0; u < PEAK_CHAINS; ++u) dmma(c[u][0], c[u][1], a, b);
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < PEAK_CHAINS; ++u) s += c[u][0] + c[u][1];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) pipe_u8_kernel(int iters, double *out) {
    int c[PEAK_CHAINS][4];
#pragma unroll
    for (int u = 0; u < PEAK_CHAINS; ++u) c[u][0] = c[u][1] = c[u][2] = c[u][3] = 0;
    const uint32_t a[4] = {threadIdx.x & 3u, 1u, 2u, 3u}, b[2] = {blockIdx.x & 1u, 1u};
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int u = 0; u < PEAK_CHAINS; ++u) imma(c[u], a, b);
    long long s = 0;
#pragma unroll
    for (int u = 0; u < PEAK_CHAINS; ++u) s += (long long)c[u][0] + c[u][1] + c[u][2] + c[u][3];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = (double)s;
}

}  // namespace alt

int modgemm_alt(const Planes &A, int64_t a_row0, int64_t a_k0, const Planes &B, int64_t b_row0, int64_t b_k0,
                uint16_t *C, int64_t ldc, int64_t M, int64_t N, int64_t K, int sign, const ModP &mp, int variant,
                cudaStream_t s, const int32_t *c_rows, const int32_t *row_lead)
{
    if (M <= 0 || N <= 0 || K <= 0) return GBLA_OK;
    if (A.nplanes < 2 || B.nplanes < 2) return GBLA_E_INTERNAL;
    if ((a_k0 % alt::BK) || (b_k0 % alt::BK)) return GBLA_E_INTERNAL;
    if ((M + alt::BM - 1) / alt::BM > 65535) return GBLA_E_INVAL;
    const dim3 grid((unsigned)((N + alt::BN - 1) / alt::BN), (unsigned)((M + alt::BM - 1) / alt::BM));
    if (variant == GBLA_GEMM_FP64) {
        static const cudaError_t attr = cudaFuncSetAttribute(
            alt::modgemm_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, alt::F64_SMEM);
        GBLA_CUDA_TRY(attr);
        alt::modgemm_f64_kernel<<<grid, alt::THREADS, alt::F64_SMEM, s>>>(A, a_row0, a_k0, B, b_row0, b_k0, C, ldc,
                                                                         c_rows, row_lead, M, N, K, sign, mp);
    } else if (variant == GBLA_GEMM_U8) {
        alt::modgemm_u8_kernel<<<grid, alt::THREADS, 0, s>>>(A, a_row0, a_k0, B, b_row0, b_k0, C, ldc, c_rows,
                                                            row_lead, M, N, K, sign, mp);
    } else {
        return GBLA_E_INVAL;
    }
    GBLA_CUDA_TRY(launch_check());
    return GBLA_OK;
}

int pipe_peak(int variant, double *tops, cudaStream_t s) {
    if (!tops || (variant != GBLA_GEMM_FP64 && variant != GBLA_GEMM_U8)) return GBLA_E_INVAL;
    const int blocks = device_sm_count() * 4, threads = 256;
    // ops of one instruction: 2 * M * N * K
    const double per_mma = variant == GBLA_GEMM_FP64 ? 2.0 * 8 * 8 * 4 : 2.0 * 16 * 8 * 32;
    double *out = nullptr;
    GBLA_TRY(dalloc_t(&out, (size_t)blocks * threads, s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = GBLA_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = GBLA_E_CUDA;
    int iters = 64, timed_iters = 0;
    float ms = 0.f;
    // one warm-up launch, then grow the loop until a launch lasts >= 20 ms
    for (int round = 0; rc == GBLA_OK && round < 16; ++round) {
        timed_iters = iters;
        cudaEventRecord(e0, s);
        if (variant == GBLA_GEMM_FP64)
            alt::pipe_f64_kernel<<<blocks, threads, 0, s>>>(iters, out);
        else
            alt::pipe_u8_kernel<<<blocks, threads, 0, s>>>(iters, out);
        if (launch_check() != cudaSuccess) { rc = GBLA_E_CUDA; break; }
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = GBLA_E_CUDA;
            break;
        }
        if (round > 0 && ms >= 20.f) break;
        if (iters >= (1 << 22)) break;
        const double grow = ms > 0.5f ? 25.0 / ms : 16.0;
        iters = (int)(iters * (grow < 2.0 ? 2.0 : (grow > 64.0 ? 64.0 : grow)));
        if (iters > (1 << 22)) iters = 1 << 22;
    }
    if (rc == GBLA_OK)
        *tops = (double)blocks * (threads / 32) * (double)timed_iters * alt::PEAK_CHAINS * per_mma / (ms * 1e-3) / 1e12;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dfree(out, s);
    cudaStreamSynchronize(s);
    return rc;
}

}  // namespace gbla
