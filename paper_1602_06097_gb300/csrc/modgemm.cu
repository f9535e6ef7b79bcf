// modgemm.cu -- exact modular matrix product C <- (C + sign * A * B) mod p.
//
// This is the dense Schur update of the FL reduction, D <- D - C*A^-1*B
// (GBLA paper Sec. 4.1 steps 2-3; Sec. 4.3 step 4 of the new order), and the
// block updates of the triangular solves and of the echelonisation of D.
//
// Tensor-core path (sm_103a).  Residues are written in balanced form and
// split into two 8-bit digits that are exact in bf16 (common.cuh).  With
// b' = 256*b mod p,
//     a*b = (256*ah + al)*b == ah*b' + al*b
//         == 256*(ah*b'h + al*bh) + (ah*b'l + al*bl)      (mod p),
// so two fp32 accumulators P = sum(ah*b'h + al*bh) and Q = sum(ah*b'l + al*bl)
// suffice.  Every digit product is at most 2^14 in magnitude and each k adds
// two of them, so over a k-block of 512 every partial sum stays below 2^24 and
// fp32 accumulation is exact whatever the order of additions.  After each
// k-block the accumulators are drained from TMEM, converted to integers and
// reduced mod p (integer arithmetic apart from one fp32 quotient estimate) into
// a running residue kept in registers.  The kernel is a persistent,
// warp-specialised tcgen05 pipeline: one thread issues TMA loads into a
// 4-stage shared-memory ring, one thread issues tcgen05.mma into a
// double-buffered TMEM accumulator pair, eight warps drain TMEM.
//
// SIMT path: exact int64 dot products on CUDA cores, used as the reference
// variant in tests and for p < 8.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdio.h>
#include <stdlib.h>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace gbla {

// ===================================================================
// u16 matrix -> digit planes
// ===================================================================
// dst(r, k) for r < round_up(R, 128), k < round_up(Kc, 128) (within the buffer):
//   transposed == false : src[g(r) * lds + col_off + h(k)]
//   transposed == true  : src[g(k) * lds + col_off + r]
// with g = row gather (or identity), h = column gather (or identity); values
// outside r < R, k < Kc, or at a negative gather index, are written as 0, and
// (not transposed) so are source rows sr with zero_if[sr] != 0.
//
// Row-wise conversion: a block covers 16 rows x 128 columns, a thread 8
// consecutive columns of one row, written as one 16-byte vector per plane.
__global__ void __launch_bounds__(256) to_planes_kernel(Planes dst, int64_t R, int64_t Kc,
                                                        const uint16_t *__restrict__ src, int64_t lds, int64_t col_off,
                                                        const int32_t *__restrict__ rgather,
                                                        const int32_t *__restrict__ cgather,
                                                        const int32_t *__restrict__ zero_if, ModP mp)
{
    const int tid = threadIdx.x;
    const int64_t r = (int64_t)blockIdx.y * 16 + (tid >> 4);
    const int64_t k0 = (int64_t)blockIdx.x * 128 + (int64_t)(tid & 15) * 8;
    int64_t sr = -1;
    if (r < R) {
        sr = rgather ? (int64_t)rgather[r] : r;
        if (sr >= 0 && zero_if && zero_if[sr]) sr = -1;
    }
    uint32_t a[8];
    if (!cgather) {
        uint16_t w[8];
        if (sr >= 0 && k0 < Kc) {
            load8_u16(src + sr * lds + col_off + k0, Kc - k0, w);
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) w[e] = 0;
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) a[e] = w[e];
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int64_t k = k0 + e;
            a[e] = 0;
            if (sr >= 0 && k < Kc) {
                const int64_t sc = cgather[k];
                if (sc >= 0) a[e] = src[sr * lds + col_off + sc];
            }
        }
    }
    store_digits8(dst, r, k0, a, mp);
}

// Transposed conversion: dst row r, column dst_col0 + k <- src[g(k)][col_off + r],
// one 64 x 64 tile per block.  With k_le_r_only, tiles whose every k exceeds every
// r are skipped (their planes are left unwritten): for the transpose of an
// upper triangular matrix those entries are zero and no product reads them.
__global__ void __launch_bounds__(256) to_planes_t_kernel(Planes dst, int64_t R, int64_t Kc,
                                                          const uint16_t *__restrict__ src, int64_t lds,
                                                          int64_t col_off, const int32_t *__restrict__ rgather,
                                                          int k_le_r_only, int64_t dst_col0, ModP mp)
{
    __shared__ TpSmem sm;
    const int64_t k0 = (int64_t)blockIdx.x * TP_TILE, r0 = (int64_t)blockIdx.y * TP_TILE;
    if (k_le_r_only && k0 > r0 + TP_TILE - 1) return;
    tp_tile(dst, 0, r0, k0, R, Kc, src, lds, col_off, rgather, mp, sm, dst_col0);
}

int to_planes(const Planes &dst, int64_t R, int64_t Kc, const uint16_t *src, int64_t lds,
              int64_t col_off, bool transposed, const int32_t *rgather, const int32_t *cgather,
              const ModP &mp, cudaStream_t s, const int32_t *zero_if, bool k_le_r_only, int64_t dst_col0)
{
    if (dst.rows <= 0 || dst.kp <= 0) return GBLA_OK;
    if (dst_col0 % 128 || (dst_col0 && !transposed)) return GBLA_E_INTERNAL;
    // Cover the logical rectangle rounded up to whole 128 x 128 tiles (the
    // product reads nothing else); the rest of the buffer is left as is.
    const int64_t rows = round_up(R > 0 ? R : 1, 128) < dst.rows ? round_up(R > 0 ? R : 1, 128) : dst.rows;
    const int64_t kav = dst.kp - dst_col0;   // columns available from dst_col0
    const int64_t ks = round_up(Kc > 0 ? Kc : 1, 128) < kav ? round_up(Kc > 0 ? Kc : 1, 128) : kav;
    if (ks <= 0) return GBLA_E_INTERNAL;
    if (transposed) {
        dim3 grid((unsigned)(ks / TP_TILE), (unsigned)(rows / TP_TILE));
        to_planes_t_kernel<<<grid, 256, 0, s>>>(dst, R, Kc, src, lds, col_off, rgather, k_le_r_only ? 1 : 0,
                                                 dst_col0, mp);
    } else {
        dim3 grid((unsigned)(ks / 128), (unsigned)(rows / 16));
        to_planes_kernel<<<grid, 256, 0, s>>>(dst, R, Kc, src, lds, col_off, rgather, cgather, zero_if, mp);
    }
    GBLA_CUDA_TRY(launch_check());
    return GBLA_OK;
}

// ===================================================================
// SIMT reference GEMM (exact int64)
// ===================================================================
__device__ __forceinline__ int bf2i(__nv_bfloat16 v) { return (int)__bfloat162float(v); }

__global__ void __launch_bounds__(256) modgemm_simt_kernel(Planes A, int64_t a_row0, int64_t a_k0, Planes B,
                                                           int64_t b_row0, int64_t b_k0, uint16_t *C, int64_t ldc,
                                                           const int32_t *__restrict__ c_rows, int64_t M, int64_t N,
                                                           int64_t K, int sign, ModP mp)
{
    __shared__ int sa[64][33];
    __shared__ int sb[64][33];
    const int tid = threadIdx.x;
    const int tr = tid / 16, tc = tid % 16;   // 16 x 16 threads, 4 x 4 outputs each
    const int64_t m0 = (int64_t)blockIdx.y * 64, n0 = (int64_t)blockIdx.x * 64;
    long long acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0;
    for (int64_t kk = 0; kk < K; kk += 32) {
        for (int e = tid; e < 64 * 32; e += 256) {
            int r = e / 32, k = e % 32;
            int va = 0, vb = 0;
            if (kk + k < K) {
                if (m0 + r < M) {
                    const int64_t ar = a_row0 + m0 + r, ak = a_k0 + kk + k;
                    va = 256 * bf2i(*A.at(0, ar, ak)) + bf2i(*A.at(1, ar, ak));
                }
                if (n0 + r < N) {
                    const int64_t br = b_row0 + n0 + r, bk = b_k0 + kk + k;
                    vb = 256 * bf2i(*B.at(0, br, bk)) + bf2i(*B.at(1, br, bk));
                }
            }
            sa[r][k] = va;
            sb[r][k] = vb;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            int a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sa[tr * 4 + i][k];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = sb[tc * 4 + j][k];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += (long long)a[i] * b[j];
        }
        __syncthreads();
    }
    const long long P = mp.p;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t r = m0 + tr * 4 + i;
        if (r >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t c = n0 + tc * 4 + j;
            if (c >= N) continue;
            long long v = acc[i][j] % P;
            if (v < 0) v += P;
            const int64_t pr = c_rows ? (int64_t)c_rows[r] : r;
            if (pr < 0) continue;
            long long cur = C[pr * ldc + c];
            long long o = sign > 0 ? (cur + v) % P : (cur - v + P) % P;
            C[pr * ldc + c] = (uint16_t)o;
        }
    }
}

// ===================================================================
// tcgen05 / TMA GEMM
// ===================================================================
namespace tc {
constexpr int BM = 128, BN = 128, BK = 32;         // K step: one 32-wide chunk of the interleaved planes
constexpr int STAGES = 4;
constexpr int KSTEPS_PER_BLOCK = 512 / BK;          // k-block of 512: exact fp32 sums
constexpr int BOX_BYTES = 128 * 128;                // one TMA box: 128 rows x 128 bytes (two planes)
constexpr int STAGE_BYTES = 3 * BOX_BYTES;          // [Ah Al] | [Bh Bl] | [B'h B'l]
constexpr int BAR_BYTES = 256;
// CTA pair (cta_group::2): one 256 x 128 tile per pair, each CTA holding 128
// rows of A and 64 rows of B per stage (32 KiB).
constexpr int PAIR_STAGES = 4;
constexpr int PAIR_B_BOX_BYTES = 64 * 128;                          // 64 rows x 128 bytes
constexpr int PAIR_STAGE_BYTES = BOX_BYTES + 2 * PAIR_B_BOX_BYTES;  // [Ah Al] | [Bh Bl] | [B'h B'l]
constexpr int64_t GROUP_M_DEFAULT = 4;              // row tiles per raster group (see tile_coords)
constexpr int EPI_WARPS = 8;                        // two drain warps per TMEM lane quarter
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + BAR_BYTES + 1024;
constexpr int PAIR_SMEM_BYTES = PAIR_STAGES * PAIR_STAGE_BYTES + BAR_BYTES + 1024;
constexpr uint32_t TMEM_COLS = 512;                 // 2 buffers x (P 128 + Q 128)
constexpr float MAGIC = 12582912.0f;                // 1.5 * 2^23
constexpr long long WAIT_LIMIT_CYCLES = 2000000000ll;  // ~1 s

struct Args {
    int64_t M, N, K;
    const GroupProb *probs;  // grouped mode: nprob problems (device), else null
    int nprob;
    int32_t a_row0, a_k0;    // first row and K column of the A and B operands
    int32_t b_row0, b_k0;
    uint16_t *C;
    int64_t ldc;
    const int32_t *c_rows;   // optional: row r of the product goes to C row c_rows[r]
    const int32_t *row_lead; // optional: ascending first nonzero K index of each A row
    int sign;
    uint32_t p;
    float pinv;              // 1/p rounded to fp32 (p >= 8)
    uint32_t *err;
    int withhold_loads;      // test hook: issue no TMA loads, so the waits expire
    int group_m;             // row tiles per raster group
    Planes xout;             // planes-out mode (xout.ptr set): the product itself, as
    int64_t xout_col0;       // A-operand digit planes at row xout_row0 + m, column
    int64_t xout_row0;       // xout_col0 + n; C unused
    int a_pitch;             // elements per 32-wide K chunk of an A row: 64 (2 planes) or
                             // 128 (a 4-plane set read as its first two planes); 0 = 64
    unsigned long long *work; // optional: += valid rows x valid columns x K run, per tile
};

__device__ __forceinline__ uint32_t smem_u32(const void *ptr) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(ptr));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: returns false (and raises the abort flag and the timeout
// bit) if the phase does not complete within WAIT_LIMIT_CYCLES, or if
// another role already aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, uint32_t *err) {
    const uint32_t addr = smem_u32(bar);
    long long start = 0;
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(addr, parity)) return true;
        if ((it & 255u) == 255u) {
            if (*abort_flag) return false;
            long long now = clock64();
            if (start == 0) start = now;
            else if (now - start > WAIT_LIMIT_CYCLES) {
                *abort_flag = 1;
                dev_fail(err, DEV_ERR_TIMEOUT);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// CTA-pair forms.  The pair's loads all complete on the leader's (rank 0)
// barrier, given as a shared::cluster address.
__device__ __forceinline__ void tma_load_2d_pair(void *dst, const CUtensorMap *map, uint32_t bar_cluster, int x,
                                                 int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
        "%4}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar_cluster), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// shared::cluster address of the variable at saddr in the CTA of the given rank
__device__ __forceinline__ uint32_t mapa_rank(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster) : "memory");
}

__device__ __forceinline__ void tcgen05_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tcgen05_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand of 128 rows with 128-byte
// rows, loaded by TMA with 128-byte swizzle.  Each 128-byte row holds two
// planes' 32-wide K chunks; an operand (one plane, 16 K values) is selected
// by the start address offset within the row (0, 32, 64 or 96 bytes), which
// the swizzle applies to like any other address bits.  8-row swizzle atoms
// are 1024 bytes apart (stride byte offset); the leading byte offset is unused
// for swizzled K-major tiles.  Layout type 2 = 128-byte swizzle; bit 46 is
// the fixed descriptor version of sm_100-family tcgen05.
__device__ __forceinline__ uint64_t make_sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                 // leading byte offset (16 B, unused)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset: 8 rows of 128 B
    d |= (uint64_t)1 << 46;                 // descriptor version
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: D = f32, A = B = bf16, both K-major,
// N = 128, M = 128.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

// CTA pair: M = 256 (rows 0..127 in the leader's TMEM, 128..255 in the peer's).
constexpr uint32_t IDESC_PAIR = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                ((uint32_t)((2 * BM) >> 4) << 24);

// One K = 16 step of the digit products for a stage: four MMAs issued by an
// elected lane of the converged MMA warp,
//   P += ah * b'h,  Q += ah * b'l,  P += al * bh,  Q += al * bl,
// with descriptor low words a (ah; al = a + 4), b1 (bh; bl = b1 + 4) and b2
// (b'h; b'l = b2 + 4) and the common high word hi.
template <bool PAIR>
__device__ __forceinline__ void mma_step(uint32_t dP, uint32_t dQ, uint32_t a, uint32_t b1, uint32_t b2, uint32_t hi,
                                         uint32_t acc0) {
    if (PAIR)
        asm volatile("{\n\t.reg .pred p, e;\n\t.reg .b32 r;\n\t.reg .b64 a0, a1, x0, x1, y0, y1;\n\t"
                     "elect.sync r|e, 0xffffffff;\n\t"
                     "setp.ne.b32 p, %7, 0;\n\t"
                     "mov.b64 a0, {%2, %5};\n\t"
                     "add.u32 r, %2, 4;\n\tmov.b64 a1, {r, %5};\n\t"
                     "mov.b64 x0, {%3, %5};\n\t"
                     "add.u32 r, %3, 4;\n\tmov.b64 x1, {r, %5};\n\t"
                     "mov.b64 y0, {%4, %5};\n\t"
                     "add.u32 r, %4, 4;\n\tmov.b64 y1, {r, %5};\n\t"
                     "@e tcgen05.mma.cta_group::2.kind::f16 [%0], a0, y0, %6, p;\n\t"
                     "@e tcgen05.mma.cta_group::2.kind::f16 [%1], a0, y1, %6, p;\n\t"
                     "@e tcgen05.mma.cta_group::2.kind::f16 [%0], a1, x0, %6, 1;\n\t"
                     "@e tcgen05.mma.cta_group::2.kind::f16 [%1], a1, x1, %6, 1;\n\t}" ::"r"(dP),
                     "r"(dQ), "r"(a), "r"(b1), "r"(b2), "r"(hi), "r"(IDESC_PAIR), "r"(acc0)
                     : "memory");
    else
        asm volatile("{\n\t.reg .pred p, e;\n\t.reg .b32 r;\n\t.reg .b64 a0, a1, x0, x1, y0, y1;\n\t"
                     "elect.sync r|e, 0xffffffff;\n\t"
                     "setp.ne.b32 p, %7, 0;\n\t"
                     "mov.b64 a0, {%2, %5};\n\t"
                     "add.u32 r, %2, 4;\n\tmov.b64 a1, {r, %5};\n\t"
                     "mov.b64 x0, {%3, %5};\n\t"
                     "add.u32 r, %3, 4;\n\tmov.b64 x1, {r, %5};\n\t"
                     "mov.b64 y0, {%4, %5};\n\t"
                     "add.u32 r, %4, 4;\n\tmov.b64 y1, {r, %5};\n\t"
                     "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a0, y0, %6, p;\n\t"
                     "@e tcgen05.mma.cta_group::1.kind::f16 [%1], a0, y1, %6, p;\n\t"
                     "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a1, x0, %6, 1;\n\t"
                     "@e tcgen05.mma.cta_group::1.kind::f16 [%1], a1, x1, %6, 1;\n\t}" ::"r"(dP),
                     "r"(dQ), "r"(a), "r"(b1), "r"(b2), "r"(hi), "r"(IDESC), "r"(acc0)
                     : "memory");
}

// tcgen05.commit from an elected lane of a converged warp.
template <bool PAIR, bool BOTH>
__device__ __forceinline__ void commit_elected(uint64_t *bar) {
    if (PAIR && BOTH)
        asm volatile("{\n\t.reg .pred e;\n\t.reg .b32 r;\n\telect.sync r|e, 0xffffffff;\n\t"
                     "@e tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;\n\t}"
                     ::"r"(smem_u32(bar)), "h"((uint16_t)3)
                     : "memory");
    else if (PAIR)
        asm volatile("{\n\t.reg .pred e;\n\t.reg .b32 r;\n\telect.sync r|e, 0xffffffff;\n\t"
                     "@e tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(
                         smem_u32(bar))
                     : "memory");
    else
        asm volatile("{\n\t.reg .pred e;\n\t.reg .b32 r;\n\telect.sync r|e, 0xffffffff;\n\t"
                     "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(
                         smem_u32(bar))
                     : "memory");
}

// Warp-uniform bounded wait: every lane polls; a completed phase stays
// complete until this warp consumes it, so any lane's success is the warp's.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t *bar, uint32_t parity, volatile int *abort_flag, uint32_t *err) {
    const uint32_t addr = smem_u32(bar);
    if (__any_sync(0xffffffffu, mbar_try_wait(addr, parity))) return true;
    long long start = clock64();
    for (uint32_t it = 0;; ++it) {
        if (__any_sync(0xffffffffu, mbar_try_wait(addr, parity))) return true;
        if ((it & 255u) == 255u) {
            if (__any_sync(0xffffffffu, *abort_flag != 0)) return false;
            if (clock64() - start > WAIT_LIMIT_CYCLES) {
                if ((threadIdx.x & 31) == 0) {
                    *abort_flag = 1;
                    dev_fail(err, DEV_ERR_TIMEOUT);
                }
                __syncwarp();
                return false;
            }
        }
    }
}



__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// One drained k-block of one element: returns (run + 256*pa + qa) mod p in
// [0, p) for run in [0, p) and exact accumulators |pa|, |qa| <= 2^24.  Both
// accumulators convert exactly to integers; pa's quotient q by p comes from
// one fused multiply-add into the 2^23 rounding window (the rounded
// reciprocal moves pa/p by at most 1/8 for p >= 8, so |pa - q*p| <= 5p/8).
// Everything else is integer work, which unlike fp32 work does not slow the
// concurrent tensor-core MMAs.  With bias = 256p + ceil(2^24/p)*p, the value
// t = run + 256*(pa - q*p) + qa + bias lies in [96p, 2^25 + 418p), below
// 2^26, so floor(t * bm / 2^32) with bm = floor(2^32 / p) is floor(t/p) or
// one less and a single conditional subtraction finishes the reduction.
__device__ __forceinline__ int drain_step(int run, float pa, float qa, float pinv, int P, int bias, uint32_t bm) {
    const int ip = __float2int_rn(pa);
    const int iq = __float2int_rn(qa);
    const int qp = __float_as_int(fmaf(pa, pinv, MAGIC)) - 0x4B400000;
    const int rp = ip - qp * P;
    const uint32_t t = (uint32_t)(run + bias + iq + 256 * rp);
    int s = (int)(t - __umulhi(t, bm) * (uint32_t)P);
    s -= (s >= P) ? P : 0;
    return s;
}

// C <- (C + sign * run) mod p on one drain thread's row segment: HC columns
// from column col0 of C (crow points at it), columns >= ncol untouched.
constexpr int HC_COLS = BN / 2;   // columns per drain warp
__device__ __forceinline__ void rmw_segment(uint16_t *crow, int64_t col0, int64_t ncol,
                                            const uint32_t (&run)[HC_COLS / 2], int sign, int P) {
    constexpr int HC = HC_COLS;
    const bool aligned = (reinterpret_cast<uintptr_t>(crow) & 15u) == 0;
    // Chunks of 8 columns: whole in-range chunks move as 16-byte vectors, a
    // ragged or unaligned chunk element by element.  Every load is issued
    // before the first store.
    uint4 cv[HC / 8];
#pragma unroll
    for (int v = 0; v < HC / 8; ++v) {
        const int64_t cbase = col0 + v * 8;
        if (aligned && cbase + 8 <= ncol) {
            cv[v] = reinterpret_cast<const uint4 *>(crow)[v];
        } else {
            uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (cbase + e < ncol) w[e >> 1] |= (uint32_t)crow[v * 8 + e] << ((e & 1) * 16);
            cv[v] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
#pragma unroll
    for (int v = 0; v < HC / 8; ++v) {
        uint32_t w[4] = {cv[v].x, cv[v].y, cv[v].z, cv[v].w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            uint32_t rr = run[v * 4 + e];
            int c0 = (int)(w[e] & 0xFFFFu), c1 = (int)(w[e] >> 16);
            int r0 = (int)(rr & 0xFFFFu), r1 = (int)(rr >> 16);
            int o0 = sign > 0 ? c0 + r0 : c0 - r0;
            int o1 = sign > 0 ? c1 + r1 : c1 - r1;
            o0 += (o0 < 0) ? P : 0; o0 -= (o0 >= P) ? P : 0;
            o1 += (o1 < 0) ? P : 0; o1 -= (o1 >= P) ? P : 0;
            w[e] = (uint32_t)o0 | ((uint32_t)o1 << 16);
        }
        cv[v] = make_uint4(w[0], w[1], w[2], w[3]);
    }
#pragma unroll
    for (int v = 0; v < HC / 8; ++v) {
        const int64_t cbase = col0 + v * 8;
        if (aligned && cbase + 8 <= ncol) {
            reinterpret_cast<uint4 *>(crow)[v] = cv[v];
        } else {
            const uint32_t w[4] = {cv[v].x, cv[v].y, cv[v].z, cv[v].w};
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (cbase + e < ncol) crow[v * 8 + e] = (uint16_t)(w[e >> 1] >> ((e & 1) * 16));
        }
    }
}

__device__ __forceinline__ void tile_coords(int64_t t, int64_t num_m, int64_t num_n, int64_t GM, int64_t &mt,
                                            int64_t &nt) {
    int64_t group = t / (GM * num_n);
    int64_t first_m = group * GM;
    int64_t gm = num_m - first_m < GM ? num_m - first_m : GM;
    int64_t in = t % (GM * num_n);
    mt = first_m + in % gm;
    nt = in / gm;
}

// First k-step of tile row mt: A rows are zero left of their lead, and with
// leads ascending the first row of the tile's raster group has the smallest
// one.  All tiles of a group start there, so the CTAs working on the group at
// the same time walk K in step and share operand tiles in L2.
__device__ __forceinline__ int tile_kstep0(const Args &g, int64_t mt, int64_t tbm) {
    if (!g.row_lead) return 0;
    const int64_t k = (int64_t)g.row_lead[(mt / g.group_m) * g.group_m * tbm] - g.a_k0;
    return k > 0 ? (int)(k / BK) & ~(STAGES - 1) : 0;   // whole rounds of the stage ring
}

struct TileInfo {
    int64_t mt, nt, M, N, c_col0;
    int a_row, b_row, ks0;
    const int32_t *c_rows;
};

// Tile t of the launch.  Pair tiles are 256 rows high: the CTA of rank 1
// loads A rows 128.. and B rows 64.. of it and drains rows 128.. of C.
template <bool PAIR>
__device__ __forceinline__ TileInfo tile_info(const Args &g, int64_t t, int64_t num_m, int64_t num_n, uint32_t rank) {
    TileInfo ti;
    if (g.probs) {
        int lo = 0, hi = g.nprob - 1;   // last problem with tile_off <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (g.probs[mid].tile_off <= t) lo = mid;
            else hi = mid - 1;
        }
        const GroupProb &P = g.probs[lo];
        const int64_t local = t - P.tile_off;
        const int64_t nm = (P.M + BM - 1) / BM;
        ti.mt = local % nm;
        ti.nt = local / nm;
        ti.M = P.M;
        ti.N = P.N;
        ti.c_col0 = P.c_col0;
        ti.c_rows = P.c_rows;
        ti.a_row = P.a_row0 + (int)(ti.mt * BM);
        ti.b_row = P.b_row0 + (int)(ti.nt * BN);
        ti.ks0 = 0;
    } else {
        constexpr int64_t TBM = PAIR ? 2 * BM : BM;
        tile_coords(t, num_m, num_n, g.group_m, ti.mt, ti.nt);
        ti.M = g.M;
        ti.N = g.N;
        ti.c_col0 = 0;
        ti.c_rows = g.c_rows;
        ti.a_row = g.a_row0 + (int)(ti.mt * TBM) + (int)rank * BM;
        ti.b_row = g.b_row0 + (int)(ti.nt * BN) + (int)rank * (BN / 2);
        ti.ks0 = tile_kstep0(g, ti.mt, TBM);
    }
    return ti;
}

// PAIR = false: one CTA per 128 x 128 tile (cta_group::1).  PAIR = true: a
// cluster of two CTAs per 256 x 128 tile (cta_group::2, launched with cluster
// dimension 2); the leader (rank 0) issues the MMAs, which read A and B from
// both CTAs' shared memory and write each CTA's 128 rows of the accumulators
// into its own TMEM.  All loads of a stage complete on the leader's full
// barrier; the MMA commits arrive on the empty and accumulator barriers of
// both CTAs; both CTAs' drain warps release an accumulator buffer on the
// leader's barrier.
template <bool PAIR>
__global__ void __launch_bounds__(tc::THREADS, 1)
    modgemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const Args g)
{
    constexpr int NST = PAIR ? PAIR_STAGES : STAGES;
    constexpr int SBYTES = PAIR ? PAIR_STAGE_BYTES : STAGE_BYTES;
    constexpr int BBOX = PAIR ? PAIR_B_BOX_BYTES : BOX_BYTES;
    constexpr int64_t TBM = PAIR ? 2 * BM : BM;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *tiles = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(tiles + NST * SBYTES);
    uint64_t *full = bars;
    uint64_t *empty = bars + NST;
    uint64_t *accf = bars + 2 * NST;
    uint64_t *acce = accf + 2;
    uint64_t *done = acce + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
    const bool leader = rank == 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], PAIR ? 2 * EPI_WARPS : EPI_WARPS);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        if (PAIR) {
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(tmem_slot)),
                         "r"(TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(tmem_slot)),
                         "r"(TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
    }
    if (warp == 0 && lane == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
    }
    tcgen05_fence_before();
    __syncthreads();
    if (PAIR) cluster_sync();   // the peer's barriers exist before any remote signal
    tcgen05_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int64_t num_m = (g.M + TBM - 1) / TBM, num_n = (g.N + BN - 1) / BN;
    const int64_t num_tiles = g.probs ? g.probs[g.nprob].tile_off : num_m * num_n;
    // K steps run in whole rounds of the 4-stage ring (steps past K read zero
    // padding): every tile starts at stage 0, and the MMA issuer's stage
    // offsets are compile-time constants.
    static_assert(STAGES == 4 && PAIR_STAGES == 4 && KSTEPS_PER_BLOCK % 4 == 0, "ring rounds");
    const int ksteps = (int)(((g.K + BK - 1) / BK + 3) & ~int64_t(3));
    const int64_t tile0 = PAIR ? (int64_t)(blockIdx.x >> 1) : (int64_t)blockIdx.x;
    const int64_t tstep = PAIR ? (int64_t)(gridDim.x >> 1) : (int64_t)gridDim.x;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer
            int stage = 0;
            uint32_t phase = 0;
            int issued[NST];
            uint32_t issued_parity[NST];
            for (int s = 0; s < NST; ++s) issued[s] = 0, issued_parity[s] = 0;
            bool ok = !g.withhold_loads;
            for (int64_t t = tile0; t < num_tiles && ok; t += tstep) {
                const TileInfo ti = tile_info<PAIR>(g, t, num_m, num_n, rank);
                const int ay = ti.a_row, by = ti.b_row;
                for (int ks = ti.ks0; ks < ksteps; ++ks) {
                    if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, g.err)) { ok = false; break; }
                    uint8_t *st = tiles + stage * SBYTES;
                    // chunk c of K sits at element 64 c of an A row (2 planes)
                    // and 128 c of a B row (4 planes)
                    const int ax = (g.a_k0 / BK + ks) * (g.a_pitch ? g.a_pitch : 2 * BK),
                              bx = (g.b_k0 / BK + ks) * 4 * BK;
                    if (PAIR) {
                        const uint32_t fb = mapa_rank(smem_u32(&full[stage]), 0);
                        if (leader) mbar_expect_tx(&full[stage], 2 * SBYTES);
                        tma_load_2d_pair(st, &tmA, fb, ax, ay);
                        tma_load_2d_pair(st + BOX_BYTES, &tmB, fb, bx, by);
                        tma_load_2d_pair(st + BOX_BYTES + BBOX, &tmB, fb, bx + 2 * BK, by);
                    } else {
                        mbar_expect_tx(&full[stage], SBYTES);
                        tma_load_2d(st, &tmA, &full[stage], ax, ay);
                        tma_load_2d(st + BOX_BYTES, &tmB, &full[stage], bx, by);
                        tma_load_2d(st + BOX_BYTES + BBOX, &tmB, &full[stage], bx + 2 * BK, by);
                    }
                    issued[stage] = 1;
                    issued_parity[stage] = phase;
                    if (++stage == NST) stage = 0, phase ^= 1u;
                }
            }
            // Never leave with copies in flight: wait (bounded) for the last
            // load issued into every stage.  A pair's copies complete on the
            // leader's barriers, which count the peer's bytes too; the peer,
            // which cannot wait on them, pauses after an abort instead.
            if (PAIR && !leader) {
                if (!ok) {
                    const long long start = clock64();
                    while (clock64() - start < 4000000ll) __nanosleep(1000);
                }
            } else {
                for (int s = 0; s < NST; ++s) {
                    if (!issued[s]) continue;
                    const uint32_t addr = smem_u32(&full[s]);
                    long long start = clock64();
                    while (!mbar_try_wait(addr, issued_parity[s])) {
                        if (clock64() - start > WAIT_LIMIT_CYCLES) {
                            dev_fail(g.err, DEV_ERR_TIMEOUT);
                            break;
                        }
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (leader) {
            // ---------------- MMA issuer: the whole warp runs the loop, an
            // elected lane issues.  The loop is unrolled over the 4 stages of
            // the ring so that every descriptor is a constant offset from one
            // register: the tensor core starves if the issuing warp spends
            // more than a few instructions between MMAs (measured).
            uint32_t phase = 0;
            uint32_t kbc = 0;
            bool ok = true;
            const uint64_t d0 = make_sdesc(smem_u32(tiles));
            const uint32_t dhi = (uint32_t)(d0 >> 32), lo0 = (uint32_t)d0;
            constexpr uint32_t SB = SBYTES >> 4, B1 = BOX_BYTES >> 4, B2 = (BOX_BYTES + BBOX) >> 4;
            for (int64_t t = tile0; t < num_tiles && ok; t += tstep) {
                const int ks0 = tile_info<PAIR>(g, t, num_m, num_n, rank).ks0;
                const int kbt = (ksteps - ks0 + KSTEPS_PER_BLOCK - 1) / KSTEPS_PER_BLOCK;
                for (int kb = 0; kb < kbt && ok; ++kb, ++kbc) {
                    const uint32_t buf = kbc & 1u, use = kbc >> 1;
                    if (!mbar_wait_warp(&acce[buf], (use & 1u) ^ 1u, abort_flag, g.err)) { ok = false; break; }
                    tcgen05_fence_after();
                    const uint32_t dP = tmem + buf * 256u, dQ = dP + 128u;
                    const int ks_beg = ks0 + kb * KSTEPS_PER_BLOCK;
                    const int ks_end = min(ksteps, ks_beg + KSTEPS_PER_BLOCK);
                    uint32_t acc0 = 0;
                    for (int ks = ks_beg; ks < ks_end && ok; ks += NST) {
#pragma unroll
                        for (int st = 0; st < NST; ++st) {
                            // the stage's operands were written by TMA and the
                            // barrier completes with them: no thread-sync fence
                            if (!mbar_wait_warp(&full[st], phase, abort_flag, g.err)) { ok = false; break; }
                            const uint32_t a = lo0 + st * SB;
                            mma_step<PAIR>(dP, dQ, a, a + B1, a + B2, dhi, acc0);
                            mma_step<PAIR>(dP, dQ, a + 2, a + 2 + B1, a + 2 + B2, dhi, 1u);   // next 16 of K
                            acc0 = 1u;
                            commit_elected<PAIR, true>(&empty[st]);
                        }
                        phase ^= 1u;
                    }
                    if (ok) commit_elected<PAIR, true>(&accf[buf]);
                }
            }
            // Wait (bounded) until every issued MMA has completed before the
            // accumulators are released.
            commit_elected<PAIR, false>(done);
            const uint32_t addr = smem_u32(done);
            long long start = clock64();
            while (!__any_sync(0xffffffffu, mbar_try_wait(addr, 0))) {
                if (clock64() - start > WAIT_LIMIT_CYCLES) {
                    if (lane == 0) dev_fail(g.err, DEV_ERR_TIMEOUT);
                    break;
                }
            }
        }
    } else {
        // ---------------- epilogue: warps 2..9.  A warp may only read the TMEM
        // lane quarter warp % 4; the two warps of a quarter split the columns.
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const int row_in_tile = quarter * 32 + lane;
        const float pinv = g.pinv;
        const int P = (int)g.p;
        // Barrett multiplier floor(2^32 / p) (p odd) and a multiple of p that
        // keeps the combined value positive
        const uint32_t bm = 0xFFFFFFFFu / g.p;
        const int bias = 256 * P + (int)(((1u << 24) + g.p - 1) / g.p) * P;
        constexpr int HC = BN / 2;    // columns per drain warp
        uint32_t kbc = 0;
        bool ok = true;
        for (int64_t t = tile0; t < num_tiles && ok; t += tstep) {
            const TileInfo ti = tile_info<PAIR>(g, t, num_m, num_n, rank);
            const int kbt = (ksteps - ti.ks0 + KSTEPS_PER_BLOCK - 1) / KSTEPS_PER_BLOCK;
            if (kbt <= 0) continue;   // the product is zero on this tile: C stays as it is
            if (g.work && warp == 2 && lane == 0) {
                const int64_t vr = min((int64_t)TBM, ti.M - ti.mt * TBM), vc = min((int64_t)BN, ti.N - ti.nt * BN);
                const int64_t kr = g.K - (int64_t)ti.ks0 * BK;
                if (vr > 0 && vc > 0 && kr > 0 && (!PAIR || rank == 0))
                    atomicAdd(g.work, (unsigned long long)(vr * vc * kr));
            }
            uint32_t run[HC / 2];
#pragma unroll
            for (int i = 0; i < HC / 2; ++i) run[i] = 0;
            for (int kb = 0; kb < kbt; ++kb, ++kbc) {
                const uint32_t buf = kbc & 1u, use = kbc >> 1;
                if (!mbar_wait(&accf[buf], use & 1u, abort_flag, g.err)) { ok = false; break; }
                tcgen05_fence_after();
                const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + buf * 256u + half * HC;
#pragma unroll
                for (int c = 0; c < HC / 16; ++c) {
                    float pv[16], qv[16];
                    tmem_ld16(tbase + c * 16, pv);
                    tmem_ld16(tbase + 128 + c * 16, qv);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 16; j += 2) {
                        uint32_t pair = run[c * 8 + j / 2];
                        const int lo16 = drain_step((int)(pair & 0xFFFFu), pv[j], qv[j], pinv, P, bias, bm);
                        const int hi16 = drain_step((int)(pair >> 16), pv[j + 1], qv[j + 1], pinv, P, bias, bm);
                        run[c * 8 + j / 2] = (uint32_t)lo16 | ((uint32_t)hi16 << 16);
                    }
                }
                tcgen05_fence_before();
                __syncwarp();
                if (lane == 0) {
                    if (PAIR) mbar_arrive_cluster(mapa_rank(smem_u32(&acce[buf]), 0));
                    else mbar_arrive(&acce[buf]);
                }
            }
            if (!ok) break;
            if (g.xout.ptr) {
                // planes-out: the product's digits, 16-byte stores per plane
                const int64_t row = ti.mt * TBM + (int64_t)rank * BM + row_in_tile;
                if (row < ti.M) {
                    const int64_t orow = g.xout_row0 + row;
                    const int64_t k0 = g.xout_col0 + ti.nt * BN + half * HC;
#pragma unroll
                    for (int v = 0; v < HC / 8; ++v) {
                        uint32_t vh[4], vl[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const uint32_t rr = run[v * 4 + e];
                            int h0, l0, h1, l1;
                            digits(rr & 0xFFFFu, g.p, h0, l0);
                            digits(rr >> 16, g.p, h1, l1);
                            vh[e] = pack_bf2(h0, h1);
                            vl[e] = pack_bf2(l0, l1);
                        }
                        *reinterpret_cast<uint4 *>(g.xout.at(0, orow, k0 + v * 8)) = make_uint4(vh[0], vh[1], vh[2], vh[3]);
                        *reinterpret_cast<uint4 *>(g.xout.at(1, orow, k0 + v * 8)) = make_uint4(vl[0], vl[1], vl[2], vl[3]);
                    }
                }
                continue;
            }
            // C <- (C + sign * run) mod p for this thread's row segment.
            const int64_t row = ti.mt * TBM + (int64_t)rank * BM + row_in_tile;
            const int64_t col0 = ti.c_col0 + ti.nt * BN + half * HC;   // column of C
            const int64_t ncol = ti.c_col0 + ti.N;                        // column limit
            const int64_t prow = (row < ti.M && ti.c_rows) ? (int64_t)ti.c_rows[row] : row;
            if (row < ti.M && col0 < ncol && prow >= 0)
                rmw_segment(g.C + prow * g.ldc + col0, col0, ncol, run, g.sign, P);
        }
    }
    tcgen05_fence_before();
    __syncthreads();
    if (PAIR) cluster_sync();   // the leader's MMAs may write the peer's TMEM until here
    if (warp == 1) {
        tcgen05_fence_after();
        if (PAIR)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                         : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                         : "memory");
    }
}

// ===================================================================
// Gathered product: the sparse operand compacted per column tile
// ===================================================================
// C[r, c] <- (C[r, c] + sign * sum_j X[r, j] * S[j, c]) mod p for the output
// column tiles nt0 .. of a compacted sparse operand S (sparse.cu): the rows j
// of S with a nonzero in tile t are listed in kidx[koff[t] .. koff[t + 1])
// (ascending, padded to a multiple of 128 entries with KIDX_PAD), and S
// restricted to those rows and the tile's 128 columns is stored densely as
// the two digit planes (hi, lo) of its residues, 32 list entries per
// 128 x 64-bf16 chunk.  The
// product's K is the list: K-compaction keeps the tensor cores on the
// nonzero part of S.  X is read through its transpose: row j of the
// A-operand plane set XT holds column j of X, so the 128 values of a row tile
// and both planes are 512 contiguous bytes; the gather warps copy them for
// every listed j into shared memory in the MN-major 128-byte-swizzled layout
// (cp.async), while one thread loads the compacted S chunk by TMA.  Rows of X
// are ascending by lead (first nonzero column), so a tile skips the list
// entries left of its first row's lead.
// The four digit products go to four fp32 accumulators,
//     a*b = 65536*(ah*bh) + 256*(ah*bl + al*bh) + al*bl   (balanced digits),
// H, M1 = sum ah*bl, M2 = sum al*bh and L (all 512 TMEM columns, one buffer:
// the MMA issuer waits for the drain between k-blocks).  Each takes one
// product of at most 2^14 per list entry, so a k-block of 1,024 entries
// keeps every sum within 2^24 and exact: the drain runs once per 32 k-steps.
// Without the 256*b mod p planes a stage is 32 KB (16 KB of gathered X^T,
// 16 KB of S), so the ring holds six stages and six copies of X^T rows are in
// flight.
// Warp roles: 0 TMA producer of the compacted operand, 1 MMA issuer, 2..9
// drain (two per TMEM lane quarter, 64 columns each), 10..15 gather (warp
// 10 + s fills ring slot s).
constexpr int G_STAGES = 6;
constexpr int G_KSTEPS_PER_BLOCK = 1024 / BK;
constexpr int G_A_BYTES = 128 * 128;                 // 32 entries x 128 rows x 2 planes
constexpr int G_B_BYTES = 128 * 128;                 // 128 columns x 32 entries x 2 planes
constexpr int G_STAGE_BYTES = G_A_BYTES + G_B_BYTES;
constexpr int G_EPI_WARPS = 8;
constexpr int G_GATHER_WARPS = G_STAGES;
constexpr int G_THREADS = 64 + 32 * G_EPI_WARPS + 32 * G_GATHER_WARPS;
// The drain's running residues (128 rows x 128 columns, two per word) live in
// shared memory after the ring, column pair major so that the 32 lanes of a
// warp (32 rows) touch 32 banks.
constexpr int G_RUN_BYTES = BM * BN * 2;
constexpr int G_SMEM_BYTES = G_STAGES * G_STAGE_BYTES + BAR_BYTES + 1024 + G_RUN_BYTES;

// Ties registers written by tcgen05.ld to the point after tcgen05.wait::ld,
// so that no use of them is scheduled before the wait.
__device__ __forceinline__ void reg_fence16(float (&v)[16]) {
#pragma unroll
    for (int i = 0; i < 16; ++i) asm volatile("" : "+f"(v[i]));
}
__device__ __forceinline__ void reg_fence8(float (&v)[8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i) asm volatile("" : "+f"(v[i]));
}
// 8 columns of a TMEM lane quarter (one 32-bit value per lane and column).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// (run + 65536 H + 256 (M1 + M2) + L) mod p for the four digit-product sums
// of the gathered product (integers of magnitude at most 2^24 in fp32), in
// full-rate float and integer operations only.  Each sum x is brought to
// r = x - q p with q = x / p rounded (|x / p| < 2^22, so adding 1.5 * 2^23
// rounds it to an integer); the fma forms r exactly, |r| <= p / 2 + 1, and
// adding 1.5 * 2^23 again leaves r + 0x4B400000 as the word's bits.  Then
// c16 * r_H + 256 (r_M1 + r_M2) + r_L (c16 = 65536 mod p, balanced) has
// magnitude below 2^30 + 2^25; biasx is a multiple of p from 2^30 + 2^26 less
// the four 0x4B400000 offsets (taken mod 2^32), so the 32-bit sum is the true
// nonnegative value, below 2^31 + 2^27, and one Barrett step with a single
// correction finishes it.
__device__ __forceinline__ uint32_t reduce_to_word(float x, float pinv, float pf) {
    const float q = fmaf(x, pinv, MAGIC) - MAGIC;
    return __float_as_uint(fmaf(-q, pf, x) + MAGIC);
}
__device__ __forceinline__ uint32_t drain_step4(uint32_t run, float ha, float m1a, float m2a, float la, float pinv,
                                                float pf, uint32_t c16, uint32_t biasx, uint32_t bm, uint32_t P) {
    const uint32_t rh = reduce_to_word(ha, pinv, pf);
    const uint32_t rm = reduce_to_word(m1a, pinv, pf) + reduce_to_word(m2a, pinv, pf);
    const uint32_t rl = reduce_to_word(la, pinv, pf);
    const uint32_t t = run + biasx + rl + 256u * rm + c16 * rh;
    const uint32_t s = t - __umulhi(t, bm) * P;
    return min(s, s - P);
}

struct GArgs {
    int64_t M, N;            // rows of X taking part; output columns (from column 0 of C)
    int64_t nt0;             // list of output tile nt is list nt0 + nt
    const int32_t *kidx;     // compacted lists
    const int64_t *koff;     // list offsets
    const __nv_bfloat16 *xt; // XT plane set (2 planes, rows = j, K = r)
    int64_t xt_row_elems;    // elements per XT row
    int64_t xt_rows;         // list entries >= xt_rows are padding (their rows of S are zero)
    const int32_t *kstart;   // [row tiles x output tiles]: first list entry of the tile's
                             // K range (0 without row leads), from gather_starts_kernel
    uint16_t *C;
    int64_t ldc;
    int sign;
    uint32_t p;
    float pinv;
    uint32_t *err;
    int group_m;
};

// First list entry at or after the first lead of the row tile, for every
// (row tile, output tile): the tile walks K from there (X is zero left of a
// row's lead, rows ascending by lead).  One thread per entry, a binary
// search.  With exec (optional), also adds the list entries the launch runs
// through (from each tile's rounded start to the list end): the executed
// product is exec * 128 * 128 multiply-adds.
__global__ void gather_starts_kernel(int64_t num_m, int64_t num_n, int64_t nt0, const int64_t *__restrict__ koff,
                                     const int32_t *__restrict__ kidx, const int32_t *__restrict__ row_lead,
                                     int32_t *__restrict__ kstart, unsigned long long *exec)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long run = 0;   // list entries this tile runs through
    if (i < num_m * num_n) {
        const int64_t mt = i / num_n, nt = i % num_n;
        const int64_t kb = koff[nt0 + nt], ke = koff[nt0 + nt + 1];
        int64_t lo = kb, hi = ke;
        if (row_lead) {
            const int32_t L = row_lead[mt * BM];
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (kidx[mid] < L) lo = mid + 1;
                else hi = mid;
            }
        }
        kstart[i] = (int32_t)(lo - kb);
        run = (unsigned long long)(ke - kb - (lo - kb) / BK * BK);   // from the start gtile rounds to
    }
    if (exec) {   // one atomic per warp
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) run += __shfl_xor_sync(0xFFFFFFFFu, run, o);
        if ((threadIdx.x & 31) == 0 && run) atomicAdd(exec, run);
    }
}

struct GTile {
    int64_t mt, nt, chunk0;
    int ks0, ksteps;
};

__device__ __forceinline__ GTile gtile(const GArgs &g, int64_t t, int64_t num_m, int64_t num_n) {
    GTile ti;
    tile_coords(t, num_m, num_n, g.group_m, ti.mt, ti.nt);
    const int64_t kb = g.koff[g.nt0 + ti.nt], ke = g.koff[g.nt0 + ti.nt + 1];
    ti.chunk0 = kb / BK;
    ti.ksteps = (int)((ke - kb) / BK);
    const int64_t s = g.kstart ? (int64_t)g.kstart[ti.mt * num_n + ti.nt] : 0;
    ti.ks0 = (int)(s / BK);
    return ti;
}

// Shared-memory descriptor of an MN-major operand with 128-byte swizzle:
// atoms of 8 K-rows x 128 bytes (64 values of M), atoms along M 1024 bytes
// apart (leading byte offset), along K 2048 bytes apart (stride byte offset).
__device__ __forceinline__ uint64_t make_sdesc_mn(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(1024 >> 4) << 16;       // leading byte offset: next 64 rows of M
    d |= (uint64_t)(2048 >> 4) << 32;       // stride byte offset: next 8 values of K
    d |= (uint64_t)1 << 46;                 // descriptor version
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}

// kind::f16 instruction descriptor with A MN-major (transposed), B K-major.
constexpr uint32_t IDESC_G = IDESC | (1u << 15);

// One K = 16 step: A planes ah (a) and al (a + 8 KB), B planes bh (b) and bl
// (b + 64 bytes);  H += ah*bh, M1 += ah*bl, M2 += al*bh, L += al*bl (TMEM
// columns d, d + 128, d + 256, d + 384).
__device__ __forceinline__ void mma_step_g4(uint32_t d, uint32_t a, uint32_t b, uint32_t ahi, uint32_t bhi,
                                            uint32_t acc0) {
    asm volatile("{\n\t.reg .pred p, e;\n\t.reg .b32 r, d1, d2, d3;\n\t.reg .b64 a0, a1, x0, x1;\n\t"
                 "elect.sync r|e, 0xffffffff;\n\t"
                 "setp.ne.b32 p, %6, 0;\n\t"
                 "add.u32 d1, %0, 128;\n\tadd.u32 d2, %0, 256;\n\tadd.u32 d3, %0, 384;\n\t"
                 "mov.b64 a0, {%1, %3};\n\t"
                 "add.u32 r, %1, 512;\n\tmov.b64 a1, {r, %3};\n\t"
                 "mov.b64 x0, {%2, %4};\n\t"
                 "add.u32 r, %2, 4;\n\tmov.b64 x1, {r, %4};\n\t"
                 "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a0, x0, %5, p;\n\t"
                 "@e tcgen05.mma.cta_group::1.kind::f16 [d1], a0, x1, %5, p;\n\t"
                 "@e tcgen05.mma.cta_group::1.kind::f16 [d2], a1, x0, %5, p;\n\t"
                 "@e tcgen05.mma.cta_group::1.kind::f16 [d3], a1, x1, %5, p;\n\t}" ::"r"(d),
                 "r"(a), "r"(b), "r"(ahi), "r"(bhi), "r"(IDESC_G), "r"(acc0)
                 : "memory");
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__global__ void __launch_bounds__(tc::G_THREADS, 1)
    modgemm_gather_kernel(const __grid_constant__ CUtensorMap tmB, const GArgs g)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *tiles = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(tiles + G_STAGES * G_STAGE_BYTES);
    uint64_t *full = bars;
    uint64_t *empty = bars + G_STAGES;
    uint64_t *accf = bars + 2 * G_STAGES;
    uint64_t *acce = accf + 1;
    uint64_t *done = acce + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    uint32_t *run_s = reinterpret_cast<uint32_t *>(tiles + G_STAGES * G_STAGE_BYTES + BAR_BYTES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < G_STAGES; ++s) {
            mbar_init(&full[s], 1 + 32);   // the TMA thread and the slot's gather warp
            mbar_init(&empty[s], 1);
        }
        mbar_init(accf, 1);
        mbar_init(acce, G_EPI_WARPS);
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (warp == 0 && lane == 0)
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
    tcgen05_fence_before();
    __syncthreads();
    tcgen05_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int64_t num_m = (g.M + BM - 1) / BM, num_n = (g.N + BN - 1) / BN;
    const int64_t num_tiles = num_m * num_n;
    const int64_t tile0 = blockIdx.x, tstep = gridDim.x;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer of the compacted operand
            int stage = 0;
            uint32_t phase = 0;
            int issued[G_STAGES];
            uint32_t issued_parity[G_STAGES];
            for (int s = 0; s < G_STAGES; ++s) issued[s] = 0, issued_parity[s] = 0;
            bool ok = true;
            for (int64_t t = tile0; t < num_tiles && ok; t += tstep) {
                const GTile ti = gtile(g, t, num_m, num_n);
                for (int ks = ti.ks0; ks < ti.ksteps; ++ks) {
                    if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, g.err)) { ok = false; break; }
                    uint8_t *st = tiles + stage * G_STAGE_BYTES;
                    const int y = (int)((ti.chunk0 + ks) * BN);
                    mbar_expect_tx(&full[stage], G_B_BYTES);
                    tma_load_2d(st + G_A_BYTES, &tmB, &full[stage], 0, y);
                    issued[stage] = 1;
                    issued_parity[stage] = phase;
                    if (++stage == G_STAGES) stage = 0, phase ^= 1u;
                }
            }
            for (int s = 0; s < G_STAGES; ++s) {   // never leave with copies in flight
                if (!issued[s]) continue;
                const uint32_t addr = smem_u32(&full[s]);
                long long start = clock64();
                while (!mbar_try_wait(addr, issued_parity[s])) {
                    if (clock64() - start > WAIT_LIMIT_CYCLES) {
                        dev_fail(g.err, DEV_ERR_TIMEOUT);
                        break;
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (converged warp, elected lane)
        uint32_t phase = 0, kbc = 0;
        int st = 0;
        bool ok = true;
        const uint32_t s0 = smem_u32(tiles);
        const uint64_t da = make_sdesc_mn(s0), db = make_sdesc(s0);
        const uint32_t ahi = (uint32_t)(da >> 32), alo = (uint32_t)da;
        const uint32_t bhi = (uint32_t)(db >> 32), blo = (uint32_t)db + (G_A_BYTES >> 4);
        constexpr uint32_t SB = G_STAGE_BYTES >> 4;
        for (int64_t t = tile0; t < num_tiles && ok; t += tstep) {
            const GTile ti = gtile(g, t, num_m, num_n);
            const int kbt = (ti.ksteps - ti.ks0 + G_KSTEPS_PER_BLOCK - 1) / G_KSTEPS_PER_BLOCK;
            for (int kb = 0; kb < kbt && ok; ++kb, ++kbc) {
                if (!mbar_wait_warp(acce, (kbc & 1u) ^ 1u, abort_flag, g.err)) { ok = false; break; }
                tcgen05_fence_after();
                const int ks_beg = ti.ks0 + kb * G_KSTEPS_PER_BLOCK;
                const int ks_end = min(ti.ksteps, ks_beg + G_KSTEPS_PER_BLOCK);
                uint32_t acc0 = 0;
                for (int ks = ks_beg; ks < ks_end; ++ks) {
                    if (!mbar_wait_warp(&full[st], phase, abort_flag, g.err)) { ok = false; break; }
                    // the gather threads' copies are made visible to the
                    // tensor core by their proxy fence before they arrive
                    tcgen05_fence_after();
                    const uint32_t a = alo + (uint32_t)st * SB, b = blo + (uint32_t)st * SB;
                    mma_step_g4(tmem, a, b, ahi, bhi, acc0);
                    mma_step_g4(tmem, a + 256, b + 2, ahi, bhi, 1u);   // next 16 of K
                    acc0 = 1u;
                    commit_elected<false, true>(&empty[st]);
                    if (++st == G_STAGES) st = 0, phase ^= 1u;
                }
                if (ok) commit_elected<false, true>(accf);
            }
        }
        commit_elected<false, false>(done);
        const uint32_t addr = smem_u32(done);
        long long start = clock64();
        while (!__any_sync(0xffffffffu, mbar_try_wait(addr, 0))) {
            if (clock64() - start > WAIT_LIMIT_CYCLES) {
                if (lane == 0) dev_fail(g.err, DEV_ERR_TIMEOUT);
                break;
            }
        }
    } else if (warp < 2 + G_EPI_WARPS) {
        // ---------------- drain: two warps per TMEM lane quarter, 64 columns
        // each (column half `half`); otherwise as in modgemm_tc_kernel
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const int row_in_tile = quarter * 32 + lane;
        const float pinv = g.pinv, pf = (float)g.p;
        const int P = (int)g.p;
        const uint32_t bm = 0xFFFFFFFFu / g.p;
        uint32_t c16 = 65536u % g.p;
        if (c16 > g.p / 2) c16 -= g.p;   // 65536 mod p, balanced (as a 32-bit word)
        const uint32_t biasx = ((1u << 30) + (1u << 26) + g.p - 1) / g.p * g.p - 0x4B400000u * (513u + c16);
        constexpr int HC = BN / 2;
        uint32_t kbc = 0;
        bool ok = true;
        for (int64_t t = tile0; t < num_tiles && ok; t += tstep) {
            const GTile ti = gtile(g, t, num_m, num_n);
            const int kbt = (ti.ksteps - ti.ks0 + G_KSTEPS_PER_BLOCK - 1) / G_KSTEPS_PER_BLOCK;
            if (kbt <= 0) continue;   // no list entry on this tile: C stays as it is
            // column pair i of this warp's half at rs[128 i]
            uint32_t *rs = run_s + half * (HC / 2) * BM + row_in_tile;
#pragma unroll 8
            for (int i = 0; i < HC / 2; ++i) rs[BM * i] = 0;
            for (int kb = 0; kb < kbt; ++kb, ++kbc) {
                if (!mbar_wait(accf, kbc & 1u, abort_flag, g.err)) { ok = false; break; }
                tcgen05_fence_after();
                const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + half * HC;
#pragma unroll 1
                for (int c = 0; c < HC / 16; ++c) {
                    float hv[16], m1v[16], m2v[16], lv[16];
                    tmem_ld16(tbase + c * 16, hv);
                    tmem_ld16(tbase + 128 + c * 16, m1v);
                    tmem_ld16(tbase + 256 + c * 16, m2v);
                    tmem_ld16(tbase + 384 + c * 16, lv);
                    tmem_wait_ld();
                    reg_fence16(hv);
                    reg_fence16(m1v);
                    reg_fence16(m2v);
                    reg_fence16(lv);
                    if (c + 1 == HC / 16) {   // every accumulator read: the MMA may go on
                        tcgen05_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(acce);
                    }
#pragma unroll
                    for (int j = 0; j < 16; j += 2) {
                        const uint32_t pair = rs[BM * (c * 8 + j / 2)];
                        const uint32_t lo16 = drain_step4(pair & 0xFFFFu, hv[j], m1v[j], m2v[j], lv[j], pinv, pf,
                                                          c16, biasx, bm, g.p);
                        const uint32_t hi16 = drain_step4(pair >> 16, hv[j + 1], m1v[j + 1], m2v[j + 1],
                                                          lv[j + 1], pinv, pf, c16, biasx, bm, g.p);
                        rs[BM * (c * 8 + j / 2)] = lo16 | (hi16 << 16);
                    }
                }
            }
            if (!ok) break;
            const int64_t row = ti.mt * BM + row_in_tile;
            const int64_t col0 = ti.nt * BN + half * HC;
            if (row < g.M && col0 < g.N) {
                uint32_t part[HC / 2];
#pragma unroll
                for (int i = 0; i < HC / 2; ++i) part[i] = rs[BM * i];
                rmw_segment(g.C + row * g.ldc + col0, col0, g.N, part, g.sign, P);
            }
        }
    } else {
        // ---------------- gather warps: warp 10 + s fills ring slot s with
        // the X^T rows of the stage's 32 listed j (MN-major, 128-byte
        // swizzle), cp.async 16 bytes at a time.  Copy i: list entry kk =
        // i / 32 (one instruction moves an entry's 512 bytes), piece q = i % 32
        // = lane, holding rows rl .. rl + 7 (rl = 32 (q / 8) + 8 (q % 4)) of
        // plane (q / 4) % 2.  The warp reads the stage's list entries with one
        // load (lane l: entry l) before its wait for the slot, waits for its
        // own copies, fences them to the tensor core's proxy and signals; the
        // other slots' warps go on independently.  (Vector loads through
        // registers in place of cp.async measured 1.9x slower here.)
        const int slot = warp - 2 - G_EPI_WARPS;
        const uint32_t abase = smem_u32(tiles) + slot * G_STAGE_BYTES;
        const int q = lane;
        const int rl = (q >> 3) * 32 + (q & 3) * 8;
        const uint32_t dst_lane = ((q >> 2) & 1) * 8192 + (rl >> 6) * 1024 + ((((rl & 63) >> 3)) << 4);
        int ring = 0;   // ring slot of the next k-step, as the producer and the MMA issuer count it
        uint32_t use = 0;
        bool ok = true;
        for (int64_t t = tile0; t < num_tiles && ok; t += tstep) {
            const GTile ti = gtile(g, t, num_m, num_n);
            const __nv_bfloat16 *xseg = g.xt + (ti.mt * BM / 32) * 64 + q * 8;   // this lane's piece
            for (int ks = ti.ks0; ks < ti.ksteps; ++ks) {
                const int mine = ring;
                if (++ring == G_STAGES) ring = 0;
                if (mine != slot) continue;
                const int64_t kbase = (ti.chunk0 + ks) * BK;
                const int32_t jl = g.kidx[kbase + lane];
                if (!mbar_wait_warp(&empty[slot], (use & 1u) ^ 1u, abort_flag, g.err)) { ok = false; break; }
#pragma unroll 8
                for (int kk = 0; kk < BK; ++kk) {
                    int64_t j = __shfl_sync(0xFFFFFFFFu, jl, kk);
                    // a padding entry's row of S is zero: any row of X^T serves
                    // (row 0; the zero-fill form of cp.async measured 9% slower)
                    if (j >= g.xt_rows) j = 0;
                    // 16-byte chunk index XOR the row within the swizzle atom
                    const uint32_t dst = abase + (kk >> 3) * 2048 + (kk & 7) * 128 + (dst_lane ^ ((kk & 7) << 4));
                    cp_async16(dst, xseg + j * g.xt_row_elems);
                }
                cp_async_commit();
                cp_async_wait<0>();
                fence_proxy_async();
                mbar_arrive(&full[slot]);
                ++use;
            }
        }
        cp_async_wait<0>();   // nothing in flight when the warp leaves
    }

    tcgen05_fence_before();
    __syncthreads();
    if (warp == 1) {
        tcgen05_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}
// ===================================================================
// Fused panel application of an echelon wave (see panel_apply)
// ===================================================================
// One work item = (job q, 128-column block cb of D from the job's first
// column).  Per item: the loader copies the job's t pivot rows of D at the
// block's columns (u16, one bulk copy per row) into a staging tile; four
// converter warps turn the tile into the B operand's two digit planes
// (B[col][k] = D[S_k][col], K-major, 128-byte swizzle, four 32-wide K steps);
// the producer loads the job's A block (K = 128) by TMA, one 16 KB K step per
// ring stage, for each of the item's 128-row tiles; the MMA warp accumulates
// the four digit products H, M1, M2, L (512 TMEM columns; K = 128 keeps every
// sum within 2^21) and eight drain warps add (65536 H + 256 (M1 + M2) + L)
// mod p into the tile's rows of D, whose old values they fetch before the
// products arrive.  B is double-buffered across items; TMEM is released as
// soon as the drain has read it.
// Warp roles: 0 A producer, 1 MMA issuer, 2..9 drain, 10 loader, 11..14
// converters.
constexpr int PA_STAGES = 4;                       // = K steps of one 128-row tile
constexpr int PA_A_BYTES = 128 * 128;              // 128 rows x (32 K x 2 planes)
constexpr int PA_B_BYTES = 4 * 128 * 128;          // 4 K steps x 128 columns x (32 K x 2 planes)
constexpr int PA_STG_BYTES = 128 * 256;            // 128 rows x 128 u16
constexpr int PA_EPI_WARPS = 8;
constexpr int PA_CONV_WARPS = 4;
constexpr int PA_THREADS = 64 + 32 * PA_EPI_WARPS + 32 + 32 * PA_CONV_WARPS;
constexpr int PA_SMEM_BYTES = PA_STAGES * PA_A_BYTES + 2 * PA_B_BYTES + PA_STG_BYTES + BAR_BYTES + 1024;
static_assert(PA_SMEM_BYTES <= 232448, "shared memory");

// The four sums of a product with K <= 128 (each at most 2^21; M1 + M2 at
// most 2^22 and exact in fp32), reduced to (65536 H + 256 (M1 + M2) + L)
// mod p: H and M1 + M2 by a rounded quotient (as reduce_to_word), L read
// straight through the 1.5 * 2^23 window.  c16 * r_H + 256 r_M + L has
// magnitude below 2^30 + 2^24; biasy is a multiple of p from 2^30 + 2^24
// less the three 0x4B400000 offsets (mod 2^32), so the 32-bit sum is the true
// nonnegative value, below 2^31 + 2^25.
__device__ __forceinline__ uint32_t drain_step4_k128(float ha, float m1a, float m2a, float la, float pinv, float pf,
                                                     uint32_t c16, uint32_t biasy, uint32_t bm, uint32_t P) {
    const uint32_t rh = reduce_to_word(ha, pinv, pf);
    const uint32_t rm = reduce_to_word(m1a + m2a, pinv, pf);
    const uint32_t lw = __float_as_uint(la + MAGIC);
    const uint32_t t = biasy + lw + 256u * rm + c16 * rh;
    const uint32_t s = t - __umulhi(t, bm) * P;
    return min(s, s - P);
}

struct PaArgs {
    const PaJob *jobs;
    int njobs;
    const int32_t *rowmap;
    uint16_t *D;
    int64_t ldd, n;
    uint32_t p;
    float pinv;
    uint32_t *err;
};

struct PaItem {
    int q, cb, nmt;
    int64_t a_row0, col0;   // col0: first column of the block
    int t, M;
    const int32_t *srows;
};

__device__ __forceinline__ PaItem pa_item(const PaArgs &g, int64_t it) {
    int lo = 0, hi = g.njobs - 1;   // last job with item_off <= it
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (g.jobs[mid].item_off <= it) lo = mid;
        else hi = mid - 1;
    }
    const PaJob &J = g.jobs[lo];
    PaItem x;
    x.q = lo;
    x.cb = (int)(it - J.item_off);
    x.M = J.M;
    x.t = J.t;
    x.nmt = (J.M + BM - 1) / BM;
    x.a_row0 = J.a_row0;
    x.col0 = J.col0 + (int64_t)x.cb * BN;
    x.srows = J.srows;
    return x;
}

// One K = 16 step, both operands K-major with two planes per 128-byte row
// (hi at the descriptor, lo 64 bytes on): H += ah*bh, M1 += ah*bl,
// M2 += al*bh, L += al*bl (TMEM columns d, d + 128, d + 256, d + 384).
__device__ __forceinline__ void mma_step_k4(uint32_t d, uint32_t a, uint32_t b, uint32_t hi, uint32_t acc0) {
    asm volatile("{\n\t.reg .pred p, e;\n\t.reg .b32 r, d1, d2, d3;\n\t.reg .b64 a0, a1, x0, x1;\n\t"
                 "elect.sync r|e, 0xffffffff;\n\t"
                 "setp.ne.b32 p, %5, 0;\n\t"
                 "add.u32 d1, %0, 128;\n\tadd.u32 d2, %0, 256;\n\tadd.u32 d3, %0, 384;\n\t"
                 "mov.b64 a0, {%1, %3};\n\t"
                 "add.u32 r, %1, 4;\n\tmov.b64 a1, {r, %3};\n\t"
                 "mov.b64 x0, {%2, %3};\n\t"
                 "add.u32 r, %2, 4;\n\tmov.b64 x1, {r, %3};\n\t"
                 "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a0, x0, %4, p;\n\t"
                 "@e tcgen05.mma.cta_group::1.kind::f16 [d1], a0, x1, %4, p;\n\t"
                 "@e tcgen05.mma.cta_group::1.kind::f16 [d2], a1, x0, %4, p;\n\t"
                 "@e tcgen05.mma.cta_group::1.kind::f16 [d3], a1, x1, %4, p;\n\t}" ::"r"(d),
                 "r"(a), "r"(b), "r"(hi), "r"(IDESC), "r"(acc0)
                 : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__global__ void __launch_bounds__(tc::PA_THREADS, 1)
    panel_apply_kernel(const __grid_constant__ CUtensorMap tmA, const PaArgs g)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sa = base;                                        // A ring
    uint8_t *sb = base + PA_STAGES * PA_A_BYTES;               // B planes, two buffers
    uint16_t *stg = reinterpret_cast<uint16_t *>(sb + 2 * PA_B_BYTES);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sb + 2 * PA_B_BYTES + PA_STG_BYTES);
    uint64_t *afull = bars;
    uint64_t *aempty = bars + PA_STAGES;
    uint64_t *bfull = bars + 2 * PA_STAGES;
    uint64_t *bempty = bfull + 2;
    uint64_t *sfull = bempty + 2;
    uint64_t *sempty = sfull + 1;
    uint64_t *accf = sempty + 1;
    uint64_t *acce = accf + 1;
    uint64_t *done = acce + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < PA_STAGES; ++s) {
            mbar_init(&afull[s], 1);
            mbar_init(&aempty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bfull[b], 32 * PA_CONV_WARPS);
            mbar_init(&bempty[b], 1);
        }
        mbar_init(sfull, 1);
        mbar_init(sempty, 32 * PA_CONV_WARPS);
        mbar_init(accf, 1);
        mbar_init(acce, PA_EPI_WARPS);
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (warp == 0 && lane == 0)
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    tcgen05_fence_before();
    __syncthreads();
    tcgen05_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t total = g.jobs[g.njobs].item_off;
    const int64_t it0 = blockIdx.x, itstep = gridDim.x;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- A producer: the item's row tiles, K step by K step
            int st = 0;
            uint32_t phase = 0;
            int issued[PA_STAGES];
            uint32_t issued_parity[PA_STAGES];
            for (int s = 0; s < PA_STAGES; ++s) issued[s] = 0, issued_parity[s] = 0;
            bool ok = true;
            for (int64_t it = it0; it < total && ok; it += itstep) {
                const PaItem x = pa_item(g, it);
                for (int mt = 0; mt < x.nmt && ok; ++mt) {
                    for (int ks = 0; ks < PA_STAGES; ++ks) {
                        if (!mbar_wait(&aempty[st], phase ^ 1u, abort_flag, g.err)) { ok = false; break; }
                        mbar_expect_tx(&afull[st], PA_A_BYTES);
                        tma_load_2d(sa + st * PA_A_BYTES, &tmA, &afull[st], ks * 2 * BK, (int)(x.a_row0 + mt * BM));
                        issued[st] = 1;
                        issued_parity[st] = phase;
                        if (++st == PA_STAGES) st = 0, phase ^= 1u;
                    }
                }
            }
            for (int s = 0; s < PA_STAGES; ++s) {   // never leave with copies in flight
                if (!issued[s]) continue;
                const uint32_t addr = smem_u32(&afull[s]);
                long long start = clock64();
                while (!mbar_try_wait(addr, issued_parity[s])) {
                    if (clock64() - start > WAIT_LIMIT_CYCLES) {
                        dev_fail(g.err, DEV_ERR_TIMEOUT);
                        break;
                    }
                }
            }
        }
    } else if (warp == 2 + PA_EPI_WARPS) {
        // ---------------- loader: the pivot rows' u16 values at the block's
        // columns, one bulk copy per row (whole 16-byte chunks inside the
        // row; the converters read a ragged tail directly)
        uint32_t use = 0;
        bool ok = true;
        int pending = 0;
        uint32_t pending_parity = 0;
        for (int64_t it = it0; it < total && ok; it += itstep, ++use) {
            const PaItem x = pa_item(g, it);
            if (!mbar_wait_warp(sempty, (use & 1u) ^ 1u, abort_flag, g.err)) { ok = false; break; }
            const int64_t avail = g.n - x.col0;                      // >= 1
            const int64_t wcols = (avail >= BN ? BN : avail) & ~int64_t(7);
            const uint32_t rbytes = (uint32_t)(wcols * 2);
            if (lane == 0) mbar_expect_tx(sfull, rbytes * (uint32_t)x.t);
            __syncwarp();
            if (rbytes > 0)
                for (int k = lane; k < x.t; k += 32)
                    bulk_copy_g2s(smem_u32(stg + k * BN), g.D + (int64_t)x.srows[k] * g.ldd + x.col0, rbytes,
                                  smem_u32(sfull));
            pending = 1;
            pending_parity = use & 1u;
        }
        if (pending) {   // never leave with copies in flight
            const uint32_t addr = smem_u32(sfull);
            long long start = clock64();
            while (!__any_sync(0xffffffffu, mbar_try_wait(addr, pending_parity))) {
                if (clock64() - start > WAIT_LIMIT_CYCLES) {
                    if (lane == 0) dev_fail(g.err, DEV_ERR_TIMEOUT);
                    break;
                }
            }
        }
    }
    else if (warp > 2 + PA_EPI_WARPS) {
        // ---------------- converters: thread j (0..127) owns column j of the
        // block and writes the 16 chunks of 8 K values of its B row: hi and lo
        // digits of D[S_k][col0 + j], k = 32 ks + 8 c .. + 7, at 16-byte chunk
        // c (hi) and 4 + c (lo) of row j of K step ks, XOR j mod 8 (128-byte
        // swizzle).
        const int j = threadIdx.x - 32 * (3 + PA_EPI_WARPS);
        const uint32_t P = g.p;
        uint32_t use = 0;
        bool ok = true;
        for (int64_t it = it0; it < total && ok; it += itstep, ++use) {
            const PaItem x = pa_item(g, it);
            const uint32_t buf = use & 1u, bu = use >> 1;
            if (!mbar_wait_warp(sfull, use & 1u, abort_flag, g.err)) { ok = false; break; }
            if (!mbar_wait_warp(&bempty[buf], (bu & 1u) ^ 1u, abort_flag, g.err)) { ok = false; break; }
            const int64_t avail = g.n - x.col0;
            const int64_t wcols = (avail >= BN ? BN : avail) & ~int64_t(7);
            const bool live = j < avail;                 // column inside D
            const bool staged = j < wcols;               // copied by the loader
            uint8_t *brow = sb + buf * PA_B_BYTES + j * 128;
#pragma unroll 1
            for (int i = 0; i < 16; ++i) {
                const int ks = i >> 2, c = i & 3, k0 = 32 * ks + 8 * c;
                uint32_t vh[4], vl[4];
#pragma unroll
                for (int e = 0; e < 8; e += 2) {
                    uint32_t a0 = 0, a1 = 0;
                    if (live && k0 + e < x.t)
                        a0 = staged ? stg[(k0 + e) * BN + j] : g.D[(int64_t)x.srows[k0 + e] * g.ldd + x.col0 + j];
                    if (live && k0 + e + 1 < x.t)
                        a1 = staged ? stg[(k0 + e + 1) * BN + j]
                                    : g.D[(int64_t)x.srows[k0 + e + 1] * g.ldd + x.col0 + j];
                    int h0, l0, h1, l1;
                    digits(a0, P, h0, l0);
                    digits(a1, P, h1, l1);
                    vh[e / 2] = pack_bf2(h0, h1);
                    vl[e / 2] = pack_bf2(l0, l1);
                }
                uint8_t *bk = brow + ks * (128 * 128);
                *reinterpret_cast<uint4 *>(bk + ((c ^ (j & 7)) << 4)) = make_uint4(vh[0], vh[1], vh[2], vh[3]);
                *reinterpret_cast<uint4 *>(bk + (((4 + c) ^ (j & 7)) << 4)) = make_uint4(vl[0], vl[1], vl[2], vl[3]);
            }
            mbar_arrive(sempty);   // the staging tile is read
            fence_proxy_async();   // the planes, to the tensor core's proxy
            mbar_arrive(&bfull[buf]);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (converged warp, elected lane)
        int st = 0;
        uint32_t phase = 0, use = 0, mtc = 0;
        bool ok = true;
        const uint64_t d0 = make_sdesc(smem_u32(base));
        const uint32_t hi = (uint32_t)(d0 >> 32), alo = (uint32_t)d0;
        const uint32_t blo = alo + ((PA_STAGES * PA_A_BYTES) >> 4);
        constexpr uint32_t SA = PA_A_BYTES >> 4, SKB = (128 * 128) >> 4, SBB = PA_B_BYTES >> 4;
        for (int64_t it = it0; it < total && ok; it += itstep, ++use) {
            const PaItem x = pa_item(g, it);
            const uint32_t buf = use & 1u, bu = use >> 1;
            if (!mbar_wait_warp(&bfull[buf], bu & 1u, abort_flag, g.err)) { ok = false; break; }
            for (int mt = 0; mt < x.nmt && ok; ++mt, ++mtc) {
                if (!mbar_wait_warp(acce, (mtc & 1u) ^ 1u, abort_flag, g.err)) { ok = false; break; }
                tcgen05_fence_after();
                for (int ks = 0; ks < PA_STAGES; ++ks) {
                    if (!mbar_wait_warp(&afull[st], phase, abort_flag, g.err)) { ok = false; break; }
                    tcgen05_fence_after();
                    const uint32_t a = alo + (uint32_t)st * SA, b = blo + buf * SBB + (uint32_t)ks * SKB;
                    mma_step_k4(tmem, a, b, hi, ks > 0 ? 1u : 0u);
                    mma_step_k4(tmem, a + 2, b + 2, hi, 1u);   // next 16 of K
                    commit_elected<false, false>(&aempty[st]);
                    if (++st == PA_STAGES) st = 0, phase ^= 1u;
                }
                if (ok) commit_elected<false, false>(accf);
            }
            if (ok) commit_elected<false, false>(&bempty[buf]);
        }
        commit_elected<false, false>(done);
        const uint32_t addr = smem_u32(done);
        long long start = clock64();
        while (!__any_sync(0xffffffffu, mbar_try_wait(addr, 0))) {
            if (clock64() - start > WAIT_LIMIT_CYCLES) {
                if (lane == 0) dev_fail(g.err, DEV_ERR_TIMEOUT);
                break;
            }
        }
    } else {
        // ---------------- drain: warp 2 + 4 h + q reads TMEM lane quarter q,
        // columns 64 h .. 64 h + 63, and updates row q * 32 + lane of the
        // tile: D <- (D + (65536 H + 256 (M1 + M2) + L)) mod p
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        constexpr int HC = BN / 2;
        const float pinv = g.pinv, pf = (float)g.p;
        const uint32_t P = g.p;
        const uint32_t bm = 0xFFFFFFFFu / g.p;
        uint32_t c16 = 65536u % g.p;
        if (c16 > g.p / 2) c16 -= g.p;
        const uint32_t biasy = ((1u << 30) + (1u << 24) + g.p - 1) / g.p * g.p - 0x4B400000u * (257u + c16);
        uint32_t mtc = 0;
        bool ok = true;
        for (int64_t it = it0; it < total && ok; it += itstep) {
            const PaItem x = pa_item(g, it);
            const int64_t col0 = x.col0 + half * HC;
            for (int mt = 0; mt < x.nmt; ++mt, ++mtc) {
                const int rl = mt * BM + quarter * 32 + lane;
                const int64_t drow = rl < x.M ? (int64_t)g.rowmap[x.a_row0 + rl] : -1;
                uint16_t *crow = drow >= 0 ? g.D + drow * g.ldd + col0 : nullptr;
                const bool vec = crow && col0 + HC <= g.n && (reinterpret_cast<uintptr_t>(crow) & 15) == 0;
                // old values first: their latency overlaps the products
                uint32_t cw[HC / 2];
                if (vec) {
#pragma unroll
                    for (int v = 0; v < HC / 8; ++v) {
                        const uint4 q4 = reinterpret_cast<const uint4 *>(crow)[v];
                        cw[4 * v] = q4.x, cw[4 * v + 1] = q4.y, cw[4 * v + 2] = q4.z, cw[4 * v + 3] = q4.w;
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < HC / 2; ++i) {
                        uint32_t w = 0;
                        if (crow && col0 + 2 * i < g.n) w = crow[2 * i];
                        if (crow && col0 + 2 * i + 1 < g.n) w |= (uint32_t)crow[2 * i + 1] << 16;
                        cw[i] = w;
                    }
                }
                if (!mbar_wait(accf, mtc & 1u, abort_flag, g.err)) { ok = false; break; }
                tcgen05_fence_after();
                const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + half * HC;
#pragma unroll
                for (int c = 0; c < HC / 8; ++c) {   // unrolled: cw stays in registers
                    float hv[8], m1v[8], m2v[8], lv[8];
                    tmem_ld8(tbase + c * 8, hv);
                    tmem_ld8(tbase + 128 + c * 8, m1v);
                    tmem_ld8(tbase + 256 + c * 8, m2v);
                    tmem_ld8(tbase + 384 + c * 8, lv);
                    tmem_wait_ld();
                    reg_fence8(hv);
                    reg_fence8(m1v);
                    reg_fence8(m2v);
                    reg_fence8(lv);
                    if (c + 1 == HC / 8) {   // every accumulator read: the MMA may go on
                        tcgen05_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(acce);
                    }
#pragma unroll
                    for (int e = 0; e < 8; e += 2) {
                        const uint32_t v0 = drain_step4_k128(hv[e], m1v[e], m2v[e], lv[e], pinv, pf, c16, biasy, bm, P);
                        const uint32_t v1 =
                            drain_step4_k128(hv[e + 1], m1v[e + 1], m2v[e + 1], lv[e + 1], pinv, pf, c16, biasy, bm, P);
                        const uint32_t w = cw[c * 4 + e / 2];
                        uint32_t o0 = (w & 0xFFFFu) + v0, o1 = (w >> 16) + v1;
                        o0 -= o0 >= P ? P : 0u;
                        o1 -= o1 >= P ? P : 0u;
                        cw[c * 4 + e / 2] = o0 | (o1 << 16);
                    }
                }
                if (vec) {
#pragma unroll
                    for (int v = 0; v < HC / 8; ++v)
                        reinterpret_cast<uint4 *>(crow)[v] =
                            make_uint4(cw[4 * v], cw[4 * v + 1], cw[4 * v + 2], cw[4 * v + 3]);
                } else if (crow) {
#pragma unroll
                    for (int i = 0; i < HC / 2; ++i) {
                        if (col0 + 2 * i < g.n) crow[2 * i] = (uint16_t)(cw[i] & 0xFFFFu);
                        if (col0 + 2 * i + 1 < g.n) crow[2 * i + 1] = (uint16_t)(cw[i] >> 16);
                    }
                }
            }
        }
    }

    tcgen05_fence_before();
    __syncthreads();
    if (warp == 1) {
        tcgen05_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}
// ===================================================================
// Wider limbs: residues of primes p < 2^31 (32-bit coefficients)
// ===================================================================
// A residue in balanced form s (|s| <= (p-1)/2 < 2^30) is split into four
// balanced 8-bit digits s = d0 + 256 d1 + 65536 d2 + 2^24 d3, each exact in
// bf16.  Then
//     a * b = sum_{i,j} a_i b_j 256^(i+j),
// and seven fp32 TMEM accumulators P_t collect the digit products with
// i + j = t.  At most four products of magnitude <= 2^14 land in one P_t
// per k, so over a k-block of 256 every partial sum stays below 2^24 and is
// exact.  The drain forms x = sum_t (P_t + 2^24) * (256^t mod p), a
// nonnegative integer below 2^59, reduces it with one Barrett step in 64-bit
// integers and removes the constant sum_t 2^24 * (256^t mod p) mod p.
// Tiles are 128 x 64 (7 x 64 = 448 TMEM columns, one buffer: the MMA issuer
// waits for the drain between k-blocks); both operand sets hold 4 digit
// planes, a 4-stage ring of 48 KB stages ([A01 | A23 | B01 | B23]).
constexpr int W_BN = 64;
constexpr int W_KSTEPS_PER_BLOCK = 256 / BK;
constexpr int W_A_BOX = 128 * 128, W_B_BOX = W_BN * 128;
constexpr int W_STAGE_BYTES = 2 * W_A_BOX + 2 * W_B_BOX;
constexpr int W_SMEM_BYTES = STAGES * W_STAGE_BYTES + BAR_BYTES + 1024;
constexpr uint32_t IDESC_W = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(W_BN >> 3) << 17) |
                             ((uint32_t)(BM >> 4) << 24);

struct WArgs {
    int64_t M, N, K;
    uint32_t *C;
    int64_t ldc;
    int sign;
    uint32_t p;
    uint64_t w[7];   // 256^t mod p
    uint64_t mu;     // floor((2^64 - 1) / p)
    uint32_t bias;   // (sum_t 2^24 * w[t]) mod p
    uint32_t *err;
};

__device__ __forceinline__ void mma_w(uint32_t d, uint32_t a, uint32_t b, uint32_t hi, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p, e;\n\t.reg .b32 r;\n\t.reg .b64 x, y;\n\t"
                 "elect.sync r|e, 0xffffffff;\n\t"
                 "setp.ne.b32 p, %4, 0;\n\t"
                 "mov.b64 x, {%1, %3};\n\t"
                 "mov.b64 y, {%2, %3};\n\t"
                 "@e tcgen05.mma.cta_group::1.kind::f16 [%0], x, y, %5, p;\n\t}" ::"r"(d),
                 "r"(a), "r"(b), "r"(hi), "r"(acc), "r"(IDESC_W)
                 : "memory");
}

__global__ void __launch_bounds__(THREADS, 1)
    modgemm32_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const WArgs g)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *tiles = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(tiles + STAGES * W_STAGE_BYTES);
    uint64_t *full = bars;
    uint64_t *empty = bars + STAGES;
    uint64_t *accf = bars + 2 * STAGES;
    uint64_t *acce = accf + 1;
    uint64_t *done = acce + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accf, 1);
        mbar_init(acce, EPI_WARPS);
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tcgen05_fence_before();
    __syncthreads();
    tcgen05_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t num_m = (g.M + BM - 1) / BM, num_n = (g.N + W_BN - 1) / W_BN, num_tiles = num_m * num_n;
    const int ksteps = (int)(((g.K + BK - 1) / BK + 3) & ~int64_t(3));   // whole rounds of the 4-stage ring
    const int kblocks = (ksteps + W_KSTEPS_PER_BLOCK - 1) / W_KSTEPS_PER_BLOCK;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer
            int stage = 0;
            uint32_t phase = 0;
            int issued[STAGES];
            uint32_t issued_parity[STAGES];
            for (int s = 0; s < STAGES; ++s) issued[s] = 0, issued_parity[s] = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < num_tiles && ok; t += gridDim.x) {
                const int ay = (int)((t / num_n) * BM), by = (int)((t % num_n) * W_BN);
                for (int ks = 0; ks < ksteps; ++ks) {
                    if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, g.err)) { ok = false; break; }
                    uint8_t *st = tiles + stage * W_STAGE_BYTES;
                    const int x = ks * 4 * BK;   // chunk ks of a 4-plane row
                    mbar_expect_tx(&full[stage], W_STAGE_BYTES);
                    tma_load_2d(st, &tmA, &full[stage], x, ay);
                    tma_load_2d(st + W_A_BOX, &tmA, &full[stage], x + 2 * BK, ay);
                    tma_load_2d(st + 2 * W_A_BOX, &tmB, &full[stage], x, by);
                    tma_load_2d(st + 2 * W_A_BOX + W_B_BOX, &tmB, &full[stage], x + 2 * BK, by);
                    issued[stage] = 1;
                    issued_parity[stage] = phase;
                    if (++stage == STAGES) stage = 0, phase ^= 1u;
                }
            }
            for (int s = 0; s < STAGES; ++s) {   // no copies left in flight
                if (!issued[s]) continue;
                const uint32_t addr = smem_u32(&full[s]);
                const long long start = clock64();
                while (!mbar_try_wait(addr, issued_parity[s])) {
                    if (clock64() - start > WAIT_LIMIT_CYCLES) {
                        dev_fail(g.err, DEV_ERR_TIMEOUT);
                        break;
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (whole warp, elected lane issues)
        uint32_t phase = 0, kbc = 0;
        bool ok = true;
        const uint64_t d0 = make_sdesc(smem_u32(tiles));
        const uint32_t dhi = (uint32_t)(d0 >> 32), lo0 = (uint32_t)d0;
        constexpr uint32_t SB = W_STAGE_BYTES >> 4, AB = W_A_BOX >> 4, BB = W_B_BOX >> 4;
        for (int64_t t = blockIdx.x; t < num_tiles && ok; t += gridDim.x) {
            for (int kb = 0; kb < kblocks && ok; ++kb, ++kbc) {
                if (!mbar_wait_warp(acce, (kbc & 1u) ^ 1u, abort_flag, g.err)) { ok = false; break; }
                tcgen05_fence_after();
                const int ks_beg = kb * W_KSTEPS_PER_BLOCK, ks_end = min(ksteps, ks_beg + W_KSTEPS_PER_BLOCK);
                bool first = true;
                for (int ks = ks_beg; ks < ks_end && ok; ks += STAGES) {
#pragma unroll
                    for (int st = 0; st < STAGES; ++st) {
                        if (!mbar_wait_warp(&full[st], phase, abort_flag, g.err)) { ok = false; break; }
                        const uint32_t a = lo0 + st * SB, b = a + 2 * AB;
#pragma unroll
                        for (int h = 0; h < 2; ++h) {   // the two 16-wide halves of the chunk
                            bool seen[7] = {false, false, false, false, false, false, false};
#pragma unroll
                            for (int i = 0; i < 4; ++i)
#pragma unroll
                                for (int j = 0; j < 4; ++j) {
                                    // plane q of a set: box q / 2, byte offset 64 (q % 2) + 32 h
                                    const uint32_t ad = a + (i >> 1) * AB + (i & 1) * 4 + 2 * h;
                                    const uint32_t bd = b + (j >> 1) * BB + (j & 1) * 4 + 2 * h;
                                    const int tt = i + j;
                                    mma_w(tmem + (uint32_t)(tt * W_BN), ad, bd, dhi,
                                          (first && h == 0 && !seen[tt]) ? 0u : 1u);
                                    seen[tt] = true;
                                }
                        }
                        first = false;
                        commit_elected<false, true>(&empty[st]);
                    }
                    phase ^= 1u;
                }
                if (ok) commit_elected<false, true>(accf);
            }
        }
        commit_elected<false, false>(done);
        const uint32_t addr = smem_u32(done);
        const long long start = clock64();
        while (!__any_sync(0xffffffffu, mbar_try_wait(addr, 0))) {
            if (clock64() - start > WAIT_LIMIT_CYCLES) {
                if (lane == 0) dev_fail(g.err, DEV_ERR_TIMEOUT);
                break;
            }
        }
    } else {
        // ---------------- drain: warps 2..9, lane quarter warp % 4, half of the 64 columns each
        const int quarter = warp & 3, half = (warp - 2) >> 2;
        const int row_in_tile = quarter * 32 + lane;
        const int64_t P = g.p;
        uint32_t kbc = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; t < num_tiles && ok; t += gridDim.x) {
            uint32_t run[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) run[i] = 0;
            for (int kb = 0; kb < kblocks; ++kb, ++kbc) {
                if (!mbar_wait(accf, kbc & 1u, abort_flag, g.err)) { ok = false; break; }
                tcgen05_fence_after();
                const uint32_t tb = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 32);
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    uint64_t v[16];
#pragma unroll
                    for (int e = 0; e < 16; ++e) v[e] = 0;
#pragma unroll
                    for (int tt = 0; tt < 7; ++tt) {
                        float f[16];
                        tmem_ld16(tb + (uint32_t)(tt * W_BN + c * 16), f);
                        tmem_wait_ld();
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            v[e] += (uint64_t)(__float2int_rn(f[e]) + (1 << 24)) * g.w[tt];
                    }
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        // x mod p (Barrett: the quotient estimate is low by at most 2)
                        const uint64_t x = v[e];
                        uint64_t r = x - __umul64hi(x, g.mu) * (uint64_t)P;
                        r -= r >= (uint64_t)P ? (uint64_t)P : 0;
                        r -= r >= (uint64_t)P ? (uint64_t)P : 0;
                        // remove the bias, add the running residue
                        r += (uint64_t)run[c * 16 + e] + (uint64_t)P - g.bias;
                        r -= r >= (uint64_t)P ? (uint64_t)P : 0;
                        r -= r >= (uint64_t)P ? (uint64_t)P : 0;
                        run[c * 16 + e] = (uint32_t)r;
                    }
                }
                tcgen05_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acce);
            }
            if (!ok) break;
            const int64_t row = (t / num_n) * BM + row_in_tile;
            const int64_t col0 = (t % num_n) * W_BN + half * 32;
            if (row < g.M) {
                uint32_t *crow = g.C + row * g.ldc + col0;
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    if (col0 + e >= g.N) break;
                    const uint64_t cur = crow[e], rv = run[e];
                    const uint64_t o = g.sign > 0 ? cur + rv : cur + (uint64_t)P - rv;
                    crow[e] = (uint32_t)(o % (uint64_t)P);
                }
            }
        }
    }
    tcgen05_fence_before();
    __syncthreads();
    tcgen05_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

}  // namespace tc

// ---------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::once_flag g_encode_once;

static int get_encode() {
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    return g_encode ? GBLA_OK : GBLA_E_UNSUPPORTED;
}

static int make_map(CUtensorMap *map, const Planes &pl, int box_rows = tc::BM) {
    GBLA_TRY(get_encode());
    // rows of kp * nplanes interleaved elements; a box is 128 rows x 64
    // elements (128 bytes: one K chunk of two planes)
    cuuint64_t dims[2] = {(cuuint64_t)pl.row_elems(), (cuuint64_t)pl.rows};
    cuuint64_t strides[1] = {(cuuint64_t)pl.row_elems() * 2};
    cuuint32_t box[2] = {2 * tc::BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)pl.ptr, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? GBLA_OK : GBLA_E_CUDA;
}

// ----------------------------------------------- per-launch timing (opt-in)
// While a reduction runs with kernel timing on, every launch of the two
// tensor-core kernels on the calling thread is bracketed by a pair of events
// on its stream (events from a per-thread pool), and the dense product
// counts its tiles' work on the device.
namespace {
struct KernelTimes {
    bool on = false;
    unsigned long long *tc_work = nullptr;   // device counter of the dense product's tile work
    std::vector<cudaEvent_t> pool;
    struct Mark {
        int kind;
        size_t ev;            // index of the start event
        int64_t M, N, K;      // the launch's product shape (-1: not known on the host)
    };
    std::vector<Mark> marks;
    size_t used = 0;
    int dev = -1;
};
thread_local KernelTimes g_kt;

cudaEvent_t kt_event() {
    if (g_kt.used == g_kt.pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_kt.pool.push_back(e);
    }
    return g_kt.pool[g_kt.used++];
}

// kind 0: modgemm_tc_kernel, 1: modgemm_gather_kernel
void kt_start(int kind, cudaStream_t s, int64_t M = -1, int64_t N = -1, int64_t K = -1) {
    if (!g_kt.on) return;
    const size_t i = g_kt.used;
    cudaEvent_t a = kt_event();
    if (a && cudaEventRecord(a, s) == cudaSuccess) g_kt.marks.push_back({kind, i, M, N, K});
}
void kt_stop(cudaStream_t s) {
    if (!g_kt.on || g_kt.marks.empty() || g_kt.marks.back().ev + 1 != g_kt.used) return;
    cudaEvent_t b = kt_event();
    if (b) cudaEventRecord(b, s);
}
}  // namespace

void kernel_times_begin(unsigned long long *tc_work_dev) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (g_kt.dev != dev) {   // events belong to the device that was current when they were made
        for (cudaEvent_t e : g_kt.pool) cudaEventDestroy(e);
        g_kt.pool.clear();
        g_kt.dev = dev;
    }
    g_kt.on = true;
    g_kt.tc_work = tc_work_dev;
    g_kt.marks.clear();
    g_kt.used = 0;
}

// GBLA_LOG=2: also one stderr line per timed launch (kind, product shape, ms).
static bool launch_trace() {
    static const bool v = [] {
        const char *e = getenv("GBLA_LOG");
        return e && atoi(e) >= 2;
    }();
    return v;
}

void kernel_times_end(KernelTimeTotals *t) {
    *t = KernelTimeTotals{};
    if (g_kt.on)
        for (const auto &mk : g_kt.marks) {
            if (mk.ev + 1 >= g_kt.used) continue;
            float ms = 0;
            if (cudaEventElapsedTime(&ms, g_kt.pool[mk.ev], g_kt.pool[mk.ev + 1]) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            t->ms[mk.kind] += ms;
            t->launches[mk.kind] += 1;
            if (launch_trace())
                fprintf(stderr, "gbla-launch %s M=%lld N=%lld K=%lld ms=%.4f\n", mk.kind ? "gather" : "tc",
                        (long long)mk.M, (long long)mk.N, (long long)mk.K, ms);
        }
    g_kt.on = false;
    g_kt.tc_work = nullptr;
    g_kt.marks.clear();
    g_kt.used = 0;
}

// The product kernel's shared-memory limit, set once per process (thread-safe).
static cudaError_t tc_kernel_attrs() {
    static const cudaError_t rc = cudaFuncSetAttribute(tc::modgemm_tc_kernel<false>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES);
    return rc;
}

// Row tiles per raster group (env GBLA_GEMM_GROUP_M overrides, for tuning).
static int gemm_group_m() {
    static const int v = [] {
        const char *e = getenv("GBLA_GEMM_GROUP_M");
        const int x = e ? atoi(e) : 0;
        return (x >= 1 && x <= 256) ? x : (int)tc::GROUP_M_DEFAULT;
    }();
    return v;
}

// Row tiles per raster group of the gathered product (env GBLA_GATHER_GROUP_M
// overrides; 0 = chosen per launch).
static int gather_group_m_env() {
    static const int v = [] {
        const char *e = getenv("GBLA_GATHER_GROUP_M");
        const int x = e ? atoi(e) : 0;
        return (x >= 1 && x <= 1024) ? x : 0;
    }();
    return v;
}

// Per-thread override of the raster group (set by a reduction that the
// autotuner configures; 0 = none).
thread_local int g_gather_group_m_override = 0;

int gather_group_m_default() { return gather_group_m_env() ? gather_group_m_env() : gemm_group_m(); }

int device_sm_count() {
    static const int n = [] {
        int dev = 0, c = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
        return c > 0 ? c : 1;
    }();
    return n;
}

bool tc_supported() {
    static const bool ok = [] {
        int dev = 0, major = 0, minor = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
        return major == 10 && minor == 3;
    }();
    return ok;
}

// Clusters of two CTAs that can be resident at once for the CTA-pair kernel
// (0 if such clusters cannot be launched or the pair kernel is not enabled;
// GBLA_GEMM_PAIR=1 enables it).
static int pair_max_clusters() {
    static const int clusters = [] {
        int n = 0;
        const char *e = getenv("GBLA_GEMM_PAIR");
        if (!e || atoi(e) == 0) return n;
        if (cudaFuncSetAttribute(tc::modgemm_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 tc::PAIR_SMEM_BYTES) != cudaSuccess) {
            cudaGetLastError();
            return n;
        }
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(2 * (unsigned)device_sm_count());
        cfg.blockDim = dim3(tc::THREADS);
        cfg.dynamicSmemBytes = tc::PAIR_SMEM_BYTES;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int c = 0;
        if (cudaOccupancyMaxActiveClusters(&c, tc::modgemm_tc_kernel<true>, &cfg) == cudaSuccess && c > 0) n = c;
        cudaGetLastError();
        return n;
    }();
    return clusters;
}

int modgemm(const Planes &A, int64_t a_row0, int64_t a_k0, const Planes &B, int64_t b_row0, int64_t b_k0,
            uint16_t *C, int64_t ldc, int64_t M, int64_t N, int64_t K, int sign, const ModP &mp, int variant,
            uint32_t *err, cudaStream_t s, GemmCounters *ctr, const int32_t *c_rows, const int32_t *row_lead,
            const int32_t *row_lead_host)
{
    if (M <= 0 || N <= 0 || K <= 0) return GBLA_OK;
    if (variant == GBLA_GEMM_AUTO) variant = (mp.p >= 8 && tc_supported()) ? GBLA_GEMM_TCGEN05 : GBLA_GEMM_SIMT;
    if (ctr) {
        ctr->launches += 1;
        // algorithmic multiply-adds: with known row leads, only the nonzero
        // part of each A row counts
        double ops = (double)M * (double)N * (double)K;
        if (row_lead_host) {
            double kk = 0;
            for (int64_t i = 0; i < M; ++i) {
                const int64_t z = (int64_t)row_lead_host[i] - a_k0;
                kk += (double)(K - (z > 0 ? (z < K ? z : K) : 0));
            }
            ops = kk * (double)N;
        }
        ctr->mod_ops += ops;
        ctr->last_ops = ops;
    }
    if (variant == GBLA_GEMM_FP64 || variant == GBLA_GEMM_U8)
        return modgemm_alt(A, a_row0, a_k0, B, b_row0, b_k0, C, ldc, M, N, K, sign, mp, variant, s, c_rows, row_lead);
    if (variant == GBLA_GEMM_SIMT) {
        dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64));
        modgemm_simt_kernel<<<grid, 256, 0, s>>>(A, a_row0, a_k0, B, b_row0, b_k0, C, ldc, c_rows, M, N, K, sign, mp);
        GBLA_CUDA_TRY(launch_check());
        return GBLA_OK;
    }
    if (variant != GBLA_GEMM_TCGEN05) return GBLA_E_INVAL;
    if (!tc_supported() || mp.p < 8) return GBLA_E_UNSUPPORTED;
    if (A.nplanes != 2 || B.nplanes != 4) return GBLA_E_INTERNAL;
    if ((a_k0 % tc::BK) || (b_k0 % tc::BK)) return GBLA_E_INTERNAL;
    // Products with more than one row tile and a long K run on CTA pairs.
    const int clusters = (M > tc::BM && K >= 256) ? pair_max_clusters() : 0;
    const bool pair = clusters > 0;
    CUtensorMap ma, mb;
    GBLA_TRY(make_map(&ma, A));
    GBLA_TRY(make_map(&mb, B, pair ? tc::BN / 2 : tc::BM));
    GBLA_CUDA_TRY(tc_kernel_attrs());
    tc::Args g{};
    g.M = M; g.N = N; g.K = K;
    g.probs = nullptr; g.nprob = 0;
    g.group_m = gemm_group_m();
    g.a_row0 = (int32_t)a_row0; g.a_k0 = (int32_t)a_k0;
    g.b_row0 = (int32_t)b_row0; g.b_k0 = (int32_t)b_k0;
    g.C = C; g.ldc = ldc; g.c_rows = c_rows; g.row_lead = row_lead; g.sign = sign;
    g.p = mp.p; g.pinv = mp.pinv;
    g.err = err;
    g.withhold_loads = 0;
    if (pair) {
        const int64_t tiles = ((M + 2 * tc::BM - 1) / (2 * tc::BM)) * ((N + tc::BN - 1) / tc::BN);
        const int nc = (int)(tiles < clusters ? tiles : clusters);
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(2 * (unsigned)nc);
        cfg.blockDim = dim3(tc::THREADS);
        cfg.dynamicSmemBytes = tc::PAIR_SMEM_BYTES;
        cfg.stream = s;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        g.work = g_kt.tc_work;
        kt_start(0, s, M, N, K);
        GBLA_CUDA_TRY(cudaLaunchKernelEx(&cfg, tc::modgemm_tc_kernel<true>, ma, mb, g));
        kt_stop(s);
        ++g_pair_launches;
    } else {
        const int64_t tiles = ((M + tc::BM - 1) / tc::BM) * ((N + tc::BN - 1) / tc::BN);
        const int grid = (int)(tiles < device_sm_count() ? tiles : device_sm_count());
        g.work = g_kt.tc_work;
        kt_start(0, s, M, N, K);
        tc::modgemm_tc_kernel<false><<<grid, tc::THREADS, tc::SMEM_BYTES, s>>>(ma, mb, g);
        kt_stop(s);
    }
    GBLA_CUDA_TRY(launch_check());
    if (ctr) ctr->tc_launches += 1;
    return GBLA_OK;
}

// Planes-out product: Out[row, out_col0 + n] <- digits of (A * B)[row, n] mod p
// for rows < M, n < round_up(N, 128); C is not involved.  Tensor-core variant
// only; Out is an A-operand (2-plane) set whose columns out_col0 .. out_col0 +
// round_up(N, 128) lie inside its padded width.
int modgemm_to_planes(const Planes &A, int64_t a_row0, const Planes &B, int64_t b_row0, const Planes &Out,
                      int64_t out_col0, int64_t M, int64_t N, int64_t K, const ModP &mp, uint32_t *err,
                      cudaStream_t s, GemmCounters *ctr, int64_t out_row0)
{
    if (M <= 0 || N <= 0 || K <= 0) return GBLA_OK;
    if (!tc_supported() || mp.p < 8) return GBLA_E_UNSUPPORTED;
    if ((A.nplanes != 2 && A.nplanes != 4) || B.nplanes != 4 || Out.nplanes != 2) return GBLA_E_INTERNAL;
    if ((out_col0 % 8) || out_col0 + round_up(N, tc::BN) > Out.kp || out_row0 < 0 || out_row0 + M > Out.rows)
        return GBLA_E_INTERNAL;
    if (ctr) ctr->launches += 1;   // the caller counts the algorithmic work
    CUtensorMap ma, mb;
    GBLA_TRY(make_map(&ma, A));
    GBLA_TRY(make_map(&mb, B));
    GBLA_CUDA_TRY(tc_kernel_attrs());
    tc::Args g{};
    g.M = M; g.N = N; g.K = K;
    g.group_m = gemm_group_m();
    g.a_row0 = (int32_t)a_row0; g.a_k0 = 0;
    g.b_row0 = (int32_t)b_row0; g.b_k0 = 0;
    g.sign = 1;
    g.p = mp.p; g.pinv = mp.pinv;
    g.err = err;
    g.xout = Out;
    g.xout_col0 = out_col0;
    g.xout_row0 = out_row0;
    g.a_pitch = 32 * A.nplanes;
    g.work = g_kt.tc_work;
    const int64_t tiles = ((M + tc::BM - 1) / tc::BM) * ((N + tc::BN - 1) / tc::BN);
    const int grid = (int)(tiles < device_sm_count() ? tiles : device_sm_count());
    kt_start(0, s, M, N, K);
    tc::modgemm_tc_kernel<false><<<grid, tc::THREADS, tc::SMEM_BYTES, s>>>(ma, mb, g);
    kt_stop(s);
    GBLA_CUDA_TRY(launch_check());
    if (ctr) ctr->tc_launches += 1;
    return GBLA_OK;
}

// Gathered product (see tc::modgemm_gather_kernel).
int modgemm_gather(const Compact &S, int64_t nt0, const Planes &XT, int64_t xt_rows, uint16_t *C, int64_t ldc,
                   int64_t M, int64_t N, int sign, const int32_t *row_lead, const ModP &mp, uint32_t *err,
                   cudaStream_t s, GemmCounters *ctr, unsigned long long *exec)
{
    if (M <= 0 || N <= 0 || S.total <= 0) return GBLA_OK;
    if (!tc_supported() || mp.p < 8) return GBLA_E_UNSUPPORTED;
    if (XT.nplanes != 2 || XT.kp % 128 || round_up(M, 128) > XT.kp || xt_rows > XT.rows || S.total % 128 ||
        nt0 < 0 || nt0 + (N + 127) / 128 > S.ntiles)
        return GBLA_E_INTERNAL;
    if (ctr) ctr->launches += 1;
    GBLA_TRY(get_encode());
    CUtensorMap mb;
    cuuint64_t dims[2] = {2 * tc::BK, (cuuint64_t)(S.total / tc::BK) * 128};
    cuuint64_t strides[1] = {2 * tc::BK * 2};
    cuuint32_t box[2] = {2 * tc::BK, 128};
    cuuint32_t estr[2] = {1, 1};
    if (g_encode(&mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)S.planes, dims, strides, box, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return GBLA_E_CUDA;
    static std::once_flag attr_once;
    static cudaError_t attr_rc = cudaSuccess;
    static int attr_threads = 0;
    std::call_once(attr_once, [] {
        attr_rc = cudaFuncSetAttribute(tc::modgemm_gather_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       tc::G_SMEM_BYTES);
        cudaFuncAttributes fa;
        if (attr_rc == cudaSuccess && (attr_rc = cudaFuncGetAttributes(&fa, tc::modgemm_gather_kernel)) == cudaSuccess)
            attr_threads = fa.maxThreadsPerBlock;
    });
    GBLA_CUDA_TRY(attr_rc);
    if (attr_threads < tc::G_THREADS) return GBLA_E_INTERNAL;   // the block would not fit the SM's registers
    tc::GArgs g{};
    g.M = M; g.N = N; g.nt0 = nt0;
    g.kidx = S.kidx; g.koff = S.koff;
    g.xt = XT.ptr; g.xt_row_elems = XT.row_elems(); g.xt_rows = xt_rows;
    g.C = C; g.ldc = ldc; g.sign = sign;
    g.p = mp.p; g.pinv = mp.pinv;
    g.err = err;
    g.group_m = g_gather_group_m_override ? g_gather_group_m_override
                                          : (gather_group_m_env() ? gather_group_m_env() : gemm_group_m());
    const int64_t num_m = (M + tc::BM - 1) / tc::BM, num_n = (N + tc::BN - 1) / tc::BN;
    int32_t *kstart = nullptr;
    if (row_lead || exec) {
        // first list entry of every (row tile, column tile) at or after the
        // row tile's first lead
        GBLA_TRY(dalloc_t(&kstart, (size_t)(num_m * num_n), s));
        tc::gather_starts_kernel<<<(unsigned)((num_m * num_n + 255) / 256), 256, 0, s>>>(
            num_m, num_n, nt0, S.koff, S.kidx, row_lead, kstart, exec);
        if (launch_check() != cudaSuccess) {
            dfree(kstart, s);
            return GBLA_E_CUDA;
        }
    }
    g.kstart = kstart;
    const int64_t tiles = num_m * num_n;
    const int grid = (int)(tiles < device_sm_count() ? tiles : device_sm_count());
    kt_start(1, s, M, N, -1);
    tc::modgemm_gather_kernel<<<grid, tc::G_THREADS, tc::G_SMEM_BYTES, s>>>(mb, g);
    kt_stop(s);
    const cudaError_t e = cudaGetLastError();
    ++g_launches;
    dfree(kstart, s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e, "modgemm_gather_kernel", __FILE__, __LINE__);
        return GBLA_E_CUDA;
    }
    if (ctr) ctr->tc_launches += 1;
    return GBLA_OK;
}

// ===================================================================
// Wider limbs: host side of the product for primes p < 2^31
// ===================================================================
// dst(h, r, k) <- digit h of the balanced residue src[r][k] (transposed: of
// src[k][r]) for r < R, k < Kc; zero elsewhere in the padded rectangle.
__global__ void __launch_bounds__(256) to_planes32_kernel(Planes dst, int64_t R, int64_t Kc,
                                                          const uint32_t *__restrict__ src, int64_t lds,
                                                          int transposed, uint32_t p)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= dst.rows * dst.kp) return;
    const int64_t r = idx / dst.kp, k = idx % dst.kp;
    uint32_t a = 0;
    if (r < R && k < Kc) a = transposed ? src[k * lds + r] : src[r * lds + k];
    int64_t x = a > (p >> 1) ? (int64_t)a - (int64_t)p : (int64_t)a;
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const int d = h < 3 ? (int)((((x % 256) + 256 + 128) % 256) - 128) : (int)x;
        *dst.at(h, r, k) = i2bf(d);
        x = (x - d) / 256;
    }
}

int modmatmul32(int64_t M, int64_t N, int64_t K, const uint32_t *A, int64_t lda, const uint32_t *B, int64_t ldb,
                uint32_t *C, int64_t ldc, uint32_t p, int sign, cudaStream_t s)
{
    if (!tc_supported()) return GBLA_E_UNSUPPORTED;
    Planes Ap{}, Bp{};
    uint32_t *err = nullptr;
    int rc = dalloc_t(&err, 4, s);
    if (rc == GBLA_OK) rc = planes_alloc(&Ap, M, K, 4, s);
    if (rc == GBLA_OK) rc = planes_alloc(&Bp, N, K, 4, s);
    if (rc == GBLA_OK && cudaMemsetAsync(err, 0, 4, s) != cudaSuccess) rc = GBLA_E_CUDA;
    if (rc == GBLA_OK) {
        to_planes32_kernel<<<(unsigned)((Ap.rows * Ap.kp + 255) / 256), 256, 0, s>>>(Ap, M, K, A, lda, 0, p);
        if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
    }
    if (rc == GBLA_OK) {
        to_planes32_kernel<<<(unsigned)((Bp.rows * Bp.kp + 255) / 256), 256, 0, s>>>(Bp, N, K, B, ldb, 1, p);
        if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
    }
    CUtensorMap ma, mb;
    if (rc == GBLA_OK) rc = make_map(&ma, Ap, tc::BM);
    if (rc == GBLA_OK) rc = make_map(&mb, Bp, tc::W_BN);
    static const cudaError_t attr = cudaFuncSetAttribute(tc::modgemm32_kernel,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize, tc::W_SMEM_BYTES);
    if (rc == GBLA_OK && attr != cudaSuccess) rc = GBLA_E_CUDA;
    if (rc == GBLA_OK) {
        tc::WArgs g{};
        g.M = M; g.N = N; g.K = K;
        g.C = C; g.ldc = ldc; g.sign = sign; g.p = p; g.err = err;
        uint64_t w = 1, bias = 0;
        for (int t = 0; t < 7; ++t) {
            g.w[t] = w;
            bias = (bias + ((uint64_t)1 << 24) % p * w) % p;
            w = (w * 256u) % p;
        }
        g.mu = ~0ull / p;
        g.bias = (uint32_t)bias;
        const int64_t tiles = ((M + tc::BM - 1) / tc::BM) * ((N + tc::W_BN - 1) / tc::W_BN);
        const int grid = (int)(tiles < device_sm_count() ? tiles : device_sm_count());
        tc::modgemm32_kernel<<<grid, tc::THREADS, tc::W_SMEM_BYTES, s>>>(ma, mb, g);
        if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == GBLA_OK) rc = GBLA_E_CUDA;
    uint32_t herr = 0;
    if (rc == GBLA_OK && readback(&herr, err, 4, s) == GBLA_OK) rc = map_dev_err(herr);
    planes_free(&Ap, s);
    planes_free(&Bp, s);
    dfree(err, s);
    cudaStreamSynchronize(s);
    return rc;
}

// Fused panel application (see tc::panel_apply_kernel).
int panel_apply(const Planes &A, const PaJob *jobs, int njobs, const int32_t *rowmap, uint16_t *D, int64_t ldd,
                int64_t n, const ModP &mp, uint32_t *err, cudaStream_t s)
{
    if (njobs <= 0 || n <= 0) return GBLA_OK;
    if (!tc_supported() || mp.p < 8) return GBLA_E_UNSUPPORTED;
    if (A.nplanes != 2 || A.kp != 128 || ldd % 8) return GBLA_E_INTERNAL;
    CUtensorMap ma;
    GBLA_TRY(make_map(&ma, A));
    static std::once_flag attr_once;
    static cudaError_t attr_rc = cudaSuccess;
    static int attr_threads = 0;
    std::call_once(attr_once, [] {
        attr_rc = cudaFuncSetAttribute(tc::panel_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       tc::PA_SMEM_BYTES);
        cudaFuncAttributes fa;
        if (attr_rc == cudaSuccess && (attr_rc = cudaFuncGetAttributes(&fa, tc::panel_apply_kernel)) == cudaSuccess)
            attr_threads = fa.maxThreadsPerBlock;
    });
    GBLA_CUDA_TRY(attr_rc);
    if (attr_threads < tc::PA_THREADS) return GBLA_E_INTERNAL;   // the block would not fit the SM's registers
    tc::PaArgs g{};
    g.jobs = jobs; g.njobs = njobs; g.rowmap = rowmap;
    g.D = D; g.ldd = ldd; g.n = n;
    g.p = mp.p; g.pinv = mp.pinv;
    g.err = err;
    tc::panel_apply_kernel<<<device_sm_count(), tc::PA_THREADS, tc::PA_SMEM_BYTES, s>>>(ma, g);
    GBLA_CUDA_TRY(launch_check());
    return GBLA_OK;
}

// Grouped product, SIMT variant: one launch of the reference kernel per
// problem (the problem table is read back; used in tests and for p < 8).
static int modgemm_grouped_simt(const Planes &A, const Planes &B, const GroupProb *probs, int nprob, int64_t K,
                                uint16_t *C, int64_t ldc, int sign, const ModP &mp, cudaStream_t s)
{
    std::vector<GroupProb> h((size_t)nprob + 1);
    GBLA_TRY(readback(h.data(), probs, sizeof(GroupProb) * h.size(), s));
    for (int i = 0; i < nprob; ++i) {
        const GroupProb &P = h[(size_t)i];
        if (P.M <= 0 || P.N <= 0) continue;
        dim3 grid((unsigned)((P.N + 63) / 64), (unsigned)((P.M + 63) / 64));
        modgemm_simt_kernel<<<grid, 256, 0, s>>>(A, P.a_row0, 0, B, P.b_row0, 0, C + P.c_col0, ldc, P.c_rows, P.M, P.N,
                                                 K, sign, mp);
        GBLA_CUDA_TRY(launch_check());
    }
    return GBLA_OK;
}

// Grouped product: the problems (device array of nprob + 1 entries, tile
// offsets filled, entry [nprob].tile_off = total tiles) share the A and B
// plane sets and K; C is one matrix with leading dimension ldc.
int modgemm_grouped(const Planes &A, const Planes &B, const GroupProb *probs, int nprob, int64_t K, uint16_t *C,
                    int64_t ldc, int sign, const ModP &mp, int variant, uint32_t *err, cudaStream_t s,
                    GemmCounters *ctr)
{
    if (nprob <= 0 || K <= 0) return GBLA_OK;
    if (variant == GBLA_GEMM_AUTO) variant = (mp.p >= 8 && tc_supported()) ? GBLA_GEMM_TCGEN05 : GBLA_GEMM_SIMT;
    if (ctr) ctr->launches += 1;
    if (variant == GBLA_GEMM_SIMT) return modgemm_grouped_simt(A, B, probs, nprob, K, C, ldc, sign, mp, s);
    if (!tc_supported() || mp.p < 8) return GBLA_E_UNSUPPORTED;
    CUtensorMap ma, mb;
    GBLA_TRY(make_map(&ma, A));
    GBLA_TRY(make_map(&mb, B));
    GBLA_CUDA_TRY(tc_kernel_attrs());
    tc::Args g{};
    g.M = 0; g.N = 0; g.K = K;
    g.probs = probs; g.nprob = nprob;
    g.group_m = gemm_group_m();
    g.C = C; g.ldc = ldc; g.sign = sign;
    g.p = mp.p; g.pinv = mp.pinv;
    g.err = err;
    g.work = g_kt.tc_work;
    kt_start(0, s);
    tc::modgemm_tc_kernel<false><<<device_sm_count(), tc::THREADS, tc::SMEM_BYTES, s>>>(ma, mb, g);
    kt_stop(s);
    GBLA_CUDA_TRY(launch_check());
    if (ctr) ctr->tc_launches += 1;
    return GBLA_OK;
}

// Test hook for the failure path of the bounded waits: one 128 x 128 x 64
// tile whose loads are withheld.  The MMA issuer's wait for the first stage
// expires after WAIT_LIMIT_CYCLES, the other roles see the abort flag, and the
// kernel frees TMEM and returns with DEV_ERR_TIMEOUT set.
int modgemm_withheld_loads(uint32_t *err, cudaStream_t s)
{
    if (!tc_supported()) return GBLA_E_UNSUPPORTED;
    Planes A{}, B{};
    int rc = planes_alloc(&A, 128, 64, 2, s);
    if (rc == GBLA_OK) rc = planes_alloc(&B, 128, 64, 4, s);
    CUtensorMap ma, mb;
    if (rc == GBLA_OK) rc = make_map(&ma, A);
    if (rc == GBLA_OK) rc = make_map(&mb, B);
    if (rc == GBLA_OK) {
        if (tc_kernel_attrs() != cudaSuccess) rc = GBLA_E_CUDA;
    }
    uint16_t *C = nullptr;
    if (rc == GBLA_OK) rc = dalloc_t(&C, 128 * 128, s);
    if (rc == GBLA_OK) {
        tc::Args g{};
        g.group_m = 1;
        g.M = 128; g.N = 128; g.K = 64;
            g.C = C; g.ldc = 128; g.sign = 1;
        const ModP mp = make_modp(65521);
        g.p = mp.p; g.pinv = mp.pinv;
        g.err = err;
        g.withhold_loads = 1;
        tc::modgemm_tc_kernel<false><<<1, tc::THREADS, tc::SMEM_BYTES, s>>>(ma, mb, g);
        if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
    }
    dfree(C, s);
    planes_free(&A, s);
    planes_free(&B, s);
    return rc;
}

}  // namespace gbla
