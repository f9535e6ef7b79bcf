// solve.cu -- the sparse reduction C <- C*A^-1 (new order of operations,
// Alg. 2 and its four-step implementation, GBLA paper Sec. 4.2), the
// triangular solve A^-1*B of the second FL pass (Sec. 4.1 step 2 and the
// reduced-echelon remark after step 5), and the echelonisation of the Schur
// complement D' (Sec. 4.1 step 4, Alg. 3 / Sec. 5.1).
//
// Triangular solves are blocked by columns of A.  A diagonal block of at
// most LEAF columns is solved by a sparse kernel that follows Alg. 1: one
// warp owns a pair of C rows (two dense accumulator rows in shared memory)
// and walks the pivots two at a time, applying the 2-multiline vector of A's
// rows (j, j+1) to both accumulator rows with the four multipliers
// lambda_{1,1..2,2} in one pass.  Accumulators are uint64 with delayed
// reduction: a value is reduced mod p only when it becomes a multiplier.
// Off-diagonal blocks are applied with the exact tensor-core product
// (modgemm.cu), recursively halving the column range so the products are
// large.
#include "common.cuh"
#include "internal.cuh"
#include "solve.cuh"

#include <algorithm>
#include <vector>

namespace gbla {

constexpr int LEAF = LEAF_COLS;
constexpr int LEAF_WARPS = 8;
// Shared memory of a leaf CTA: the block's multiline entries (at most 127 per
// pair inside a block of 128 columns) as (column - j0, value) plus per-pair
// offsets, then the warps' accumulator rows.
constexpr int LEAF_CAP = (LEAF / 2) * (LEAF - 1);
constexpr int LEAF_SMEM_TAB = LEAF_CAP * 5 + (LEAF / 2 + 1) * 4;
constexpr int LEAF_SMEM_UPPER = ((LEAF_SMEM_TAB + 15) & ~15) + LEAF_WARPS * 2 * LEAF * 8;
constexpr int LEAF_SMEM_LOWER = ((LEAF_SMEM_TAB + 15) & ~15) + LEAF_WARPS * 2 * LEAF * 4;

struct LeafTab {
    uint32_t *val;   // [LEAF_CAP]
    uint8_t *pos;    // [LEAF_CAP] column - j0
    int *off;        // [LEAF/2 + 1]
};

// Copy the multiline entries of the block's pivot pairs that fall inside the
// block into shared memory (all warps of the CTA read them many times).
__device__ __forceinline__ LeafTab load_leaf_tab(uint8_t *smem, int64_t j0, int W, const int64_t *__restrict__ mlptr,
                                                 const int32_t *__restrict__ mlpos,
                                                 const uint32_t *__restrict__ mlval,
                                                 const int32_t *__restrict__ inblk)
{
    LeafTab T;
    T.val = reinterpret_cast<uint32_t *>(smem);
    T.pos = smem + LEAF_CAP * 4;
    T.off = reinterpret_cast<int *>(smem + LEAF_CAP * 5);
    const int npairs = (W + 1) / 2;
    const int64_t q0 = j0 / 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (warp == 0) {
        // exclusive prefix of the in-block counts, two pairs per lane
        const int a = (2 * lane < npairs) ? inblk[q0 + 2 * lane] : 0;
        const int b = (2 * lane + 1 < npairs) ? inblk[q0 + 2 * lane + 1] : 0;
        int incl = a + b;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += t;
        }
        const int excl = incl - a - b;
        if (2 * lane < npairs) T.off[2 * lane] = excl;
        if (2 * lane + 1 < npairs) T.off[2 * lane + 1] = excl + a;
        if (lane == 31) T.off[npairs] = incl;
    }
    __syncthreads();
    for (int q = warp; q < npairs; q += LEAF_WARPS) {
        const int64_t e0 = mlptr[q0 + q];
        const int cnt = T.off[q + 1] - T.off[q];
        for (int i = lane; i < cnt; i += 32) {
            T.val[T.off[q] + i] = mlval[e0 + i];
            T.pos[T.off[q] + i] = (uint8_t)(mlpos[e0 + i] - j0);
        }
    }
    __syncthreads();
    return T;
}

// ------------------------------------------------------------ upper leaf
// X_J * A_JJ = C_J for the column block J = [j0, j0 + W), rows [0, mrows),
// where C_J already holds C_J - X_{<J} * A_{<J,J}.  X_J overwrites C_J
// (uint16) and is written to the A-operand digit planes Xp.
__global__ void __launch_bounds__(256) trsm_upper_leaf_kernel(int64_t mrows, int64_t j0, int W,
                                                              const int64_t *__restrict__ mlptr,
                                                              const int32_t *__restrict__ mlpos,
                                                              const uint32_t *__restrict__ mlval,
                                                              const int32_t *__restrict__ inblk, uint16_t *C16,
                                                              int64_t ldc, Planes Xp, ModP mp)
{
    extern __shared__ __align__(16) uint8_t leaf_smem[];
    const LeafTab T = load_leaf_tab(leaf_smem, j0, W, mlptr, mlpos, mlval, inblk);
    unsigned long long(*acc_s)[2][LEAF] =
        reinterpret_cast<unsigned long long(*)[2][LEAF]>(leaf_smem + ((LEAF_SMEM_TAB + 15) & ~15));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t pair = (int64_t)blockIdx.x * LEAF_WARPS + warp;
    const int64_t r1 = 2 * pair, r2 = 2 * pair + 1;
    if (r1 >= mrows) return;
    const bool has2 = r2 < mrows;
    unsigned long long(*acc)[LEAF] = acc_s[warp];
    for (int c = lane; c < LEAF; c += 32) {
        acc[0][c] = (c < W) ? C16[r1 * ldc + j0 + c] : 0;
        acc[1][c] = (c < W && has2) ? C16[r2 * ldc + j0 + c] : 0;
    }
    __syncwarp();
    const uint64_t P = mp.p;
    for (int jl = 0; jl < W; jl += 2) {
        const int e0 = T.off[jl >> 1], e1 = T.off[(jl >> 1) + 1];
        const bool has_b = jl + 1 < W;
        const bool coupling = e0 < e1 && T.pos[e0] == jl + 1;
        const uint32_t a01 = coupling ? (T.val[e0] & 0xFFFFu) : 0u;
        // multipliers: lambda for pivot j (x?a) and pivot j+1 (x?b), both C rows
        const uint32_t x1a = mod40(acc[0][jl], mp), x2a = mod40(acc[1][jl], mp);
        uint32_t x1b = 0, x2b = 0;
        if (has_b) {
            x1b = mod40(acc[0][jl + 1] + (P - x1a) * a01, mp);
            x2b = mod40(acc[1][jl + 1] + (P - x2a) * a01, mp);
        }
        __syncwarp();
        if (lane == 0) {
            acc[0][jl] = x1a;
            acc[1][jl] = x2a;
            if (has_b) {
                acc[0][jl + 1] = x1b;
                acc[1][jl + 1] = x2b;
            }
        }
        // Alg. 1: both accumulator rows minus the multiline of A rows (j, j+1)
        const uint64_t n1a = P - x1a, n1b = P - x1b, n2a = P - x2a, n2b = P - x2b;
        for (int e = e0 + (coupling ? 1 : 0) + lane; e < e1; e += 32) {
            const int kl = T.pos[e];
            const uint32_t v = T.val[e];
            const uint64_t v1 = v & 0xFFFFu, v2 = v >> 16;
            acc[0][kl] += n1a * v1 + n1b * v2;
            acc[1][kl] += n2a * v1 + n2b * v2;
        }
        __syncwarp();
    }
    // write back X_J
    const uint32_t p = mp.p;
    for (int c = lane; c < W; c += 32) {
        const uint32_t x1 = (uint32_t)acc[0][c];
        C16[r1 * ldc + j0 + c] = (uint16_t)x1;
        int hi, lo;
        digits(x1, p, hi, lo);
        size_t off = (size_t)r1 * Xp.kp + (size_t)(j0 + c);
        Xp.plane(0)[off] = i2bf(hi);
        Xp.plane(1)[off] = i2bf(lo);
        if (has2) {
            const uint32_t x2 = (uint32_t)acc[1][c];
            C16[r2 * ldc + j0 + c] = (uint16_t)x2;
            digits(x2, p, hi, lo);
            off = (size_t)r2 * Xp.kp + (size_t)(j0 + c);
            Xp.plane(0)[off] = i2bf(hi);
            Xp.plane(1)[off] = i2bf(lo);
        }
    }
}

// Rows whose lead is >= bound (a prefix count, leads ascending).
static int64_t rows_before(const TrsmUpper &T, int64_t bound)
{
    if (!T.lead_host) return T.mrows;
    const auto &L = *T.lead_host;
    return std::lower_bound(L.begin(), L.end(), (int32_t)bound) - L.begin();
}

static int trsm_upper_rec(const TrsmUpper &T, int64_t lo, int64_t hi)
{
    if (hi - lo <= LEAF) {
        // rows leading at or after hi have a zero block here (C and X alike)
        const int64_t rows = rows_before(T, hi);
        const int64_t pairs = (rows + 1) / 2;
        if (pairs == 0) return GBLA_OK;
        trsm_upper_leaf_kernel<<<(unsigned)((pairs + LEAF_WARPS - 1) / LEAF_WARPS), 32 * LEAF_WARPS,
                                 LEAF_SMEM_UPPER, T.s>>>(rows, lo, (int)(hi - lo), T.ml->ptr, T.ml->pos, T.ml->val,
                                                         T.ml->inblk, T.C16, T.ldc, *T.Xp, *T.mp);
        GBLA_CUDA_TRY(launch_check());
        return GBLA_OK;
    }
    const int64_t mid = lo + round_up((hi - lo) / 2, LEAF);
    GBLA_TRY(trsm_upper_rec(T, lo, mid));
    // C[:, mid:hi] -= X[:, lo:mid] * A[lo:mid, mid:hi]   (A^T planes: row = column of A);
    // only rows leading before mid have X[:, lo:mid] != 0.
    const int64_t rows = rows_before(T, mid);
    if (rows > 0)
        GBLA_TRY(modgemm(*T.Xp, 0, lo, *T.At, mid, lo, T.C16 + mid, T.ldc, rows, hi - mid, mid - lo, -1, *T.mp,
                         T.variant, T.err, T.s, T.ctr, nullptr, T.lead_dev,
                         T.lead_host ? T.lead_host->data() : nullptr));
    return trsm_upper_rec(T, mid, hi);
}

// ------------------------------------------------------------ lower leaf
// X'_J * A'_JJ = C'_J with A' = A^T (lower unit triangular): for j descending,
// x'_j = c'_j - sum_{k > j} A[j][k] x'_k.  One warp per pair of C' rows; each
// pivot pair (j, j+1) contributes two dot products with its multiline.
__global__ void __launch_bounds__(256) trsm_lower_leaf_kernel(int64_t mrows, int64_t j0, int W,
                                                              const int64_t *__restrict__ mlptr,
                                                              const int32_t *__restrict__ mlpos,
                                                              const uint32_t *__restrict__ mlval,
                                                              const int32_t *__restrict__ inblk, uint16_t *C16,
                                                              int64_t ldc, Planes Xp, ModP mp)
{
    extern __shared__ __align__(16) uint8_t leaf_smem[];
    const LeafTab T = load_leaf_tab(leaf_smem, j0, W, mlptr, mlpos, mlval, inblk);
    uint32_t(*xs_s)[2][LEAF] = reinterpret_cast<uint32_t(*)[2][LEAF]>(leaf_smem + ((LEAF_SMEM_TAB + 15) & ~15));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t pair = (int64_t)blockIdx.x * LEAF_WARPS + warp;
    const int64_t r1 = 2 * pair, r2 = 2 * pair + 1;
    if (r1 >= mrows) return;
    const bool has2 = r2 < mrows;
    uint32_t(*xs)[LEAF] = xs_s[warp];
    for (int c = lane; c < LEAF; c += 32) {
        xs[0][c] = (c < W) ? C16[r1 * ldc + j0 + c] : 0;
        xs[1][c] = (c < W && has2) ? C16[r2 * ldc + j0 + c] : 0;
    }
    __syncwarp();
    const uint64_t P = mp.p;
    const int start = ((W - 1) & ~1);   // local index of the last pair's first column
    for (int jl = start; jl >= 0; jl -= 2) {
        const int e0 = T.off[jl >> 1], e1 = T.off[(jl >> 1) + 1];
        const bool has_b = jl + 1 < W;
        const bool coupling = e0 < e1 && T.pos[e0] == jl + 1;
        const uint32_t a01 = coupling ? (T.val[e0] & 0xFFFFu) : 0u;
        unsigned long long d1r1 = 0, d2r1 = 0, d1r2 = 0, d2r2 = 0;  // d1: A row j, d2: A row j+1
        for (int e = e0 + (coupling ? 1 : 0) + lane; e < e1; e += 32) {
            const int kl = T.pos[e];
            const uint32_t v = T.val[e];
            const uint64_t v1 = v & 0xFFFFu, v2 = v >> 16;
            const uint64_t y1 = xs[0][kl], y2 = xs[1][kl];
            d1r1 += v1 * y1;
            d2r1 += v2 * y1;
            d1r2 += v1 * y2;
            d2r2 += v2 * y2;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            d1r1 += __shfl_xor_sync(0xFFFFFFFFu, d1r1, o);
            d2r1 += __shfl_xor_sync(0xFFFFFFFFu, d2r1, o);
            d1r2 += __shfl_xor_sync(0xFFFFFFFFu, d1r2, o);
            d2r2 += __shfl_xor_sync(0xFFFFFFFFu, d2r2, o);
        }
        if (lane == 0) {
            const uint32_t s2r1 = mod40(d2r1, mp), s2r2 = mod40(d2r2, mp);
            uint32_t xb1 = 0, xb2 = 0;
            if (has_b) {
                xb1 = mod40((uint64_t)xs[0][jl + 1] + P - s2r1, mp);
                xb2 = mod40((uint64_t)xs[1][jl + 1] + P - s2r2, mp);
                xs[0][jl + 1] = xb1;
                xs[1][jl + 1] = xb2;
            }
            const uint64_t t1 = (uint64_t)mod40(d1r1, mp) + (uint64_t)a01 * xb1;
            const uint64_t t2 = (uint64_t)mod40(d1r2, mp) + (uint64_t)a01 * xb2;
            xs[0][jl] = mod40((uint64_t)xs[0][jl] + P * P - mod40(t1, mp), mp);
            xs[1][jl] = mod40((uint64_t)xs[1][jl] + P * P - mod40(t2, mp), mp);
        }
        __syncwarp();
    }
    const uint32_t p = mp.p;
    for (int c = lane; c < W; c += 32) {
        const uint32_t x1 = xs[0][c];
        C16[r1 * ldc + j0 + c] = (uint16_t)x1;
        int hi, lo;
        digits(x1, p, hi, lo);
        size_t off = (size_t)r1 * Xp.kp + (size_t)(j0 + c);
        Xp.plane(0)[off] = i2bf(hi);
        Xp.plane(1)[off] = i2bf(lo);
        if (has2) {
            const uint32_t x2 = xs[1][c];
            C16[r2 * ldc + j0 + c] = (uint16_t)x2;
            digits(x2, p, hi, lo);
            off = (size_t)r2 * Xp.kp + (size_t)(j0 + c);
            Xp.plane(0)[off] = i2bf(hi);
            Xp.plane(1)[off] = i2bf(lo);
        }
    }
}

static int leaf_attrs()
{
    static bool done = false;
    if (!done) {
        GBLA_CUDA_TRY(cudaFuncSetAttribute(trsm_upper_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           LEAF_SMEM_UPPER));
        GBLA_CUDA_TRY(cudaFuncSetAttribute(trsm_lower_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           LEAF_SMEM_LOWER));
        done = true;
    }
    return GBLA_OK;
}

int trsm_upper(const TrsmUpper &T)
{
    if (T.mrows <= 0 || T.npiv <= 0) return GBLA_OK;
    GBLA_TRY(leaf_attrs());
    return trsm_upper_rec(T, 0, T.npiv);
}

static int trsm_lower_rec(const TrsmLower &T, int64_t lo, int64_t hi)
{
    if (hi - lo <= LEAF) {
        const int64_t pairs = (T.mrows + 1) / 2;
        trsm_lower_leaf_kernel<<<(unsigned)((pairs + LEAF_WARPS - 1) / LEAF_WARPS), 32 * LEAF_WARPS,
                                 LEAF_SMEM_LOWER, T.s>>>(T.mrows, lo, (int)(hi - lo), T.ml->ptr, T.ml->pos, T.ml->val,
                                                         T.ml->inblk, T.C16, T.ldc, *T.Xp, *T.mp);
        GBLA_CUDA_TRY(launch_check());
        return GBLA_OK;
    }
    const int64_t mid = lo + round_up((hi - lo) / 2, LEAF);
    GBLA_TRY(trsm_lower_rec(T, mid, hi));
    // C'[:, lo:mid] -= X'[:, mid:hi] * A'[mid:hi, lo:mid],  A'[k][n] = A[n][k]
    GBLA_TRY(modgemm(*T.Xp, 0, mid, *T.Arow, lo, mid, T.C16 + lo, T.ldc, T.mrows, mid - lo, hi - mid, -1, *T.mp,
                     T.variant, T.err, T.s, T.ctr));
    return trsm_lower_rec(T, lo, mid);
}

int trsm_lower(const TrsmLower &T)
{
    if (T.mrows <= 0 || T.npiv <= 0) return GBLA_OK;
    GBLA_TRY(leaf_attrs());
    return trsm_lower_rec(T, 0, T.npiv);
}

// ================================================================ echelon
// Reduced echelon form of D' (Sec. 4.1 step 4; Alg. 3 and its parallel form
// in Sec. 5.1), in two passes.
//
// Forward pass, column panels of width <= 128.  Rows of D' are kept with
// their current leading column.  The panel starts at the smallest leading
// column among the rows that are not pivots yet; its candidates are the
// non-pivot rows whose leading column falls inside it (the others are zero
// there and are not touched).  One CTA takes the candidates in order; each is
// reduced by the panel basis found so far (reduced echelon form over the
// panel's columns) and, if something is left, becomes a new basis row,
// normalised at its leftmost nonzero (Alg. 3's "normalise, reduce by matching
// heads", restricted to the panel).  Each candidate carries the coefficients
// expressing it in the chosen rows S, so G * D[S, panel] = U with U in
// reduced echelon form at pivot columns pc.  Then, on the tensor cores,
//     D[S, c0:]    <- G * D[S, c0:]
//     D[cand, c0:] <- D[cand, c0:] - D[cand, pc] * D[S, c0:]   (cand outside S)
// and the candidates that did not become pivots get their new leading column.
// The pivot rows end in echelon form with unit pivots and identity blocks
// on each panel's pivot columns.
//
// Backward pass: with R = the pivot rows in pivot-column order and
// T = R[:, P_D] (unit upper triangular), RREF(D') = T^-1 R.  This is a
// left-sided triangular solve done by recursive halving: the off-diagonal
// updates R_top -= R_top[:, P_D(bottom)] * R_bottom are tensor-core
// products, and each diagonal block of <= 128 rows is applied as
// R_J <- R_J - (I - T_JJ^-1) R_J.
constexpr int PANEL = 128;

// First nonzero column >= from of each listed row (or every row), -1 if none.
__global__ void row_leads_kernel(const uint16_t *__restrict__ D, int64_t ldd, int64_t n, int64_t m,
                                 const int32_t *__restrict__ rows, const int32_t *__restrict__ count_dev,
                                 int64_t from, const int32_t *__restrict__ skip, int32_t *__restrict__ lead)
{
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t cnt = count_dev ? *count_dev : m;
    if (w >= cnt) return;
    const int64_t r = rows ? rows[w] : w;
    if (skip && skip[r]) return;
    const uint16_t *row = D + r * ldd;
    int64_t found = -1;
    for (int64_t base = from; base < n && found < 0; base += 32 * 8) {
        int64_t best = INT64_MAX;
        for (int e = 0; e < 8; ++e) {
            const int64_t c = base + (int64_t)e * 32 + lane;
            if (c < n && row[c] != 0) { best = c; break; }
        }
        // minimum over the warp
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int64_t t = __shfl_xor_sync(0xFFFFFFFFu, best, o);
            best = t < best ? t : best;
        }
        if (best != INT64_MAX) found = best;
    }
    if (lane == 0) lead[r] = (int32_t)found;
}

// One CTA: c0 = smallest leading column of a non-pivot row; candidates =
// non-pivot rows with leading column in [c0, c0 + PANEL), in row order.
__global__ void __launch_bounds__(1024) candidates_kernel(int64_t m, const int32_t *__restrict__ lead,
                                                          const int32_t *__restrict__ is_piv_row,
                                                          int32_t *__restrict__ cand, int32_t *__restrict__ info)
{
    __shared__ int smin;
    __shared__ int wsum[32];
    __shared__ int base;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) { smin = INT32_MAX; base = 0; }
    __syncthreads();
    int lmin = INT32_MAX;
    for (int64_t r = tid; r < m; r += blockDim.x) {
        const int l = lead[r];
        if (!is_piv_row[r] && l >= 0 && l < lmin) lmin = l;
    }
    atomicMin(&smin, lmin);
    __syncthreads();
    const int c0 = smin;
    for (int64_t r0 = 0; r0 < m; r0 += blockDim.x) {
        const int64_t r = r0 + tid;
        int f = 0;
        if (r < m && c0 != INT32_MAX) {
            const int l = lead[r];
            f = (!is_piv_row[r] && l >= 0 && l < c0 + PANEL) ? 1 : 0;
        }
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, f);
        if (lane == 0) wsum[wid] = __popc(bal);
        __syncthreads();
        int off = base;
        for (int k = 0; k < wid; ++k) off += wsum[k];
        if (f) cand[off + __popc(bal & ((1u << lane) - 1u))] = (int32_t)r;
        __syncthreads();
        if (tid == 0) {
            int tot = 0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot += wsum[k];
            base += tot;
        }
        __syncthreads();
    }
    if (tid == 0) {
        info[0] = (c0 == INT32_MAX) ? -1 : c0;
        info[1] = base;
    }
}

// Inverses of all residues (0 -> 0), for the panel kernel's table.
__global__ void inverse_table_kernel(uint16_t *__restrict__ tab, ModP mp)
{
    const uint32_t a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < mp.p) tab[a] = (uint16_t)(a ? invmod(a, mp) : 0u);
}

constexpr size_t PANEL_SMEM = (size_t)PANEL * 2 * PANEL * sizeof(uint16_t) + 65536 * sizeof(uint16_t);

__global__ void __launch_bounds__(256) panel_kernel(const uint16_t *__restrict__ D, int64_t ldd,
                                                    const int32_t *__restrict__ info, int64_t n,
                                                    const int32_t *__restrict__ cand,
                                                    const uint16_t *__restrict__ inv_tab,
                                                    int32_t *__restrict__ is_piv_row, int32_t *__restrict__ t_out,
                                                    int32_t *__restrict__ S_out, int32_t *__restrict__ Spos_out,
                                                    int32_t *__restrict__ pc_out, uint16_t *__restrict__ Gm_out,
                                                    int32_t *__restrict__ prow, int32_t *__restrict__ pcol,
                                                    int32_t *__restrict__ rank_dev, ModP mp)
{
    extern __shared__ __align__(16) uint16_t panel_smem[];
    uint16_t(*aug)[2 * PANEL] = reinterpret_cast<uint16_t(*)[2 * PANEL]>(panel_smem);  // [PANEL][256]
    uint16_t *inv_s = panel_smem + PANEL * 2 * PANEL;                                  // [p]
    __shared__ uint32_t cand_v[2 * PANEL];
    __shared__ uint32_t fk[PANEL], coef[PANEL];
    __shared__ int bcol[PANEL], brow[PANEL], S[PANEL], Spos[PANEL], rnk[PANEL];
    __shared__ int wmin[8];
    const int c = threadIdx.x;  // column of the augmented row: [panel | coefficients]
    const int lane = c & 31, warp = c >> 5;
    const int64_t c0 = info[0];
    const int ncand = info[1];
    const int bw = (int)((n - c0) < PANEL ? (n - c0) : PANEL);
    const int64_t rank0 = *rank_dev;
    const uint32_t p = mp.p;
    // inverse table into shared memory (16-byte copies; p <= 65536 entries)
    {
        const int nvec = (int)((p + 7) / 8);
        const uint4 *src = reinterpret_cast<const uint4 *>(inv_tab);
        uint4 *dst = reinterpret_cast<uint4 *>(inv_s);
        for (int i = c; i < nvec; i += 2 * PANEL) dst[i] = src[i];
    }
    if (c < PANEL) brow[c] = -1;     // basis row whose pivot is panel column c
    __syncthreads();
    int t = 0;
    // software pipeline: the next candidate's panel entry is loaded while the
    // current one is processed
    uint32_t vnext = 0;
    if (ncand > 0 && c < bw) vnext = D[(int64_t)cand[0] * ldd + c0 + c];
    for (int ci = 0; ci < ncand && t < bw; ++ci) {
        uint32_t v = vnext;
        if (ci + 1 < ncand && c < bw) vnext = D[(int64_t)cand[ci + 1] * ldd + c0 + c];
        if (c >= PANEL) v = (c - PANEL == t) ? 1u : 0u;
        // the basis is in reduced echelon form, so the multiplier of basis
        // row k is this candidate's entry at that row's pivot column
        if (c < bw && brow[c] >= 0) coef[brow[c]] = p - v;
        if (!__syncthreads_or(c < bw && v != 0)) continue;
        unsigned long long a0 = v, a1 = 0, a2 = 0, a3 = 0;   // four chains
        int k = 0;
        for (; k + 4 <= t; k += 4) {
            a0 += (uint64_t)coef[k] * aug[k][c];
            a1 += (uint64_t)coef[k + 1] * aug[k + 1][c];
            a2 += (uint64_t)coef[k + 2] * aug[k + 2][c];
            a3 += (uint64_t)coef[k + 3] * aug[k + 3][c];
        }
        for (; k < t; ++k) a0 += (uint64_t)coef[k] * aug[k][c];
        const uint32_t nv = mod40(a0 + a1 + a2 + a3, mp);
        // leftmost nonzero of the reduced panel part
        int mine = (c < bw && nv != 0) ? c : (1 << 30);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mine = min(mine, __shfl_xor_sync(0xFFFFFFFFu, mine, o));
        if (lane == 0) wmin[warp] = mine;
        cand_v[c] = nv;
        __syncthreads();
        int cs = wmin[0];
#pragma unroll
        for (int w = 1; w < 8; ++w) cs = min(cs, wmin[w]);
        if (cs >= bw) continue;           // dependent on the rows taken so far
        const uint32_t inv = inv_s[cand_v[cs]];
        if (c < t) fk[c] = aug[c][cs];
        __syncthreads();
        const uint32_t nrm = mulmod(nv, inv, mp);
        for (int kk = 0; kk < t; ++kk) {
            const uint32_t f = fk[kk];
            if (f) {
                const uint32_t sub = mulmod(f, nrm, mp);
                const uint32_t x = aug[kk][c];
                aug[kk][c] = (uint16_t)(x >= sub ? x - sub : x + p - sub);
            }
        }
        aug[t][c] = (uint16_t)nrm;
        if (c == cs) brow[c] = t;
        if (c == 0) {
            bcol[t] = cs;
            S[t] = (int)cand[ci];
            Spos[t] = ci;
        }
        ++t;
        __syncthreads();
    }
    __syncthreads();
    // order the basis rows by pivot column
    if (c < t) {
        int r = 0;
        for (int kk = 0; kk < t; ++kk) r += (bcol[kk] < bcol[c]) ? 1 : 0;
        rnk[c] = r;
    }
    __syncthreads();
    if (c == 0) {
        *t_out = t;
        *rank_dev = (int32_t)(rank0 + t);
    }
    if (c < PANEL) {
        // rows beyond t are sentinels (-1): the products skip them
        S_out[c] = (c < t) ? S[c] : -1;
        Spos_out[c] = (c < t) ? Spos[c] : -1;
        if (c < t) {
            pc_out[rnk[c]] = bcol[c];
            is_piv_row[S[c]] = 1;
        } else {
            pc_out[c] = -1;
        }
    }
    __syncthreads();
    // the pivot with the c-th smallest column lands in physical row S[c]
    if (c < t) {
        prow[rank0 + c] = S[c];
        pcol[rank0 + c] = (int32_t)(c0 + pc_out[c]);
    }
    for (int kk = 0; kk < PANEL; ++kk) {
        // Gm row rnk[kk] = coefficient part of basis row kk minus the identity;
        // rows and columns beyond t are zero
        if (c < PANEL) {
            if (kk < t) {
                uint32_t g = (c < t) ? aug[kk][PANEL + c] : 0u;
                if (c == rnk[kk]) g = (g + p - 1) % p;
                Gm_out[rnk[kk] * PANEL + c] = (uint16_t)g;
            } else {
                Gm_out[kk * PANEL + c] = 0;
            }
        }
    }
}

__global__ void gather_rows_kernel(const uint16_t *__restrict__ D, int64_t ldd, const int32_t *__restrict__ rows,
                                   int64_t nrows, int64_t n, uint16_t *__restrict__ R, int64_t ldr)
{
    for (int64_t k = blockIdx.y; k < nrows; k += gridDim.y) {
        const uint16_t *src = D + (int64_t)rows[k] * ldd;
        uint16_t *dst = R + k * ldr;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            dst[i] = src[i];
    }
}

// For every diagonal block b of 128 rows: Nm_b = I - T^-1 with
// T = R[lo + i][pcol[lo + j]], lo = 128 b (w x w, unit upper triangular).
// The off-diagonal updates of the back-substitution only touch columns at or
// right of the next block's pivots, so these blocks are final from the start
// and all inverses are formed in one launch.
__global__ void __launch_bounds__(128) leaf_inverse_kernel(const uint16_t *__restrict__ R, int64_t ldr, int64_t rank,
                                                           const int32_t *__restrict__ pcol,
                                                           uint16_t *__restrict__ Nm_all, ModP mp)
{
    const int64_t lo = (int64_t)blockIdx.x * 128;
    const int w = (int)((rank - lo) < 128 ? (rank - lo) : 128);
    uint16_t *Nm = Nm_all + (size_t)blockIdx.x * PANEL * PANEL;
    extern __shared__ uint16_t inv_smem[];
    uint16_t(*T)[129] = reinterpret_cast<uint16_t(*)[129]>(inv_smem);             // [128][129]
    uint16_t(*Z)[129] = reinterpret_cast<uint16_t(*)[129]>(inv_smem + 128 * 129);  // [128][129]
    const int j = threadIdx.x;
    for (int i = 0; i < w; ++i)
        T[i][j] = (j < w) ? R[(lo + i) * ldr + pcol[lo + j]] : 0;
    __syncthreads();
    const uint64_t P = mp.p;
    // column j of Z = T^-1, rows from the bottom: Z[i][j] = d_ij - sum_{i<k<=j} T[i][k] Z[k][j]
    for (int i = w - 1; i >= 0; --i) {
        if (j < w) {
            uint64_t acc = (i == j) ? 1 : 0;
            uint64_t sub = 0;
            for (int k = i + 1; k <= j; ++k) sub += (uint64_t)T[i][k] * Z[k][j];
            Z[i][j] = (uint16_t)((j < i) ? 0u : mod40(acc + P * P - mod40(sub, mp), mp));
        }
        __syncthreads();
    }
    for (int i = 0; i < w; ++i)
        if (j < PANEL) {
            uint32_t z = (j < w) ? Z[i][j] : 0u;
            uint32_t v = ((i == j) ? 1u : 0u) + mp.p - z;
            Nm[i * PANEL + j] = (uint16_t)(v % mp.p);
        }
}

constexpr int LEAF_INV_SMEM = 2 * 128 * 129 * (int)sizeof(uint16_t);

struct EchScratch {
    int32_t *info, *cand, *t_dev, *S, *Spos, *pc, *lead;
    uint16_t *Gm, *inv_tab;
    Planes Gp, Bs, H;
};

static int backsub_rec(const EchelonD &E, uint16_t *R, int64_t ldr, const int32_t *pcol_dev,
                       const std::vector<int32_t> &pcol, int64_t lo, int64_t hi, Planes &Ap, Planes &Bp,
                       const uint16_t *Nm_all)
{
    const ModP &mp = *E.mp;
    cudaStream_t s = E.s;
    const int64_t n = E.n;
    if (hi - lo <= PANEL) {
        // leaves are the 128-row blocks (splits fall on multiples of 128)
        const int w = (int)(hi - lo);
        const int64_t cs = pcol[lo] & ~int64_t(63);   // rows lo.. are zero left of pcol[lo]
        const uint16_t *Nm = Nm_all + (size_t)(lo / PANEL) * PANEL * PANEL;
        GBLA_TRY(to_planes(Ap, w, w, Nm, PANEL, 0, false, nullptr, nullptr, mp, s));
        GBLA_TRY(to_planes(Bp, n - cs, w, R + lo * ldr, ldr, cs, true, nullptr, nullptr, mp, s));
        return modgemm(Ap, 0, 0, Bp, 0, 0, R + lo * ldr + cs, ldr, w, n - cs, w, -1, mp, E.variant, E.err, s,
                       E.ctr);
    }
    const int64_t mid = lo + round_up((hi - lo) / 2, PANEL);
    GBLA_TRY(backsub_rec(E, R, ldr, pcol_dev, pcol, mid, hi, Ap, Bp, Nm_all));
    // R[lo:mid] -= R[lo:mid, P_D[mid:hi]] * R[mid:hi]   (rows mid.. are zero left of P_D[mid])
    const int64_t cs = pcol[mid] & ~int64_t(63);
    GBLA_TRY(to_planes(Ap, mid - lo, hi - mid, R + lo * ldr, ldr, 0, false, nullptr, pcol_dev + mid, mp, s));
    GBLA_TRY(to_planes(Bp, n - cs, hi - mid, R + mid * ldr, ldr, cs, true, nullptr, nullptr, mp, s));
    GBLA_TRY(modgemm(Ap, 0, 0, Bp, 0, 0, R + lo * ldr + cs, ldr, mid - lo, n - cs, hi - mid, -1, mp, E.variant,
                     E.err, s, E.ctr));
    return backsub_rec(E, R, ldr, pcol_dev, pcol, lo, mid, Ap, Bp, Nm_all);
}

int echelon_d(const EchelonD &E, int64_t *rank_out)
{
    *rank_out = 0;
    const int64_t m = E.m, n = E.n;
    if (m <= 0 || n <= 0) return GBLA_OK;
    cudaStream_t s = E.s;
    const ModP &mp = *E.mp;
    EchScratch X{};
    int rc = GBLA_OK;
    int64_t rank = 0;
    int32_t info_h[2];
    GBLA_CUDA_TRY(cudaMemsetAsync(E.is_piv_row, 0, sizeof(int32_t) * (size_t)m, s));
    GBLA_TRY(dalloc_t(&X.info, 4, s));
    GBLA_TRY(dalloc_t(&X.cand, (size_t)m + 1, s));
    GBLA_TRY(dalloc_t(&X.t_dev, 4, s));
    GBLA_TRY(dalloc_t(&X.S, PANEL, s));
    GBLA_TRY(dalloc_t(&X.Spos, PANEL, s));
    GBLA_TRY(dalloc_t(&X.pc, PANEL, s));
    GBLA_TRY(dalloc_t(&X.lead, (size_t)m + 1, s));
    GBLA_TRY(dalloc_t(&X.Gm, (size_t)PANEL * PANEL, s));
    GBLA_TRY(dalloc_t(&X.inv_tab, 65536, s));
    inverse_table_kernel<<<(mp.p + 255) / 256, 256, 0, s>>>(X.inv_tab, mp);
    GBLA_CUDA_TRY(launch_check());
    GBLA_TRY(planes_alloc(&X.Gp, PANEL, PANEL, 2, s));
    GBLA_TRY(planes_alloc(&X.Bs, n, PANEL, 4, s));
    GBLA_TRY(planes_alloc(&X.H, m, PANEL, 2, s));
    static bool attr = false;
    if (!attr) {
        GBLA_CUDA_TRY(cudaFuncSetAttribute(panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PANEL_SMEM));
        GBLA_CUDA_TRY(cudaFuncSetAttribute(leaf_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           LEAF_INV_SMEM));
        attr = true;
    }
    row_leads_kernel<<<(unsigned)((m * 32 + 255) / 256), 256, 0, s>>>(E.D16, E.ldd, n, m, nullptr, nullptr, 0,
                                                                     nullptr, X.lead);
    GBLA_CUDA_TRY(launch_check());
    // ---- forward pass (one host synchronisation per panel, to size the launches)
    int32_t *rank_dev = nullptr;
    GBLA_TRY(dalloc_t(&rank_dev, 1, s));
    GBLA_CUDA_TRY(cudaMemsetAsync(rank_dev, 0, sizeof(int32_t), s));
    for (int64_t iter = 0;; ++iter) {
        // every panel turns at least its first candidate into a pivot
        if (iter > m) { rc = GBLA_E_INTERNAL; break; }
        candidates_kernel<<<1, 1024, 0, s>>>(m, X.lead, E.is_piv_row, X.cand, X.info);
        if (launch_check() != cudaSuccess) { rc = GBLA_E_CUDA; break; }
        if (cudaMemcpyAsync(info_h, X.info, sizeof(info_h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) { rc = GBLA_E_CUDA; break; }
        const int64_t c0 = info_h[0];
        const int ncand = info_h[1];
        if (c0 < 0 || ncand == 0) break;
        const int bw = (int)((n - c0) < PANEL ? (n - c0) : PANEL);
        // at most min(ncand, bw) pivots; the launches below are sized by that
        // bound and the sentinel rows of S make the surplus a no-op
        const int tb = ncand < bw ? ncand : bw;
        // Rows of S and the candidates are zero left of c0, so the products may
        // start at the 64-aligned column c0a (they add zeros there); this keeps
        // the C rows 16-byte aligned for the vectorised epilogue.
        const int64_t c0a = c0 & ~int64_t(63);
        const int64_t nc = n - c0a;
        panel_kernel<<<1, 2 * PANEL, PANEL_SMEM, s>>>(E.D16, E.ldd, X.info, n, X.cand, X.inv_tab, E.is_piv_row,
                                                      X.t_dev, X.S, X.Spos, X.pc, X.Gm, E.prow, E.pcol, rank_dev, mp);
        if (launch_check() != cudaSuccess) { rc = GBLA_E_CUDA; break; }
        // D[S, c0:] <- G * D[S, c0:]  as  D[S] += (G - I) * D[S]
        if ((rc = to_planes(X.Gp, tb, tb, X.Gm, PANEL, 0, false, nullptr, nullptr, mp, s))) break;
        if ((rc = to_planes(X.Bs, nc, tb, E.D16, E.ldd, c0a, true, X.S, nullptr, mp, s))) break;
        if ((rc = modgemm(X.Gp, 0, 0, X.Bs, 0, 0, E.D16 + c0a, E.ldd, tb, nc, tb, +1, mp, E.variant, E.err, s, E.ctr,
                          X.S))) break;
        if (ncand > 1) {
            // D[cand, c0:] -= D[cand, c0 + pc] * D[S, c0:]   (rows of S have a zero multiplier row)
            if ((rc = to_planes(X.Bs, nc, tb, E.D16, E.ldd, c0a, true, X.S, nullptr, mp, s))) break;
            Planes Hc = X.H;
            // (rows that just became pivots read as zero rows)
            if ((rc = to_planes(Hc, ncand, tb, E.D16, E.ldd, c0, false, X.cand, X.pc, mp, s, E.is_piv_row))) break;
            if ((rc = modgemm(Hc, 0, 0, X.Bs, 0, 0, E.D16 + c0a, E.ldd, ncand, nc, tb, -1, mp, E.variant, E.err, s,
                              E.ctr, X.cand))) break;
            row_leads_kernel<<<(unsigned)(((int64_t)ncand * 32 + 255) / 256), 256, 0, s>>>(
                E.D16, E.ldd, n, m, X.cand, X.info + 1, c0 + bw, E.is_piv_row, X.lead);
            if (launch_check() != cudaSuccess) { rc = GBLA_E_CUDA; break; }
        }
    }
    {
        int32_t r32 = 0;
        if (cudaMemcpyAsync(&r32, rank_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) rc = GBLA_E_CUDA;
        rank = r32;
    }
    dfree(rank_dev, s);
    // ---- backward pass: RREF rows into R (pivot column order)
    if (rc == GBLA_OK && rank > 0) {
        const int64_t ldr = E.ldd;
        std::vector<int32_t> pcol_h((size_t)rank);
        uint16_t *Nm = nullptr;
        Planes Ap{}, Bp{};
        rc = dalloc_t(&E.R[0], (size_t)rank * (size_t)ldr, s);
        if (rc == GBLA_OK && cudaMemcpyAsync(pcol_h.data(), E.pcol, sizeof(int32_t) * (size_t)rank,
                                             cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = GBLA_E_CUDA;
        if (rc == GBLA_OK) {
            dim3 grid((unsigned)((n + 255) / 256 < 64 ? (n + 255) / 256 : 64), (unsigned)(rank < 65535 ? rank : 65535));
            gather_rows_kernel<<<grid, 256, 0, s>>>(E.D16, E.ldd, E.prow, rank, n, E.R[0], ldr);
            if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
        }
        if (rc == GBLA_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = GBLA_E_CUDA;
        const int64_t nleaves = (rank + PANEL - 1) / PANEL;
        if (rc == GBLA_OK) rc = dalloc_t(&Nm, (size_t)nleaves * PANEL * PANEL, s);
        if (rc == GBLA_OK) {
            leaf_inverse_kernel<<<(unsigned)nleaves, 128, LEAF_INV_SMEM, s>>>(E.R[0], ldr, rank, E.pcol, Nm, mp);
            if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
        }
        if (rc == GBLA_OK) rc = planes_alloc(&Ap, rank, rank < 2 * PANEL ? PANEL : rank, 2, s);
        if (rc == GBLA_OK) rc = planes_alloc(&Bp, n, rank < 2 * PANEL ? PANEL : rank, 4, s);
        if (rc == GBLA_OK) rc = backsub_rec(E, E.R[0], ldr, E.pcol, pcol_h, 0, rank, Ap, Bp, Nm);
        dfree(Nm, s);
        planes_free(&Ap, s);
        planes_free(&Bp, s);
    }
    dfree(X.info, s);
    dfree(X.cand, s);
    dfree(X.t_dev, s);
    dfree(X.S, s);
    dfree(X.Spos, s);
    dfree(X.pc, s);
    dfree(X.lead, s);
    dfree(X.Gm, s);
    dfree(X.inv_tab, s);
    planes_free(&X.Gp, s);
    planes_free(&X.Bs, s);
    planes_free(&X.H, s);
    *rank_out = rank;
    return rc;
}

}  // namespace gbla
