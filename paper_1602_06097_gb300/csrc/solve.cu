// solve.cu -- the sparse reduction C <- C*A^-1 (new order of operations,
// Alg. 2 and its four-step implementation, GBLA paper Sec. 4.3), the
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
        *Xp.at(0, r1, j0 + c) = i2bf(hi);
        *Xp.at(1, r1, j0 + c) = i2bf(lo);
        if (has2) {
            const uint32_t x2 = (uint32_t)acc[1][c];
            C16[r2 * ldc + j0 + c] = (uint16_t)x2;
            digits(x2, p, hi, lo);
            *Xp.at(0, r2, j0 + c) = i2bf(hi);
            *Xp.at(1, r2, j0 + c) = i2bf(lo);
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
    const bool tc_leaf = T.Zt && T.Ct;
    const int64_t LW = tc_leaf ? T.tc_leaf : LEAF;   // leaf width
    if (hi - lo <= LW) {
        // rows leading at or after hi have a zero block here (C and X alike)
        const int64_t rows = rows_before(T, hi);
        if (rows == 0) return GBLA_OK;
        if (tc_leaf) {
            // X_J = C_J * A_JJ^-1: digit planes of C_J, then one product whose
            // epilogue writes the digit planes of X_J
            const int w = (int)(hi - lo);
            GBLA_TRY(to_planes(*T.Ct, rows, w, T.C16 + lo, T.ldc, 0, false, nullptr, nullptr, *T.mp, T.s));
            return modgemm_to_planes(*T.Ct, 0, *T.Zt, lo, *T.Xp, lo, rows, w, w, *T.mp, T.err, T.s, T.ctr);
        }
        const int64_t pairs = (rows + 1) / 2;
        trsm_upper_leaf_kernel<<<(unsigned)((pairs + LEAF_WARPS - 1) / LEAF_WARPS), 32 * LEAF_WARPS,
                                 LEAF_SMEM_UPPER, T.s>>>(rows, lo, (int)(hi - lo), T.ml->ptr, T.ml->pos, T.ml->val,
                                                         T.ml->inblk, T.C16, T.ldc, *T.Xp, *T.mp);
        GBLA_CUDA_TRY(launch_check());
        return GBLA_OK;
    }
    const int64_t mid = lo + round_up((hi - lo) / 2, LW);
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
        *Xp.at(0, r1, j0 + c) = i2bf(hi);
        *Xp.at(1, r1, j0 + c) = i2bf(lo);
        if (has2) {
            const uint32_t x2 = xs[1][c];
            C16[r2 * ldc + j0 + c] = (uint16_t)x2;
            digits(x2, p, hi, lo);
            *Xp.at(0, r2, j0 + c) = i2bf(hi);
            *Xp.at(1, r2, j0 + c) = i2bf(lo);
        }
    }
}

static int leaf_attrs()
{
    static const cudaError_t rc = [] {
        cudaError_t e = cudaFuncSetAttribute(trsm_upper_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             LEAF_SMEM_UPPER);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(trsm_lower_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     LEAF_SMEM_LOWER);
        return e;
    }();
    GBLA_CUDA_TRY(rc);
    return GBLA_OK;
}

int trsm_upper(const TrsmUpper &T)
{
    if (T.mrows <= 0 || T.npiv <= 0) return GBLA_OK;
    GBLA_TRY(leaf_attrs());
    return trsm_upper_rec(T, 0, T.npiv);
}

// dst[r][c] <- the residue whose digits X holds at (r, c), r < rows, c < cols.
__global__ void __launch_bounds__(256) planes_to_u16_kernel(Planes X, int64_t rows, int64_t cols, uint16_t *dst,
                                                            int64_t ld, ModP mp)
{
    const int64_t r = blockIdx.x;   // one block per row
    if (r >= rows) return;
    for (int64_t c = threadIdx.x; c < cols; c += 256) {
        const int v = 256 * __float2int_rz(__bfloat162float(*X.at(0, r, c))) +
                      __float2int_rz(__bfloat162float(*X.at(1, r, c)));
        dst[r * ld + c] = (uint16_t)(v < 0 ? v + (int)mp.p : v);
    }
}

static int trsm_lower_rec(const TrsmLower &T, int64_t lo, int64_t hi)
{
    const bool tc_leaf = T.Zr && T.Ct && T.tc_leaf > 0;
    if (tc_leaf && hi - lo <= T.tc_leaf) {
        // X'_J = C'_J Z_J^T: digit planes of C'_J, then one product whose
        // epilogue writes the digit planes of X'_J
        const int w = (int)(hi - lo);
        GBLA_TRY(to_planes(*T.Ct, T.mrows, w, T.C16 + lo, T.ldc, 0, false, nullptr, nullptr, *T.mp, T.s));
        return modgemm_to_planes(*T.Ct, 0, *T.Zr, lo, *T.Xp, lo, T.mrows, w, w, *T.mp, T.err, T.s, T.ctr);
    }
    if (!tc_leaf && hi - lo <= LEAF) {
        const int64_t pairs = (T.mrows + 1) / 2;
        trsm_lower_leaf_kernel<<<(unsigned)((pairs + LEAF_WARPS - 1) / LEAF_WARPS), 32 * LEAF_WARPS,
                                 LEAF_SMEM_LOWER, T.s>>>(T.mrows, lo, (int)(hi - lo), T.ml->ptr, T.ml->pos, T.ml->val,
                                                         T.ml->inblk, T.C16, T.ldc, *T.Xp, *T.mp);
        GBLA_CUDA_TRY(launch_check());
        return GBLA_OK;
    }
    const int64_t mid = lo + round_up((hi - lo) / 2, tc_leaf ? T.tc_leaf : LEAF);
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
    GBLA_TRY(trsm_lower_rec(T, 0, T.npiv));
    if (T.Zr && T.Ct && T.tc_leaf > 0) {
        // the tensor-core leaves wrote X' as digit planes only: its residues
        planes_to_u16_kernel<<<(unsigned)T.mrows, 256, 0, T.s>>>(*T.Xp, T.mrows, T.npiv, T.C16, T.ldc, *T.mp);
        GBLA_CUDA_TRY(launch_check());
    }
    return GBLA_OK;
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

// First nonzero column of each listed row (or every row), -1 if none.  The
// search starts at `from`, or, with from < 0, at the panel boundary after
// the row's current lead (the row was just cleared on its lead's panel).
// Rows: rows[seg[0] .. seg[1]) with seg on the device, else rows[0 .. count)
// (or rows 0 .. count when rows is null).  One warp per row; every lane loads
// two 16-byte vectors (8 columns each; the start is a multiple of 8 and ldd a
// multiple of 64, so they are aligned and inside the row) before testing any,
// so a step covers 512 columns with a single memory round trip.
__global__ void row_leads_kernel(const uint16_t *__restrict__ D, int64_t ldd, int64_t n, int64_t count,
                                 const int32_t *__restrict__ rows, const int64_t *__restrict__ seg,
                                 int64_t from, const int32_t *__restrict__ skip, int32_t *__restrict__ lead)
{
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t b = seg ? seg[0] : 0, cnt = seg ? seg[1] - seg[0] : count;
    if (w >= cnt) return;
    const int64_t r = rows ? rows[b + w] : w;
    if (skip && skip[r]) return;
    const uint16_t *row = D + r * ldd;
    const int64_t start = from >= 0 ? from : ((int64_t)lead[r] / PANEL + 1) * PANEL;
    int64_t found = -1;
    for (int64_t base = start; base < n && found < 0; base += 512) {
        uint4 v[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t c0 = base + u * 256 + lane * 8;
            v[u] = (c0 < n) ? *reinterpret_cast<const uint4 *>(row + c0) : make_uint4(0u, 0u, 0u, 0u);
        }
        int64_t best = INT64_MAX;
#pragma unroll
        for (int u = 1; u >= 0; --u) {   // the lower vector last: its hit wins
            const uint32_t wd[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
            int idx = -1;
#pragma unroll
            for (int q = 3; q >= 0; --q)
                if (wd[q]) idx = 2 * q + ((wd[q] & 0xFFFFu) ? 0 : 1);
            const int64_t c = base + u * 256 + lane * 8 + idx;
            if (idx >= 0 && c < n) best = c;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int64_t t = __shfl_xor_sync(0xFFFFFFFFu, best, o);
            best = t < best ? t : best;
        }
        if (best != INT64_MAX) found = best;
    }
    if (lane == 0) lead[r] = (int32_t)found;
}

// Candidate lists of the fixed panels (panel k = columns [128k, 128k + 128)):
// the non-pivot rows whose lead falls in the panel, in row order.
__global__ void panel_count_kernel(int64_t m, const int32_t *__restrict__ lead, const int32_t *__restrict__ is_piv_row,
                                   int64_t *__restrict__ cnt)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < m && !is_piv_row[r] && lead[r] >= 0)
        atomicAdd(reinterpret_cast<unsigned long long *>(&cnt[lead[r] / PANEL]), 1ull);
}

__global__ void panel_scatter_kernel(int64_t m, const int32_t *__restrict__ lead, const int32_t *__restrict__ is_piv_row,
                                     const int64_t *__restrict__ off, int32_t *__restrict__ fill,
                                     int32_t *__restrict__ cand)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m || is_piv_row[r] || lead[r] < 0) return;
    const int k = lead[r] / PANEL;
    cand[off[k] + atomicAdd(&fill[k], 1)] = (int32_t)r;
}

// Each panel's candidate list into ascending row order (lists longer than
// 2048 are left as they are): one CTA per panel, a bitonic sort in shared
// memory over the list padded to a power of two.
constexpr int PANEL_SORT_MAX = 2048;
__global__ void __launch_bounds__(256) panel_sort_kernel(int64_t npan, const int64_t *__restrict__ off,
                                                         int32_t *__restrict__ cand)
{
    __shared__ int32_t sv[PANEL_SORT_MAX];
    const int64_t k = blockIdx.x;
    if (k >= npan) return;
    const int64_t b = off[k];
    const int64_t len = off[k + 1] - b;
    if (len <= 1 || len > PANEL_SORT_MAX) return;
    int n2 = 2;
    while (n2 < len) n2 <<= 1;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) sv[i] = (i < len) ? cand[b + i] : INT32_MAX;
    __syncthreads();
    for (int size = 2; size <= n2; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < n2 / 2; i += blockDim.x) {
                const int lo = 2 * stride * (i / stride) + (i % stride), hi = lo + stride;
                const int32_t x = sv[lo], y = sv[hi];
                if ((x > y) == ((lo & size) == 0)) {
                    sv[lo] = y;
                    sv[hi] = x;
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < len; i += blockDim.x) cand[b + i] = sv[i];
}

// Jobs of a wave: the panels with candidates, ascending; seg[j] = offset of
// job j's candidates (candidates of consecutive non-empty panels are
// contiguous).  njobs -> info[0].  One CTA.
__global__ void __launch_bounds__(1024) make_jobs_kernel(int64_t npan, const int64_t *__restrict__ off,
                                                         int32_t *__restrict__ job_slot, int64_t *__restrict__ seg,
                                                         int32_t *__restrict__ info)
{
    __shared__ int wsum[32];
    __shared__ int base;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) base = 0;
    __syncthreads();
    for (int64_t k0 = 0; k0 < npan; k0 += blockDim.x) {
        const int64_t k = k0 + tid;
        const int f = (k < npan && off[k + 1] > off[k]) ? 1 : 0;
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, f);
        if (lane == 0) wsum[wid] = __popc(bal);
        __syncthreads();
        int o = base;
        for (int q = 0; q < wid; ++q) o += wsum[q];
        if (f) {
            const int j = o + __popc(bal & ((1u << lane) - 1u));
            job_slot[j] = (int32_t)k;
            seg[j] = off[k];
        }
        __syncthreads();
        if (tid == 0) {
            int tot = 0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += wsum[q];
            base += tot;
        }
        __syncthreads();
    }
    if (tid == 0) {
        seg[base] = off[npan];
        info[0] = base;
    }
}

// Inverses of all residues (0 -> 0), for the panel kernel's table.
__global__ void inverse_table_kernel(uint16_t *__restrict__ tab, ModP mp)
{
    const uint32_t a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < mp.p) tab[a] = (uint16_t)(a ? invmod(a, mp) : 0u);
}

constexpr size_t PANEL_SMEM = (size_t)PANEL * 2 * PANEL * sizeof(uint16_t) + 65536 * sizeof(uint16_t);

// One CTA per job.  Job j works on panel slot = job_slot[j] (or j), columns
// [128 slot, 128 slot + 128), with candidate rows cand[seg[j] .. seg[j+1]);
// the slot's pivots from earlier waves are its first basis rows.  Outputs of
// the slot: t, S (physical row of the pivot with the i-th smallest column,
// -1 beyond t), pc (pivot columns in the panel, ascending, -1 beyond t),
// Gm = G - I (128 x 128, zero beyond t) over all t pivot rows.
__global__ void __launch_bounds__(256) panel_kernel(const uint16_t *__restrict__ D, int64_t ldd, int64_t n,
                                                    const int64_t *__restrict__ seg, const int32_t *__restrict__ cand,
                                                    const int32_t *__restrict__ job_slot,
                                                    const uint16_t *__restrict__ inv_tab,
                                                    int32_t *__restrict__ is_piv_row, int32_t *__restrict__ t_slot,
                                                    int32_t *__restrict__ S_slot, int32_t *__restrict__ pc_slot,
                                                    uint16_t *__restrict__ Gm_all, int32_t *__restrict__ wave_slot,
                                                    ModP mp)
{
    extern __shared__ __align__(16) uint16_t panel_smem[];
    uint16_t(*aug)[2 * PANEL] = reinterpret_cast<uint16_t(*)[2 * PANEL]>(panel_smem);  // [PANEL][256]
    uint16_t *inv_s = panel_smem + PANEL * 2 * PANEL;                                  // [p]
    __shared__ uint32_t cand_v[2 * PANEL];
    __shared__ uint32_t fk[PANEL], coef[PANEL];
    __shared__ int bcol[PANEL], brow[PANEL], S[PANEL], rnk[PANEL];
    __shared__ int wmin[8];
    const int c = threadIdx.x;  // column of the augmented row: [panel | coefficients]
    const int lane = c & 31, warp = c >> 5;
    const int job = blockIdx.x;
    const int slot = job_slot ? job_slot[job] : job;
    if (slot < 0) return;
    const int64_t c0 = (int64_t)slot * PANEL;
    const int32_t *cl = cand + seg[job];
    const int ncand = (int)(seg[job + 1] - seg[job]);
    const int bw = (int)((n - c0) < PANEL ? (n - c0) : PANEL);
    const uint32_t p = mp.p;
    int32_t *S_out = S_slot + (int64_t)slot * PANEL;
    int32_t *pc_out = pc_slot + (int64_t)slot * PANEL;
    uint16_t *Gm_out = Gm_all + (int64_t)slot * PANEL * PANEL;
    if (ncand == 0) return;   // nothing new: the slot keeps its outputs
    {
        // inverse table into shared memory (16-byte copies; p <= 65536 entries)
        const int nvec = (int)((p + 7) / 8);
        const uint4 *src = reinterpret_cast<const uint4 *>(inv_tab);
        uint4 *dst = reinterpret_cast<uint4 *>(inv_s);
        for (int i = c; i < nvec; i += 2 * PANEL) dst[i] = src[i];
    }
    if (c < PANEL) brow[c] = -1;     // basis row whose pivot is panel column c
    // The slot's pivots from earlier waves are in reduced echelon form on the
    // panel (identity at their columns): they enter the basis as they are,
    // with unit coefficient rows.
    const int tpre = t_slot[slot];
    for (int i = 0; i < tpre; ++i) {
        const int64_t row = S_out[i];
        aug[i][c] = (uint16_t)((c < bw) ? D[row * ldd + c0 + c] : ((c - PANEL == i) ? 1u : 0u));
    }
    if (c < tpre) {
        bcol[c] = pc_out[c];
        S[c] = S_out[c];
    }
    __syncthreads();
    if (c < tpre) brow[bcol[c]] = c;
    __syncthreads();
    int t = tpre;
    // software pipeline: the next candidate's panel entry is loaded while the
    // current one is processed
    uint32_t vnext = 0;
    if (ncand > 0 && c < bw) vnext = D[(int64_t)cl[0] * ldd + c0 + c];
    for (int ci = 0; ci < ncand && t < bw; ++ci) {
        uint32_t v = vnext;
        if (ci + 1 < ncand && c < bw) vnext = D[(int64_t)cl[ci + 1] * ldd + c0 + c];
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
            S[t] = (int)cl[ci];
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
        t_slot[slot] = t;
        // this wave: new pivots, and candidates that stayed dependent
        wave_slot[2 * slot] = t - tpre;
        wave_slot[2 * slot + 1] = ncand - (t - tpre);
    }
    if (c < PANEL) {
        // the pivot with the c-th smallest column lands in physical row S[c];
        // entries beyond t are sentinels (-1): the products skip them
        S_out[c] = (c < t) ? S[c] : -1;
        if (c < t) {
            pc_out[rnk[c]] = bcol[c];
            is_piv_row[S[c]] = 1;
        } else {
            pc_out[c] = -1;
        }
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

// Per panel of a chunk: where its rows of the D[S]^T plane set start, its
// slot and its column count n - 128 slot.
struct PanelPlan {
    int64_t boff;
    int32_t slot, nc;
};

// A-operand planes of G - I for the jobs of a chunk: rows q * 128 + i of dst
// = row i of the slot's Gm (blockIdx.y = q, blockIdx.x = i).
__global__ void gather_gm_planes_kernel(Planes dst, const uint16_t *__restrict__ Gm_all,
                                        const PanelPlan *__restrict__ plan, uint32_t p)
{
    const int q = blockIdx.y, i = blockIdx.x, j = threadIdx.x;
    const uint32_t a = Gm_all[(int64_t)plan[q].slot * PANEL * PANEL + i * PANEL + j];
    int hi, lo;
    digits(a, p, hi, lo);
    *dst.at(0, (int64_t)q * PANEL + i, j) = i2bf(hi);
    *dst.at(1, (int64_t)q * PANEL + i, j) = i2bf(lo);
}

// B-operand planes of D[S]^T for every panel of a chunk (blockIdx.z):
// dst[boff + i][j] = D[S_j][128 slot + i] for j < t, else 0.
__global__ void __launch_bounds__(256) gather_t_planes_kernel(Planes dst, const uint16_t *__restrict__ D,
                                                              int64_t ldd, const PanelPlan *__restrict__ plan,
                                                              const int32_t *__restrict__ S_slot,
                                                              const int32_t *__restrict__ t_slot, ModP mp)
{
    __shared__ TpSmem sm;
    const PanelPlan pl = plan[blockIdx.z];
    const int64_t r0 = (int64_t)blockIdx.x * TP_TILE, k0 = (int64_t)blockIdx.y * TP_TILE;
    if (r0 >= round_up(pl.nc, 128)) return;
    tp_tile(dst, pl.boff, r0, k0, pl.nc, t_slot[pl.slot], D, ldd, (int64_t)pl.slot * PANEL,
            S_slot + (int64_t)pl.slot * PANEL, mp, sm);
}

// A-operand planes of the candidates' entries at their panel's pivot columns:
// row r - row_base of dst = D[cand[r]][128 slot + pc_j] for j < t (zero for
// rows that are pivots now).  blockIdx.y = job of the chunk.
__global__ void gather_h_planes_kernel(Planes dst, uint16_t *__restrict__ H16, const uint16_t *__restrict__ D,
                                       int64_t ldd, const int64_t *__restrict__ seg, const int32_t *__restrict__ cand,
                                       const int32_t *__restrict__ job_slot, int job0, int64_t row_base,
                                       const int32_t *__restrict__ pc_slot, const int32_t *__restrict__ t_slot,
                                       const int32_t *__restrict__ is_piv_row, uint32_t p)
{
    const int job = job0 + blockIdx.y;
    const int slot = job_slot ? job_slot[job] : job;
    if (slot < 0) return;
    const int t = t_slot[slot];
    const int j = threadIdx.x;   // 128 threads: K column
    const int pcj = (j < t) ? pc_slot[(int64_t)slot * PANEL + j] : -1;
    for (int64_t r = seg[job] + blockIdx.x; r < seg[job + 1]; r += gridDim.x) {
        const int64_t row = cand[r];
        uint32_t a = 0;
        if (pcj >= 0 && !is_piv_row[row]) a = D[row * ldd + (int64_t)slot * PANEL + pcj];
        int hi, lo;
        digits(a, p, hi, lo);
        *dst.at(0, r - row_base, j) = i2bf(hi);
        *dst.at(1, r - row_base, j) = i2bf(lo);
        H16[(r - row_base) * PANEL + j] = (uint16_t)a;
    }
}

// B-operand planes of (G - I)^T for the jobs of a chunk: row q * 128 + j,
// column k <- (G - I)[k][j] of the slot's Gm (blockIdx.y = q, blockIdx.x = j).
__global__ void gather_gmt_planes_kernel(Planes dst, const uint16_t *__restrict__ Gm_all,
                                         const PanelPlan *__restrict__ plan, ModP mp)
{
    const int q = blockIdx.y, j = blockIdx.x, k = threadIdx.x;
    const uint32_t a = Gm_all[(int64_t)plan[q].slot * PANEL * PANEL + k * PANEL + j];
    const int64_t row = (int64_t)q * PANEL + j;
    int hi, lo;
    digits(a, mp.p, hi, lo);
    *dst.at(0, row, k) = i2bf(hi);
    *dst.at(1, row, k) = i2bf(lo);
    digits(mod32(a * mp.r256, mp), mp.p, hi, lo);
    *dst.at(2, row, k) = i2bf(hi);
    *dst.at(3, row, k) = i2bf(lo);
}

__global__ void iota_kernel(int32_t *v, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (int32_t)i;
}

// Exclusive prefix sum of v across the block (blockDim.x a multiple of 32,
// at most 1024); *total receives the block's sum.  All threads must call it.
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *total)
{
    __shared__ int64_t wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < nw) wsum[lane] = w;   // inclusive warp prefixes
    }
    __syncthreads();
    const int64_t before = warp > 0 ? wsum[warp - 1] : 0;
    *total = wsum[nw - 1];
    __syncthreads();   // wsum is reused by the next call
    return before + incl - v;
}

// Problem tables of the grouped products of a chunk (one block, the jobs in
// chunks of blockDim.x, tile offsets by a block-wide prefix sum).
// mode 1: D[S] += (G - I) * D[S];  mode 2: D[cand] -= (H G) * D[S]_old;
// mode 3: H16 += H * (G - I), i.e. H16 <- H G, where H = D[cand, pc].
__global__ void make_probs_kernel(GroupProb *probs, int nprob, int mode, const PanelPlan *__restrict__ plan,
                                  const int32_t *__restrict__ t_slot, const int32_t *__restrict__ S_slot,
                                  const int32_t *__restrict__ wave_slot, const int64_t *__restrict__ seg,
                                  const int32_t *__restrict__ cand, int job0, int64_t row_base,
                                  const int32_t *__restrict__ iota)
{
    int64_t off = 0;   // tiles of the chunks before
    for (int q0 = 0; q0 < nprob; q0 += blockDim.x) {
        const int q = q0 + (int)threadIdx.x;
        GroupProb P{};
        int64_t cnt = 0;
        if (q < nprob) {
            const PanelPlan pl = plan[q];
            const int t = t_slot[pl.slot];
            P.b_row0 = (int32_t)pl.boff;
            P.N = pl.nc;
            P.c_col0 = (int64_t)pl.slot * PANEL;
            if (mode == 1) {
                // no new pivot on the panel: G = I, nothing to do
                P.a_row0 = q * PANEL;
                P.M = wave_slot[2 * pl.slot] > 0 ? t : 0;
                P.c_rows = S_slot + (int64_t)pl.slot * PANEL;
            } else if (mode == 3) {
                // H G = H when G = I; nothing needed without dependent candidates
                const int64_t b = seg[job0 + q], e = seg[job0 + q + 1];
                P.a_row0 = (int32_t)(b - row_base);
                P.b_row0 = q * PANEL;
                P.N = t;
                P.c_col0 = 0;
                P.M = (wave_slot[2 * pl.slot] > 0 && wave_slot[2 * pl.slot + 1] > 0) ? (int32_t)(e - b) : 0;
                P.c_rows = iota + (b - row_base);
            } else {
                // no dependent candidate: nothing to clear
                const int64_t b = seg[job0 + q], e = seg[job0 + q + 1];
                P.a_row0 = (int32_t)(b - row_base);
                P.M = wave_slot[2 * pl.slot + 1] > 0 ? (int32_t)(e - b) : 0;
                P.c_rows = cand + b;
            }
            if (t == 0) P.M = 0;
            cnt = (P.M > 0 && P.N > 0) ? ((int64_t)(P.M + 127) / 128) * ((int64_t)(P.N + 127) / 128) : 0;
        }
        int64_t total = 0;
        const int64_t ex = block_exclusive_scan(cnt, &total);
        if (q < nprob) {
            P.tile_off = off + ex;
            probs[q] = P;
        }
        off += total;
    }
    if (threadIdx.x == 0) probs[nprob].tile_off = off;
}

// Job table of the fused panel application (panel_apply) for the jobs of a
// chunk: job q updates its new pivot rows (if the wave found new pivots on
// its panel: D[S] <- G D[S]) and its dependent candidates (D[cand] -= H G
// D[S]); its A block stacks G - I and -H G, rows a_row0 ..  One block.
__global__ void pa_jobs_kernel(PaJob *jobs, int nj, const PanelPlan *__restrict__ plan,
                               const int32_t *__restrict__ t_slot, const int32_t *__restrict__ S_slot,
                               const int32_t *__restrict__ wave_slot, const int64_t *__restrict__ seg, int job0)
{
    int64_t arow = 0, items = 0;
    for (int q0 = 0; q0 < nj; q0 += blockDim.x) {
        const int q = q0 + (int)threadIdx.x;
        PaJob J{};
        int64_t m = 0, k = 0;
        if (q < nj) {
            const PanelPlan pl = plan[q];
            const int t = t_slot[pl.slot];
            const int64_t b = seg[job0 + q], e = seg[job0 + q + 1];
            const int tn = wave_slot[2 * pl.slot] > 0 ? t : 0;                  // rows of G - I
            const int64_t nd = wave_slot[2 * pl.slot + 1] > 0 ? e - b : 0;     // dependent candidates
            J.t = t;
            J.M = t > 0 ? (int32_t)(tn + nd) : 0;
            J.pad = tn;
            J.nc = pl.nc;
            J.col0 = (int64_t)pl.slot * PANEL;
            J.srows = S_slot + (int64_t)pl.slot * PANEL;
            m = J.M;
            k = J.M > 0 ? (pl.nc + 127) / 128 : 0;
        }
        int64_t tot_m = 0, tot_k = 0;
        const int64_t em = block_exclusive_scan(m, &tot_m);
        const int64_t ek = block_exclusive_scan(k, &tot_k);
        if (q < nj) {
            J.a_row0 = arow + em;
            J.item_off = items + ek;
            jobs[q] = J;
        }
        arow += tot_m;
        items += tot_k;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        PaJob end{};
        end.a_row0 = arow;
        end.item_off = items;
        jobs[nj] = end;
    }
}

// A blocks and row maps of the jobs (blockIdx.y = job, rows strided over
// blockIdx.x, thread k = K column): row m < tn is row m of G - I, row tn + r
// is -(H G) of the job's r-th candidate (H G rows as in H16, from row_base);
// K columns past t are 0.  A candidate that became a pivot in this wave is
// also one of the rows G - I updates: its own row (zero multipliers) maps to
// -1, so that the fused drain does not write its old values back.
__global__ void pa_fill_kernel(Planes A, int32_t *__restrict__ rowmap, const PaJob *__restrict__ jobs,
                               const PanelPlan *__restrict__ plan, const uint16_t *__restrict__ Gm_all,
                               const uint16_t *__restrict__ HG, const int64_t *__restrict__ seg,
                               const int32_t *__restrict__ cand, const int32_t *__restrict__ is_piv_row, int job0,
                               int64_t row_base, uint32_t p)
{
    const int q = blockIdx.y, k = threadIdx.x;
    const PaJob J = jobs[q];
    const int tn = J.pad;
    const int64_t b = seg[job0 + q];
    const uint16_t *G = Gm_all + (int64_t)plan[q].slot * PANEL * PANEL;
    for (int64_t m = blockIdx.x; m < J.M; m += gridDim.x) {
        uint32_t a = 0;
        if (k < J.t) {
            if (m < tn) {
                a = G[m * PANEL + k];
            } else {
                const uint32_t h = HG[(b - row_base + (m - tn)) * PANEL + k];
                a = h ? p - h : 0u;
            }
        }
        int hi, lo;
        digits(a, p, hi, lo);
        const int64_t row = J.a_row0 + m;
        *A.at(0, row, k) = i2bf(hi);
        *A.at(1, row, k) = i2bf(lo);
        if (k == 0) {
            int32_t r = m < tn ? J.srows[m] : cand[b + (m - tn)];
            if (m >= tn && is_piv_row[r]) r = -1;
            rowmap[row] = r;
        }
    }
}

// Pivot records in pivot-column order (slots ascending, columns ascending
// inside a slot); *rank receives their number.  One block: a thread per slot,
// record offsets by a block-wide prefix sum.
__global__ void __launch_bounds__(1024) compact_slots_kernel(int64_t npan, const int32_t *__restrict__ t_slot,
                                                             const int32_t *__restrict__ S_slot,
                                                             const int32_t *__restrict__ pc_slot,
                                                             int32_t *__restrict__ prow, int32_t *__restrict__ pcol,
                                                             int64_t *rank)
{
    int64_t off = 0;
    for (int64_t k0 = 0; k0 < npan; k0 += blockDim.x) {
        const int64_t k = k0 + threadIdx.x;
        const int t = k < npan ? t_slot[k] : 0;
        int64_t total = 0;
        const int64_t r = off + block_exclusive_scan(t, &total);
        for (int i = 0; i < t; ++i) {
            prow[r + i] = S_slot[k * PANEL + i];
            pcol[r + i] = (int32_t)(k * PANEL + pc_slot[k * PANEL + i]);
        }
        off += total;
    }
    if (threadIdx.x == 0) *rank = off;
}

// Z = T^-1 for the unit upper triangular w x w block T (shared memory), by
// rows from the bottom: Z[i][j] = d_ij - sum_{i<k<=j} T[i][k] Z[k][j].  Thread
// j owns column j; rows and columns w.. of Z are left untouched.
__device__ __forceinline__ void unit_upper_inverse(const uint16_t (*T)[129], uint16_t (*Z)[129], int w,
                                                   const ModP &mp)
{
    const int j = threadIdx.x;
    const uint64_t P = mp.p;
    for (int i = w - 1; i >= 0; --i) {
        if (j < w) {
            uint64_t acc = (i == j) ? 1 : 0;
            uint64_t sub = 0;
            for (int k = i + 1; k <= j; ++k) sub += (uint64_t)T[i][k] * Z[k][j];
            Z[i][j] = (uint16_t)((j < i) ? 0u : mod40(acc + P * P - mod40(sub, mp), mp));
        }
        __syncthreads();
    }
}

// Inverses of the diagonal blocks of width L (a power of two, multiple of
// 128) of a unit upper triangular n x n matrix T, given as T[i][j] =
// A[r(i) * lda + c(j)] with r, c optional row / column maps (identity when
// null): A itself for the leaf solves X_J = C_J * A_JJ^-1, the echelon rows
// at the pivot columns for the back-substitution.  Z_J = T_JJ^-1 is built in
// ZN (u16, row-major, leaf J at rows J L .. J L + L, row length L, zero
// outside the upper triangle and outside T):
//   1. the 128-blocks on the diagonal, inverted in shared memory;
//   2. for w = 128, 256, .. < L, every pair of neighbouring w-blocks (o1, o2 =
//      o1 + w) of a leaf gets its upper-right block from the block inverse
//      formula  Z12 = -Z11 * A12 * Z22  (two batched products);
//   3. the B-operand planes of Z_J^T (row J L + j, column k <- Z_J[k][j]).
__global__ void __launch_bounds__(128) upper_inverse128_kernel(const uint16_t *__restrict__ A, int64_t lda,
                                                               const int32_t *__restrict__ rmap,
                                                               const int32_t *__restrict__ cmap, int64_t npiv, int L,
                                                               uint16_t *__restrict__ ZN, ModP mp)
{
    const int64_t lo = (int64_t)blockIdx.x * 128;
    const int w = (int)((npiv - lo) < 128 ? (npiv - lo) : 128);
    extern __shared__ uint16_t inv_smem[];
    uint16_t(*T)[129] = reinterpret_cast<uint16_t(*)[129]>(inv_smem);
    uint16_t(*Z)[129] = reinterpret_cast<uint16_t(*)[129]>(inv_smem + 128 * 129);
    const int j = threadIdx.x;
    const int64_t cj = (j < w) ? (cmap ? (int64_t)cmap[lo + j] : lo + j) : 0;
    for (int i = 0; i < w; ++i)
        T[i][j] = (j < w) ? A[(rmap ? (int64_t)rmap[lo + i] : lo + i) * lda + cj] : 0;
    __syncthreads();
    unit_upper_inverse(T, Z, w, mp);
    // lo = J L + o: rows lo + k of ZN, columns o + j
    const int64_t o = lo % L;
    if (j < w)
        for (int k = 0; k <= j; ++k) ZN[(lo + k) * L + o + j] = Z[k][j];
}

// One level of the block inverse formula, batched over all block pairs
// (blockIdx.z = pair; 64 x 64 output tile per CTA, exact uint64 sums):
//   mode 0: T1_b = A[lo+o1.., lo+o2..] * Z22,   mode 1: Z12 = -Z11 * T1_b.
__global__ void __launch_bounds__(256) tri_combine_kernel(int mode, int w, int L, const uint16_t *__restrict__ A,
                                                          int64_t lda, const int32_t *__restrict__ rmap,
                                                          const int32_t *__restrict__ cmap, int64_t npiv,
                                                          uint16_t *__restrict__ ZN, uint16_t *__restrict__ T1,
                                                          ModP mp)
{
    __shared__ uint32_t sx[64][33];
    __shared__ uint32_t sy[32][65];
    const int pairs_per_leaf = L / (2 * w);
    const int64_t b = blockIdx.z;
    const int64_t lo = (b / pairs_per_leaf) * L;
    const int o1 = 2 * w * (int)(b % pairs_per_leaf), o2 = o1 + w;
    const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
    const int tid = threadIdx.x, tr = tid / 16, tc = tid % 16;
    uint16_t *t1 = T1 + b * (int64_t)w * w;
    unsigned long long acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = 0;
    for (int k0 = 0; k0 < w; k0 += 32) {
        for (int e = tid; e < 64 * 32; e += 256) {
            const int r = e >> 5, k = e & 31;
            uint32_t v;
            if (mode == 0) {
                const int64_t ar = lo + o1 + i0 + r, ac = lo + o2 + k0 + k;
                v = (ar < npiv && ac < npiv)
                        ? A[(rmap ? (int64_t)rmap[ar] : ar) * lda + (cmap ? (int64_t)cmap[ac] : ac)]
                        : 0u;
            } else {
                v = ZN[(lo + o1 + i0 + r) * L + o1 + k0 + k];
            }
            sx[r][k] = v;
        }
        for (int e = tid; e < 32 * 64; e += 256) {
            const int k = e >> 6, c = e & 63;
            sy[k][c] = (mode == 0) ? ZN[(lo + o2 + k0 + k) * L + o2 + j0 + c] : t1[(int64_t)(k0 + k) * w + j0 + c];
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            uint32_t xv[4], yv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) xv[i] = sx[tr * 4 + i][k];
#pragma unroll
            for (int q = 0; q < 4; ++q) yv[q] = sy[k][tc * 4 + q];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[i][q] += (unsigned long long)xv[i] * yv[q];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t r = mod64(acc[i][q], mp);
            const int row = i0 + tr * 4 + i, col = j0 + tc * 4 + q;
            if (mode == 0) t1[(int64_t)row * w + col] = (uint16_t)r;
            else ZN[(lo + o1 + row) * L + o2 + col] = (uint16_t)(r ? mp.p - r : 0u);
        }
}

// The same level on the tensor cores, for w >= 256: with pair b's w x w
// operands at plane rows b w .. of shared plane sets,
//   U = Z11 * A12 (into scratch, rows b w ..),  Z12 = -U * Z22 (into ZN),
// two grouped products.  Digit planes of the operands:
//   mode 0: A-operand Z11    row i, K k  <- ZN[lo+o1+i][o1+k]
//   mode 1: B-operand A12^T  row j, K i  <- T[lo+o1+i][lo+o2+j]
//   mode 2: A-operand U      row i, K k  <- U[b w+i][k]
//   mode 3: B-operand Z22^T  row j, K i  <- ZN[lo+o2+i][o2+j]
// 64 x 64 tiles (blockIdx.x: K, blockIdx.y: rows, blockIdx.z: pair), read
// along the source rows into shared memory, written as 16-byte digit vectors.
__global__ void __launch_bounds__(256) pair_planes_kernel(int mode, int w, int L, const uint16_t *__restrict__ A,
                                                          int64_t lda, const int32_t *__restrict__ rmap,
                                                          const int32_t *__restrict__ cmap, int64_t npiv,
                                                          const uint16_t *__restrict__ ZN,
                                                          const uint16_t *__restrict__ U, Planes dst, ModP mp)
{
    __shared__ uint16_t t[TP_TILE][TP_TILE + 2];
    const int pairs_per_leaf = L / (2 * w);
    const int64_t b = blockIdx.z;
    const int64_t lo = (b / pairs_per_leaf) * L;
    const int o1 = 2 * w * (int)(b % pairs_per_leaf), o2 = o1 + w;
    const int k0 = blockIdx.x * TP_TILE, r0 = blockIdx.y * TP_TILE;
    const bool transposed = (mode == 1 || mode == 3);
#pragma unroll 4
    for (int e = threadIdx.x; e < TP_TILE * TP_TILE; e += 256) {
        const int sr = e / TP_TILE, sc = e % TP_TILE;   // source row / column within the tile
        const int i = transposed ? sc : sr, k = transposed ? sr : sc;   // operand row / K
        const int rr = r0 + i, kk = k0 + k;
        uint16_t v;
        if (mode == 0) {
            v = ZN[(lo + o1 + rr) * (int64_t)L + o1 + kk];
        } else if (mode == 2) {
            v = U[(b * w + rr) * (int64_t)w + kk];
        } else if (mode == 1) {
            const int64_t ar = lo + o1 + kk, ac = lo + o2 + rr;
            v = (ar < npiv && ac < npiv) ? A[(rmap ? (int64_t)rmap[ar] : ar) * lda + (cmap ? (int64_t)cmap[ac] : ac)]
                                         : (uint16_t)0;
        } else {
            v = ZN[(lo + o2 + kk) * (int64_t)L + o2 + rr];
        }
        t[i][k] = v;
    }
    __syncthreads();
    for (int it = threadIdx.x; it < TP_TILE * 8; it += 256) {
        const int c = it & 7, i = it >> 3;
        uint32_t a[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) a[e] = t[i][c * 8 + e];
        store_digits8(dst, b * w + r0 + i, k0 + c * 8, a, mp);
    }
}

// Problem tables of the two grouped products of a tensor-core level:
// pu[b]: U rows b w .. (ldc w), pz[b]: ZN rows lo + o1 .. at column o2.
__global__ void pair_probs_kernel(int64_t npairs, int w, int L, const int32_t *__restrict__ iota,
                                  GroupProb *__restrict__ pu, GroupProb *__restrict__ pz)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b > npairs) return;
    const int64_t tiles = (int64_t)(w / 128) * (w / 128);
    GroupProb g{};
    g.tile_off = b * tiles;
    if (b < npairs) {
        const int pairs_per_leaf = L / (2 * w);
        const int64_t lo = (b / pairs_per_leaf) * L;
        const int o1 = 2 * w * (int)(b % pairs_per_leaf);
        g.a_row0 = (int32_t)(b * w);
        g.b_row0 = (int32_t)(b * w);
        g.M = w;
        g.N = w;
        g.c_col0 = 0;
        g.c_rows = iota + b * w;
        pu[b] = g;
        g.c_col0 = o1 + w;
        g.c_rows = iota + lo + o1;
        pz[b] = g;
    } else {
        pu[b] = g;
        pz[b] = g;
    }
}

// Zt row J L + j, column k <- Z_J[k][j]  (tiles of 64 x 64, blockIdx.z = leaf)
__global__ void __launch_bounds__(256) zt_planes_kernel(const uint16_t *__restrict__ ZN, int L, Planes Zt, ModP mp)
{
    __shared__ TpSmem sm;
    const int64_t J = blockIdx.z;
    tp_tile(Zt, J * L, (int64_t)blockIdx.x * TP_TILE, (int64_t)blockIdx.y * TP_TILE, L, L, ZN + J * L * L, L, 0,
            nullptr, mp, sm);
}

constexpr int LEAF_INV_SMEM = 2 * 128 * 129 * (int)sizeof(uint16_t);

// ZN (nleaves L x L, allocated by the caller) <- the block inverses Z_J.
// With use_tc the levels w >= 256 run as grouped tensor-core products
// (err: the device status word of those products).
static int block_inverses(const uint16_t *A, int64_t lda, const int32_t *rmap, const int32_t *cmap, int64_t n, int L,
                          uint16_t *ZN, const ModP &mp, bool use_tc, uint32_t *err, cudaStream_t s)
{
    if (L < 128 || L % 128 || (L & (L - 1)) != 0) return GBLA_E_INTERNAL;
    const int64_t nleaves = (n + L - 1) / L;
    static const cudaError_t attr_rc =
        cudaFuncSetAttribute(upper_inverse128_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, LEAF_INV_SMEM);
    GBLA_CUDA_TRY(attr_rc);
    use_tc = use_tc && L >= 512 && mp.p >= 8 && tc_supported();
    uint16_t *T1 = nullptr;
    int32_t *iota = nullptr;
    GroupProb *probs = nullptr;
    Planes Ap{}, Bp{};
    const int64_t level_rows = nleaves * L / 2;   // rows of a level's operands, all pairs
    int rc = dalloc_t(&T1, (size_t)nleaves * L * L / 4 + 1, s);
    if (rc == GBLA_OK && cudaMemsetAsync(ZN, 0, sizeof(uint16_t) * (size_t)nleaves * L * L, s) != cudaSuccess)
        rc = GBLA_E_CUDA;
    if (rc == GBLA_OK && use_tc) {
        const int64_t max_pairs = nleaves * (L / 512);   // at w = 256
        rc = dalloc_t(&iota, (size_t)(nleaves * L), s);
        if (rc == GBLA_OK) rc = dalloc_t(&probs, (size_t)(2 * (max_pairs + 1)), s);
        if (rc == GBLA_OK) rc = planes_alloc(&Ap, level_rows, L / 2, 2, s);
        if (rc == GBLA_OK) rc = planes_alloc(&Bp, level_rows, L / 2, 4, s);
        if (rc == GBLA_OK) {
            iota_kernel<<<(unsigned)((nleaves * L + 255) / 256), 256, 0, s>>>(iota, nleaves * L);
            if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
        }
    }
    if (rc == GBLA_OK) {
        upper_inverse128_kernel<<<(unsigned)((n + 127) / 128), 128, LEAF_INV_SMEM, s>>>(A, lda, rmap, cmap, n, L, ZN,
                                                                                        mp);
        if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
    }
    for (int w = 128; rc == GBLA_OK && w < L; w *= 2) {
        const int64_t npairs = nleaves * (L / (2 * w));
        if (use_tc && w >= 256) {
            const Planes Aw{Ap.ptr, npairs * w, w, 2}, Bw{Bp.ptr, npairs * w, w, 4};
            GroupProb *pu = probs, *pz = probs + (npairs + 1);
            const dim3 g((unsigned)(w / TP_TILE), (unsigned)(w / TP_TILE), (unsigned)npairs);
            pair_probs_kernel<<<(unsigned)((npairs + 1 + 255) / 256), 256, 0, s>>>(npairs, w, L, iota, pu, pz);
            if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
            if (rc == GBLA_OK) {
                pair_planes_kernel<<<g, 256, 0, s>>>(0, w, L, A, lda, rmap, cmap, n, ZN, T1, Aw, mp);
                if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
            }
            if (rc == GBLA_OK) {
                pair_planes_kernel<<<g, 256, 0, s>>>(1, w, L, A, lda, rmap, cmap, n, ZN, T1, Bw, mp);
                if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
            }
            if (rc == GBLA_OK &&
                cudaMemsetAsync(T1, 0, sizeof(uint16_t) * (size_t)(npairs * w) * (size_t)w, s) != cudaSuccess)
                rc = GBLA_E_CUDA;
            if (rc == GBLA_OK)
                rc = modgemm_grouped(Aw, Bw, pu, (int)npairs, w, T1, w, +1, mp, GBLA_GEMM_TCGEN05, err, s, nullptr);
            if (rc == GBLA_OK) {
                pair_planes_kernel<<<g, 256, 0, s>>>(2, w, L, A, lda, rmap, cmap, n, ZN, T1, Aw, mp);
                if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
            }
            if (rc == GBLA_OK) {
                pair_planes_kernel<<<g, 256, 0, s>>>(3, w, L, A, lda, rmap, cmap, n, ZN, T1, Bw, mp);
                if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
            }
            if (rc == GBLA_OK)
                rc = modgemm_grouped(Aw, Bw, pz, (int)npairs, w, ZN, L, -1, mp, GBLA_GEMM_TCGEN05, err, s, nullptr);
            continue;
        }
        const dim3 grid((unsigned)(w / 64), (unsigned)(w / 64), (unsigned)npairs);
        tri_combine_kernel<<<grid, 256, 0, s>>>(0, w, L, A, lda, rmap, cmap, n, ZN, T1, mp);
        if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
        if (rc != GBLA_OK) break;
        tri_combine_kernel<<<grid, 256, 0, s>>>(1, w, L, A, lda, rmap, cmap, n, ZN, T1, mp);
        if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
    }
    planes_free(&Ap, s);
    planes_free(&Bp, s);
    dfree(probs, s);
    dfree(iota, s);
    dfree(T1, s);
    return rc;
}

int upper_leaf_inverses(const uint16_t *A16, int64_t lda, int64_t npiv, int L, const Planes &Zt, const ModP &mp,
                        uint32_t *err, cudaStream_t s, const Planes *Zr)
{
    if (npiv <= 0) return GBLA_OK;
    const int64_t nleaves = (npiv + L - 1) / L;
    if (Zt.nplanes != 4 || Zt.kp != L || Zt.rows < nleaves * L) return GBLA_E_INTERNAL;
    uint16_t *ZN = nullptr;
    int rc = dalloc_t(&ZN, (size_t)nleaves * L * L, s);
    if (rc == GBLA_OK) rc = block_inverses(A16, lda, nullptr, nullptr, npiv, L, ZN, mp, true, err, s);
    if (rc == GBLA_OK) {
        zt_planes_kernel<<<dim3((unsigned)(L / TP_TILE), (unsigned)(L / TP_TILE), (unsigned)nleaves), 256, 0, s>>>(
            ZN, L, Zt, mp);
        if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
    }
    // ZN is nleaves L x L row-major: as an (nleaves L) x L matrix its rows are Zr's
    if (rc == GBLA_OK && Zr) rc = to_planes(*Zr, nleaves * L, L, ZN, L, 0, false, nullptr, nullptr, mp, s);
    dfree(ZN, s);
    return rc;
}

// cmap[j] = j % L: column map of the diagonal-block storage Adiag.
__global__ void iota_mod_kernel(int32_t *v, int64_t n, int L)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (int32_t)(i % L);
}

int upper_leaf_inverses_diag(const uint16_t *Adiag, int64_t npiv, int L, const Planes &Zt, const ModP &mp,
                             uint32_t *err, cudaStream_t s, const Planes *Zr)
{
    if (npiv <= 0) return GBLA_OK;
    const int64_t nleaves = (npiv + L - 1) / L;
    if (Zt.nplanes != 4 || Zt.kp != L || Zt.rows < nleaves * L) return GBLA_E_INTERNAL;
    uint16_t *ZN = nullptr;
    int32_t *cmap = nullptr;
    int rc = dalloc_t(&ZN, (size_t)nleaves * L * L, s);
    if (rc == GBLA_OK) rc = dalloc_t(&cmap, (size_t)npiv, s);
    if (rc == GBLA_OK) {
        iota_mod_kernel<<<(unsigned)((npiv + 255) / 256), 256, 0, s>>>(cmap, npiv, L);
        if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
    }
    // T[i][j] = Adiag[i * L + j % L]: row i, column j of A inside i's block
    if (rc == GBLA_OK) rc = block_inverses(Adiag, L, nullptr, cmap, npiv, L, ZN, mp, true, err, s);
    if (rc == GBLA_OK) {
        zt_planes_kernel<<<dim3((unsigned)(L / TP_TILE), (unsigned)(L / TP_TILE), (unsigned)nleaves), 256, 0, s>>>(
            ZN, L, Zt, mp);
        if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
    }
    if (rc == GBLA_OK && Zr) rc = to_planes(*Zr, nleaves * L, L, ZN, L, 0, false, nullptr, nullptr, mp, s);
    dfree(cmap, s);
    dfree(ZN, s);
    return rc;
}

int trsm_sparse(const TrsmSparse &T)
{
    const int64_t L = T.L;
    if (T.npiv <= 0 || T.mrows <= 0) return GBLA_OK;
    if (L % 128 || T.Ct->nplanes != 4 || T.Ct->kp < L || T.Zt->kp != L) return GBLA_E_INTERNAL;
    const auto rows_before = [&](int64_t bound) -> int64_t {
        if (!T.lead_host) return T.mrows;
        const auto &ld = *T.lead_host;
        return std::lower_bound(ld.begin(), ld.end(), (int32_t)bound) - ld.begin();
    };
    for (int64_t lo = 0; lo < T.npiv; lo += L) {
        const int64_t hi = std::min(lo + L, T.npiv), w = hi - lo;
        const int64_t rows_hi = rows_before(hi);   // rows with X_J != 0 possible
        if (rows_hi == 0) continue;
        const int64_t rows_lo = rows_before(lo);   // rows with X_{<J} != 0 possible
        // C_J -= X_{<J} * A_{<J,J}: the lists of J's column tiles hold only rows
        // of earlier leaves
        if (rows_lo > 0)
            GBLA_TRY(modgemm_gather(*T.SA, lo / 128, *T.XT, T.npiv, T.C16 + lo, T.ldc, rows_lo, w, -1, T.lead_dev,
                                    *T.mp, T.err, T.s, T.ctr));
        // X_J^T = Z_J^T * C_J^T: A-operand = the inverse's planes (row j, K k
        // = Z_J[k][j]), B-operand = C_J (row r, K k), out = XT rows lo..hi
        GBLA_TRY(to_planes(*T.Ct, rows_hi, w, T.C16 + lo, T.ldc, 0, false, nullptr, nullptr, *T.mp, T.s));
        GBLA_TRY(modgemm_to_planes(*T.Zt, lo, *T.Ct, 0, *T.XT, 0, w, rows_hi, w, *T.mp, T.err, T.s, T.ctr, lo));
    }
    return GBLA_OK;
}

// Nm = I - Z elementwise (u16, n_total elements of L x L blocks).
__global__ void i_minus_kernel(uint16_t *__restrict__ Z, int L, int64_t total, uint32_t p)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int64_t i = (e / L) % L, j = e % L;
    const uint32_t z = Z[e];
    const uint32_t v = (i == j ? 1u : 0u) + p - z;
    Z[e] = (uint16_t)(v >= p ? v - p : v);
}



// Column map of the echelon rows: colmap[c] = index of c among the non-pivot
// columns, or -(j + 1) if c = pcol[j]; npc[i] = i-th non-pivot column.  pcol
// is ascending, so the pivots left of c are found by binary search.
__global__ void colmap_np_kernel(const int32_t *__restrict__ pcol, int64_t rank, int64_t n, int32_t *__restrict__ colmap,
                                 int32_t *__restrict__ npc)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    int64_t lo = 0, hi = rank;   // first j with pcol[j] >= c
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (pcol[mid] < c) lo = mid + 1;
        else hi = mid;
    }
    if (lo < rank && pcol[lo] == c) {
        colmap[c] = -(int32_t)(lo + 1);
    } else {
        colmap[c] = (int32_t)(c - lo);
        npc[c - lo] = (int32_t)c;
    }
}

// Rnp[k][i] = D[rows[k]][npc[i]]: the echelon rows at the non-pivot columns.
// A thread owns 8 consecutive outputs of a row (one 16-byte store; ldnp is a
// multiple of 64, so rows start 128-byte aligned) and keeps their column
// indices in registers for all the rows its block visits.
__global__ void gather_np_kernel(const uint16_t *__restrict__ D, int64_t ldd, const int32_t *__restrict__ rows,
                                 int64_t nrows, const int32_t *__restrict__ npc, int64_t nnp, uint16_t *__restrict__ Rnp,
                                 int64_t ldnp)
{
    for (int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 8; i0 < nnp;
         i0 += (int64_t)gridDim.x * blockDim.x * 8) {
        int32_t col[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) col[e] = (i0 + e < nnp) ? npc[i0 + e] : -1;
        for (int64_t k = blockIdx.y; k < nrows; k += gridDim.y) {
            const uint16_t *src = D + (int64_t)rows[k] * ldd;
            uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (col[e] >= 0) w[e >> 1] |= (uint32_t)src[col[e]] << ((e & 1) * 16);
            if (i0 + 8 <= ldnp) *reinterpret_cast<uint4 *>(Rnp + k * ldnp + i0) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// RREF rows in full: R[k][c] = Rnp[k][colmap[c]] at non-pivot columns, the
// unit vector at the pivot columns (R[k][pcol[j]] = [j == k]).  8 columns per
// thread, one 16-byte store (ldr is a multiple of 64); the column map of a
// thread's 8 columns stays in registers for all the rows its block visits.
__global__ void expand_rref_kernel(const uint16_t *__restrict__ Rnp, int64_t ldnp, const int32_t *__restrict__ colmap,
                                   int64_t nrows, int64_t n, uint16_t *__restrict__ R, int64_t ldr)
{
    for (int64_t c0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 8; c0 < n;
         c0 += (int64_t)gridDim.x * blockDim.x * 8) {
        int32_t m[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) m[e] = (c0 + e < n) ? colmap[c0 + e] : INT32_MIN;
        for (int64_t k = blockIdx.y; k < nrows; k += gridDim.y) {
            const uint16_t *src = Rnp + k * ldnp;
            uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                uint32_t v = 0;
                if (m[e] >= 0) v = src[m[e]];
                else if (m[e] != INT32_MIN && (int64_t)(-m[e] - 1) == k) v = 1u;
                w[e >> 1] |= v << ((e & 1) * 16);
            }
            if (c0 + 8 <= ldr) *reinterpret_cast<uint4 *>(R + k * ldr + c0) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// Rnp <- T^-1 Rnp for the rows [lo, hi), where Rnp holds the echelon rows at
// the non-pivot columns only (the pivot columns of the reduced form are the
// unit vectors, nothing to compute) and T = the echelon rows at the pivot
// columns (unit upper triangular; read from D through the row map, never
// modified: the updates below only touch non-pivot columns).  By halving: the
// lower half first, then its product into the upper half, then the upper
// half.  RT holds the B-operand planes of Rnp^T (row = non-pivot column, K =
// row); a 128-row block is written there before its leaf product (which reads
// the block itself) and again once final, so the products of the internal
// nodes read final rows without converting them.  Rows lo.. are zero left of
// pcol[lo], i.e. left of non-pivot column pcol[lo] - lo.
static int backsub_rec(const EchelonD &E, uint16_t *Rnp, int64_t ldnp, int64_t nnp, const int32_t *pcol_dev,
                       const std::vector<int32_t> &pcol, int64_t lo, int64_t hi, Planes &Ap, Planes &RT,
                       const uint16_t *Nm_all, int BL)
{
    const ModP &mp = *E.mp;
    cudaStream_t s = E.s;
    if (hi - lo <= BL) {
        // leaves are the BL-row blocks (splits fall on multiples of BL):
        // Rnp_J <- Rnp_J - (I - T_JJ^-1) Rnp_J
        const int w = (int)(hi - lo);
        const int64_t cs = (pcol[lo] - lo) & ~int64_t(63);
        const uint16_t *Nm = Nm_all + (size_t)(lo / BL) * BL * BL;
        GBLA_TRY(to_planes(Ap, w, w, Nm, BL, 0, false, nullptr, nullptr, mp, s));
        GBLA_TRY(to_planes(RT, nnp, w, Rnp + lo * ldnp, ldnp, 0, true, nullptr, nullptr, mp, s, nullptr, false, lo));
        GBLA_TRY(modgemm(Ap, 0, 0, RT, cs, lo, Rnp + lo * ldnp + cs, ldnp, w, nnp - cs, w, -1, mp, E.variant, E.err,
                         s, E.ctr));
        return to_planes(RT, nnp, w, Rnp + lo * ldnp, ldnp, 0, true, nullptr, nullptr, mp, s, nullptr, false, lo);
    }
    const int64_t mid = lo + round_up((hi - lo) / 2, BL);
    GBLA_TRY(backsub_rec(E, Rnp, ldnp, nnp, pcol_dev, pcol, mid, hi, Ap, RT, Nm_all, BL));
    // Rnp[lo:mid] -= T[lo:mid, mid:hi] * Rnp[mid:hi]
    const int64_t cs = (pcol[mid] - mid) & ~int64_t(63);
    GBLA_TRY(to_planes(Ap, mid - lo, hi - mid, E.D16, E.ldd, 0, false, E.prow + lo, pcol_dev + mid, mp, s));
    GBLA_TRY(modgemm(Ap, 0, 0, RT, cs, mid, Rnp + lo * ldnp + cs, ldnp, mid - lo, nnp - cs, hi - mid, -1, mp,
                     E.variant, E.err, s, E.ctr));
    return backsub_rec(E, Rnp, ldnp, nnp, pcol_dev, pcol, lo, mid, Ap, RT, Nm_all, BL);
}

// Apply the panel bases of jobs [job0, job0 + njobs) (slots given by
// job_slot or equal to the job index): D[S] <- G * D[S], then clear the other
// candidates on their panel and find their new leads.
struct PanelWork {
    int32_t *t_slot, *S_slot, *pc_slot, *wave_slot;
    uint16_t *Gm_all;
    int32_t *lead;
    PanelPlan *plan_dev;
    GroupProb *probs;
    Planes Gp, Bs, H, GmT;
    uint16_t *H16;    // multipliers H = D[cand, pc], then H G (rows as in H)
    int32_t *iota;    // 0, 1, 2, .. (row maps of the H G products)
    // fused application (tensor cores): job table, stacked A blocks, row maps
    PaJob *pajobs;
    Planes Apa;
    int32_t *rowmap;
    bool fused;
};

static int apply_panels(const EchelonD &E, PanelWork &W, const std::vector<PanelPlan> &plan, const int64_t *seg,
                        const int32_t *cand, const int32_t *job_slot, int job0, int64_t row_base, int64_t rows_max)
{
    const ModP &mp = *E.mp;
    cudaStream_t s = E.s;
    const int nj = (int)plan.size();
    if (nj == 0) return GBLA_OK;
    int64_t ncmax = 0;
    for (const auto &pl : plan) ncmax = pl.nc > ncmax ? pl.nc : ncmax;
    GBLA_CUDA_TRY(cudaMemcpyAsync(W.plan_dev, plan.data(), sizeof(PanelPlan) * (size_t)nj, cudaMemcpyHostToDevice, s));
    if (W.fused) {
        // H = D[cand, pc], then H G = H + H (G - I) (grouped product), then
        // both updates of every job in one fused launch that reads D[S] once
        const unsigned rb = (unsigned)(rows_max < 64 ? (rows_max > 0 ? rows_max : 1) : 64);
        gather_h_planes_kernel<<<dim3(rb, (unsigned)nj), PANEL, 0, s>>>(
            W.H, W.H16, E.D16, E.ldd, seg, cand, job_slot, job0, row_base, W.pc_slot, W.t_slot, E.is_piv_row, mp.p);
        GBLA_CUDA_TRY(launch_check());
        gather_gmt_planes_kernel<<<dim3(PANEL, (unsigned)nj), PANEL, 0, s>>>(W.GmT, W.Gm_all, W.plan_dev, mp);
        GBLA_CUDA_TRY(launch_check());
        make_probs_kernel<<<1, 256, 0, s>>>(W.probs, nj, 3, W.plan_dev, W.t_slot, W.S_slot, W.wave_slot, seg, cand,
                                           job0, row_base, W.iota);
        GBLA_CUDA_TRY(launch_check());
        GBLA_TRY(modgemm_grouped(W.H, W.GmT, W.probs, nj, PANEL, W.H16, PANEL, +1, mp, E.variant, E.err, s, E.ctr));
        pa_jobs_kernel<<<1, 1024, 0, s>>>(W.pajobs, nj, W.plan_dev, W.t_slot, W.S_slot, W.wave_slot, seg, job0);
        GBLA_CUDA_TRY(launch_check());
        pa_fill_kernel<<<dim3(64, (unsigned)nj), PANEL, 0, s>>>(W.Apa, W.rowmap, W.pajobs, W.plan_dev, W.Gm_all,
                                                              W.H16, seg, cand, E.is_piv_row, job0, row_base,
                                                              mp.p);
        GBLA_CUDA_TRY(launch_check());
        return panel_apply(W.Apa, W.pajobs, nj, W.rowmap, E.D16, E.ldd, E.n, mp, E.err, s);
    }
    // G - I of the jobs' slots as the A operand (rows q * 128 ..), and D[S]^T
    // as the B operand, converted once: both products below read D[S] as it
    // is before the first one updates it.
    gather_gm_planes_kernel<<<dim3(PANEL, (unsigned)nj), PANEL, 0, s>>>(W.Gp, W.Gm_all, W.plan_dev, mp.p);
    GBLA_CUDA_TRY(launch_check());
    dim3 gt((unsigned)(round_up(ncmax, 128) / TP_TILE), PANEL / TP_TILE, (unsigned)nj);
    gather_t_planes_kernel<<<gt, 256, 0, s>>>(W.Bs, E.D16, E.ldd, W.plan_dev, W.S_slot, W.t_slot, mp);
    GBLA_CUDA_TRY(launch_check());
    // H = D[cand, pc] (zero for rows that are pivots now), as planes and u16
    const unsigned rows_blocks = (unsigned)(rows_max < 64 ? (rows_max > 0 ? rows_max : 1) : 64);
    gather_h_planes_kernel<<<dim3(rows_blocks, (unsigned)nj), PANEL, 0, s>>>(
        W.H, W.H16, E.D16, E.ldd, seg, cand, job_slot, job0, row_base, W.pc_slot, W.t_slot, E.is_piv_row, mp.p);
    GBLA_CUDA_TRY(launch_check());
    gather_gmt_planes_kernel<<<dim3(PANEL, (unsigned)nj), PANEL, 0, s>>>(W.GmT, W.Gm_all, W.plan_dev, mp);
    GBLA_CUDA_TRY(launch_check());
    // D[S] += (G - I) * D[S]
    make_probs_kernel<<<1, 256, 0, s>>>(W.probs, nj, 1, W.plan_dev, W.t_slot, W.S_slot, W.wave_slot, seg, cand, job0,
                                       row_base, W.iota);
    GBLA_CUDA_TRY(launch_check());
    GBLA_TRY(modgemm_grouped(W.Gp, W.Bs, W.probs, nj, PANEL, E.D16, E.ldd, +1, mp, E.variant, E.err, s, E.ctr));
    // H G = H + H (G - I), then its planes replace those of H
    make_probs_kernel<<<1, 256, 0, s>>>(W.probs, nj, 3, W.plan_dev, W.t_slot, W.S_slot, W.wave_slot, seg, cand, job0,
                                       row_base, W.iota);
    GBLA_CUDA_TRY(launch_check());
    GBLA_TRY(modgemm_grouped(W.H, W.GmT, W.probs, nj, PANEL, W.H16, PANEL, +1, mp, E.variant, E.err, s, E.ctr));
    GBLA_TRY(to_planes(W.H, W.H.rows, PANEL, W.H16, PANEL, 0, false, nullptr, nullptr, mp, s));
    // D[cand] -= (H G) * D[S]_old  (= H * D[S]_new; pivot rows have zero multipliers)
    make_probs_kernel<<<1, 256, 0, s>>>(W.probs, nj, 2, W.plan_dev, W.t_slot, W.S_slot, W.wave_slot, seg, cand, job0,
                                       row_base, W.iota);
    GBLA_CUDA_TRY(launch_check());
    GBLA_TRY(modgemm_grouped(W.H, W.Bs, W.probs, nj, PANEL, E.D16, E.ldd, -1, mp, E.variant, E.err, s, E.ctr));
    return GBLA_OK;
}

int echelon_d(const EchelonD &E, int64_t *rank_out)
{
    *rank_out = 0;
    const int64_t m = E.m, n = E.n;
    if (m <= 0 || n <= 0) return GBLA_OK;
    cudaStream_t s = E.s;
    const ModP &mp = *E.mp;
    const int64_t npan = (n + PANEL - 1) / PANEL;
    int rc = GBLA_OK;
    int64_t rank = 0;
    PanelWork W{};
    int32_t *cand = nullptr, *fill = nullptr, *info = nullptr, *job_slot = nullptr;
    int64_t *off = nullptr, *seg = nullptr, *rank_dev = nullptr;
    uint16_t *inv_tab = nullptr;
    // Phase B works on chunks of panels whose D[S]^T planes fit this many rows.
    const int64_t BS_ROWS = int64_t(1) << 20;
    static const cudaError_t attr_rc =
        cudaFuncSetAttribute(panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PANEL_SMEM);
    GBLA_CUDA_TRY(attr_rc);
#define ESTEP(expr)                         \
    do {                                    \
        if ((rc = (expr)) != GBLA_OK) goto done; \
    } while (0)
#define ECUDA(expr)                                   \
    do {                                              \
        if ((expr) != cudaSuccess) { rc = GBLA_E_CUDA; goto done; } \
    } while (0)
    if (E.method == 1 || E.method == 2) {
        // sparse SGE (for the automatic choice only on a sparse enough D'); if
        // its pivot pool fills up, the panels finish the job
        double dens = 0.0;
        ESTEP(dprime_density(E, &dens));
        if (E.density) *E.density = dens;
        if (E.method == 1 || dens <= SGE_MAX_DENSITY) {
            bool overflow = false;
            ESTEP(sge_forward(E, dens, &rank, &overflow));
            if (E.sge_completed) *E.sge_completed = overflow ? 0 : 1;
            if (!overflow) goto backward;
        }
    }
    {
        ESTEP(dalloc_t(&W.lead, (size_t)m + 1, s));
        ESTEP(dalloc_t(&cand, (size_t)m + PANEL + 1, s));
        ESTEP(dalloc_t(&fill, (size_t)npan + 1, s));
        ESTEP(dalloc_t(&off, (size_t)npan + 2, s));
        ESTEP(dalloc_t(&info, 4, s));
        ESTEP(dalloc_t(&seg, (size_t)npan + 2, s));
        ESTEP(dalloc_t(&job_slot, (size_t)npan + 1, s));
        ESTEP(dalloc_t(&rank_dev, 2, s));
        ESTEP(dalloc_t(&W.t_slot, (size_t)npan + 1, s));
        ESTEP(dalloc_t(&W.S_slot, (size_t)npan * PANEL, s));
        ESTEP(dalloc_t(&W.pc_slot, (size_t)npan * PANEL, s));
        ESTEP(dalloc_t(&W.wave_slot, (size_t)npan * 2 + 2, s));
        ESTEP(dalloc_t(&W.Gm_all, (size_t)npan * PANEL * PANEL, s));
        ESTEP(dalloc_t(&W.plan_dev, (size_t)npan + 1, s));
        ESTEP(dalloc_t(&W.probs, (size_t)npan + 2, s));
        ESTEP(dalloc_t(&inv_tab, 65536, s));
        W.fused = E.variant != GBLA_GEMM_SIMT && mp.p >= 8 && tc_supported();
        if (!W.fused) {   // the separate products' operands
            ESTEP(planes_alloc(&W.Bs, BS_ROWS + n, PANEL, 4, s));
            ESTEP(planes_alloc(&W.Gp, npan * PANEL, PANEL, 2, s));
        }
        ESTEP(planes_alloc(&W.H, m + PANEL, PANEL, 2, s));
        ESTEP(planes_alloc(&W.GmT, npan * PANEL, PANEL, 4, s));
        ESTEP(dalloc_t(&W.H16, (size_t)W.H.rows * PANEL, s));
        ESTEP(dalloc_t(&W.iota, (size_t)W.H.rows, s));
        if (W.fused) {
            // a chunk's A blocks: at most PANEL rows of G - I per job plus its
            // candidates; the last block's TMA box may read PANEL rows past it
            const int64_t arows = m + (npan + 2) * PANEL;
            ESTEP(dalloc_t(&W.pajobs, (size_t)npan + 2, s));
            ESTEP(planes_alloc(&W.Apa, arows, PANEL, 2, s));
            ECUDA(cudaMemsetAsync(W.Apa.ptr, 0, W.Apa.plane_elems() * (size_t)W.Apa.nplanes * sizeof(__nv_bfloat16), s));
            ESTEP(dalloc_t(&W.rowmap, (size_t)arows, s));
        }
        iota_kernel<<<(unsigned)((W.H.rows + 255) / 256), 256, 0, s>>>(W.iota, W.H.rows);
        ECUDA(launch_check());
        ECUDA(cudaMemsetAsync(E.is_piv_row, 0, sizeof(int32_t) * (size_t)m, s));
        ECUDA(cudaMemsetAsync(W.t_slot, 0, sizeof(int32_t) * (size_t)(npan + 1), s));
        inverse_table_kernel<<<(mp.p + 255) / 256, 256, 0, s>>>(inv_tab, mp);
        ECUDA(launch_check());
        // ---- leads of all rows
        row_leads_kernel<<<(unsigned)((m * 32 + 255) / 256), 256, 0, s>>>(E.D16, E.ldd, n, m, nullptr, nullptr, 0,
                                                                         nullptr, W.lead);
        ECUDA(launch_check());
        // ---- waves: every panel with candidates (non-pivot rows leading in
        // it) is processed at once; rows that were dependent on their panel
        // move right and are candidates of the next wave.  Leads only grow,
        // so there are at most npan waves.
        std::vector<int32_t> slots_h((size_t)npan + 1);
        std::vector<int64_t> seg_h((size_t)npan + 2);
        for (int64_t wave = 0;; ++wave) {
            if (wave > npan) { rc = GBLA_E_INTERNAL; goto done; }
            ECUDA(cudaMemsetAsync(fill, 0, sizeof(int32_t) * (size_t)(npan + 1), s));
            ECUDA(cudaMemsetAsync(off, 0, sizeof(int64_t) * (size_t)(npan + 2), s));
            panel_count_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(m, W.lead, E.is_piv_row, off);
            ECUDA(launch_check());
            ESTEP(scan_i64(off, off, npan + 1, nullptr, s));
            panel_scatter_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(m, W.lead, E.is_piv_row, off, fill,
                                                                             cand);
            ECUDA(launch_check());
            panel_sort_kernel<<<(unsigned)npan, 256, 0, s>>>(npan, off, cand);
            ECUDA(launch_check());
            make_jobs_kernel<<<1, 1024, 0, s>>>(npan, off, job_slot, seg, info);
            ECUDA(launch_check());
            int32_t njobs = 0;
            ESTEP(readback(&njobs, info, sizeof(int32_t), s));
            if (njobs == 0) break;
            ESTEP(readback(slots_h.data(), job_slot, sizeof(int32_t) * (size_t)njobs, s));
            ESTEP(readback(seg_h.data(), seg, sizeof(int64_t) * (size_t)(njobs + 1), s));
            panel_kernel<<<(unsigned)njobs, 2 * PANEL, PANEL_SMEM, s>>>(E.D16, E.ldd, n, seg, cand, job_slot, inv_tab,
                                                                      E.is_piv_row, W.t_slot, W.S_slot, W.pc_slot,
                                                                      W.Gm_all, W.wave_slot, mp);
            ECUDA(launch_check());
            ECUDA(cudaStreamSynchronize(s));
            // apply the new bases, chunk by chunk of jobs (grouped products)
            for (int j0 = 0; j0 < njobs;) {
                std::vector<PanelPlan> plan;
                int64_t boff = 0;
                int j1 = j0;
                while (j1 < njobs) {
                    const int32_t nc = (int32_t)(n - (int64_t)slots_h[(size_t)j1] * PANEL);
                    if (!plan.empty() && boff + round_up(nc, 128) > BS_ROWS) break;
                    plan.push_back(PanelPlan{boff, slots_h[(size_t)j1], nc});
                    boff += round_up(nc, 128);
                    ++j1;
                }
                const int64_t rows = seg_h[(size_t)j1] - seg_h[(size_t)j0];
                ESTEP(apply_panels(E, W, plan, seg, cand, job_slot, j0, seg_h[(size_t)j0], rows));
                j0 = j1;
            }
            // the candidates that did not become pivots lead right of their panel now
            const int64_t ncand = seg_h[(size_t)njobs];
            row_leads_kernel<<<(unsigned)((ncand * 32 + 255) / 256), 256, 0, s>>>(E.D16, E.ldd, n, ncand, cand,
                                                                                  nullptr, -1, E.is_piv_row, W.lead);
            ECUDA(launch_check());
        }
        compact_slots_kernel<<<1, 1024, 0, s>>>(npan, W.t_slot, W.S_slot, W.pc_slot, E.prow, E.pcol, rank_dev);
        ECUDA(launch_check());
        ESTEP(readback(&rank, rank_dev, sizeof(int64_t), s));
    }
    // ---- backward pass: RREF rows into R (pivot column order)
backward:
    if (E.back_start) cudaEventRecord(E.back_start, s);
    if (rank > 0) {
        const int64_t ldr = E.ldd;
        const int64_t nnp = n - rank;
        const int64_t ldnp = round_up(nnp > 0 ? nnp : 1, 64);
        std::vector<int32_t> pcol_h((size_t)rank);
        uint16_t *Nm = nullptr, *Rnp = nullptr;
        int32_t *colmap = nullptr, *npc = nullptr;
        Planes Ap{}, Bp{};
        if (!E.np_out) rc = dalloc_t(&E.R[0], (size_t)rank * (size_t)ldr, s);
        if (rc == GBLA_OK) rc = dalloc_t(&colmap, (size_t)n, s);
        if (rc == GBLA_OK) rc = dalloc_t(&npc, (size_t)(nnp > 0 ? nnp : 1), s);
        if (rc == GBLA_OK) rc = dalloc_t(&Rnp, (size_t)rank * (size_t)ldnp, s);
        if (rc == GBLA_OK) rc = readback(pcol_h.data(), E.pcol, sizeof(int32_t) * (size_t)rank, s);
        if (rc == GBLA_OK) {
            colmap_np_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(E.pcol, rank, n, colmap, npc);
            if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
        }
        const int64_t xb = (n + 8 * 256 - 1) / (8 * 256);
        const dim3 rgrid((unsigned)(xb < 64 ? xb : 64), (unsigned)(rank < 1024 ? rank : 1024));
        if (rc == GBLA_OK && nnp > 0) {
            gather_np_kernel<<<rgrid, 256, 0, s>>>(E.D16, E.ldd, E.prow, rank, npc, nnp, Rnp, ldnp);
            if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
        }
        if (rc == GBLA_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = GBLA_E_CUDA;
        // leaves of BL rows: the inverses of T's diagonal BL-blocks in one go
        const int BL = E.back_leaf > 0 ? E.back_leaf : PANEL;
        const int64_t nleaves = (rank + BL - 1) / BL;
        if (rc == GBLA_OK && nnp > 0) rc = dalloc_t(&Nm, (size_t)nleaves * BL * BL, s);
        if (rc == GBLA_OK && nnp > 0)
            rc = block_inverses(E.D16, E.ldd, E.prow, E.pcol, rank, BL, Nm, mp, E.variant != GBLA_GEMM_SIMT, E.err, s);
        if (rc == GBLA_OK && nnp > 0) {
            const int64_t total = nleaves * BL * BL;
            i_minus_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(Nm, BL, total, mp.p);
            if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
        }
        if (rc == GBLA_OK && nnp > 0) rc = planes_alloc(&Ap, rank, rank, 2, s);   // K up to a leaf or half the rows
        if (rc == GBLA_OK && nnp > 0) rc = planes_alloc(&Bp, nnp, rank, 4, s);   // Rnp^T
        if (rc == GBLA_OK && nnp > 0) rc = backsub_rec(E, Rnp, ldnp, nnp, E.pcol, pcol_h, 0, rank, Ap, Bp, Nm, BL);
        if (rc == GBLA_OK && E.np_out) {
            // hand the non-pivot part over instead of the dense rows
            E.np_out->Rnp = Rnp;
            E.np_out->ldnp = ldnp;
            E.np_out->npc = npc;
            E.np_out->nnp = nnp;
            Rnp = nullptr;
            npc = nullptr;
        } else if (rc == GBLA_OK) {
            expand_rref_kernel<<<rgrid, 256, 0, s>>>(Rnp, ldnp, colmap, rank, n, E.R[0], ldr);
            if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
        }
        dfree(Nm, s);
        dfree(Rnp, s);
        dfree(colmap, s);
        dfree(npc, s);
        planes_free(&Ap, s);
        planes_free(&Bp, s);
    }
done:
#undef ESTEP
#undef ECUDA
    dfree(W.lead, s);
    dfree(cand, s);
    dfree(fill, s);
    dfree(off, s);
    dfree(info, s);
    dfree(seg, s);
    dfree(job_slot, s);
    dfree(rank_dev, s);
    dfree(W.t_slot, s);
    dfree(W.S_slot, s);
    dfree(W.pc_slot, s);
    dfree(W.wave_slot, s);
    dfree(W.Gm_all, s);
    dfree(W.plan_dev, s);
    dfree(W.probs, s);
    dfree(inv_tab, s);
    planes_free(&W.Bs, s);
    planes_free(&W.Gp, s);
    planes_free(&W.H, s);
    planes_free(&W.GmT, s);
    dfree(W.H16, s);
    dfree(W.iota, s);
    dfree(W.pajobs, s);
    planes_free(&W.Apa, s);
    dfree(W.rowmap, s);
    *rank_out = rank;
    return rc;
}

}  // namespace gbla
