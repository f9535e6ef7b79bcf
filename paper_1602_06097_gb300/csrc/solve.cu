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

namespace gbla {

constexpr int LEAF = 128;

// ------------------------------------------------------------ upper leaf
// X_J * A_JJ = C_J for the column block J = [j0, j0 + W), all rows, where C_J
// already holds C_J - X_{<J} * A_{<J,J}.  X_J overwrites C_J (uint16) and is
// written to the A-operand digit planes Xp.
__global__ void __launch_bounds__(256) trsm_upper_leaf_kernel(int64_t mrows, int64_t npiv, int64_t j0, int W,
                                                              const int64_t *__restrict__ mlptr,
                                                              const int32_t *__restrict__ mlpos,
                                                              const uint32_t *__restrict__ mlval, uint16_t *C16,
                                                              int64_t ldc, Planes Xp, ModP mp)
{
    __shared__ unsigned long long acc_s[8][2][LEAF];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t pair = (int64_t)blockIdx.x * 8 + warp;
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
        const int64_t q = (j0 + jl) >> 1;
        const int64_t e0 = mlptr[q], e1 = mlptr[q + 1];
        const bool has_b = jl + 1 < W;
        uint32_t a01 = 0;
        bool first_is_coupling = false;
        if (e0 < e1 && mlpos[e0] == j0 + jl + 1) {
            a01 = mlval[e0] & 0xFFFFu;
            first_is_coupling = true;
        }
        // multipliers: lambda for row j (x?a) and row j+1 (x?b), both C rows
        const uint32_t x1a = mod64(acc[0][jl], mp), x2a = mod64(acc[1][jl], mp);
        uint32_t x1b = 0, x2b = 0;
        if (has_b) {
            x1b = mod64(acc[0][jl + 1] + (P - x1a) * a01, mp);
            x2b = mod64(acc[1][jl + 1] + (P - x2a) * a01, mp);
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
        const int64_t lim = j0 + W;
        for (int64_t e = e0 + (first_is_coupling ? 1 : 0) + lane; e < e1; e += 32) {
            const int64_t k = mlpos[e];
            if (k >= lim) break;
            const uint32_t v = mlval[e];
            const uint64_t v1 = v & 0xFFFFu, v2 = v >> 16;
            const int kl = (int)(k - j0);
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

static int trsm_upper_rec(const TrsmUpper &T, int64_t lo, int64_t hi)
{
    if (hi - lo <= LEAF) {
        const int64_t pairs = (T.mrows + 1) / 2;
        trsm_upper_leaf_kernel<<<(unsigned)((pairs + 7) / 8), 256, 0, T.s>>>(
            T.mrows, T.npiv, lo, (int)(hi - lo), T.ml->ptr, T.ml->pos, T.ml->val, T.C16, T.ldc, *T.Xp, *T.mp);
        GBLA_CUDA_TRY(cudaGetLastError());
        return GBLA_OK;
    }
    const int64_t mid = lo + round_up((hi - lo) / 2, LEAF);
    GBLA_TRY(trsm_upper_rec(T, lo, mid));
    // C[:, mid:hi] -= X[:, lo:mid] * A[lo:mid, mid:hi]   (A^T planes: row = column of A)
    GBLA_TRY(modgemm(*T.Xp, 0, lo, *T.At, mid, lo, T.C16 + mid, T.ldc, T.mrows, hi - mid, mid - lo, -1, *T.mp,
                     T.variant, T.err, T.s, T.ctr));
    return trsm_upper_rec(T, mid, hi);
}

int trsm_upper(const TrsmUpper &T)
{
    if (T.mrows <= 0 || T.npiv <= 0) return GBLA_OK;
    return trsm_upper_rec(T, 0, T.npiv);
}

// ------------------------------------------------------------ lower leaf
// X'_J * A'_JJ = C'_J with A' = A^T (lower unit triangular): for j descending,
// x'_j = c'_j - sum_{k > j} A[j][k] x'_k.  One warp per pair of C' rows; each
// pivot pair (j, j+1) contributes two dot products with its multiline.
__global__ void __launch_bounds__(256) trsm_lower_leaf_kernel(int64_t mrows, int64_t npiv, int64_t j0, int W,
                                                              const int64_t *__restrict__ mlptr,
                                                              const int32_t *__restrict__ mlpos,
                                                              const uint32_t *__restrict__ mlval, uint16_t *C16,
                                                              int64_t ldc, Planes Xp, ModP mp)
{
    __shared__ uint32_t xs_s[8][2][LEAF];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t pair = (int64_t)blockIdx.x * 8 + warp;
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
    const int64_t lim = j0 + W;
    const int start = ((W - 1) & ~1);   // local index of the last pair's first column
    for (int jl = start; jl >= 0; jl -= 2) {
        const int64_t q = (j0 + jl) >> 1;
        const int64_t e0 = mlptr[q], e1 = mlptr[q + 1];
        const bool has_b = jl + 1 < W;
        uint32_t a01 = 0;
        bool first_is_coupling = false;
        if (e0 < e1 && mlpos[e0] == j0 + jl + 1) {
            a01 = mlval[e0] & 0xFFFFu;
            first_is_coupling = true;
        }
        unsigned long long d1r1 = 0, d2r1 = 0, d1r2 = 0, d2r2 = 0;  // d1: A row j, d2: A row j+1
        for (int64_t e = e0 + (first_is_coupling ? 1 : 0) + lane; e < e1; e += 32) {
            const int64_t k = mlpos[e];
            if (k >= lim) break;
            const uint32_t v = mlval[e];
            const uint64_t v1 = v & 0xFFFFu, v2 = v >> 16;
            const int kl = (int)(k - j0);
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
            const uint32_t s2r1 = mod64(d2r1, mp), s2r2 = mod64(d2r2, mp);
            uint32_t xb1 = 0, xb2 = 0;
            if (has_b) {
                xb1 = mod64((uint64_t)xs[0][jl + 1] + P - s2r1, mp);
                xb2 = mod64((uint64_t)xs[1][jl + 1] + P - s2r2, mp);
                xs[0][jl + 1] = xb1;
                xs[1][jl + 1] = xb2;
            }
            const uint64_t t1 = (uint64_t)mod64(d1r1, mp) + (uint64_t)a01 * xb1;
            const uint64_t t2 = (uint64_t)mod64(d1r2, mp) + (uint64_t)a01 * xb2;
            xs[0][jl] = mod64((uint64_t)xs[0][jl] + P * P - mod64(t1, mp), mp);
            xs[1][jl] = mod64((uint64_t)xs[1][jl] + P * P - mod64(t2, mp), mp);
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

static int trsm_lower_rec(const TrsmLower &T, int64_t lo, int64_t hi)
{
    if (hi - lo <= LEAF) {
        const int64_t pairs = (T.mrows + 1) / 2;
        trsm_lower_leaf_kernel<<<(unsigned)((pairs + 7) / 8), 256, 0, T.s>>>(
            T.mrows, T.npiv, lo, (int)(hi - lo), T.ml->ptr, T.ml->pos, T.ml->val, T.C16, T.ldc, *T.Xp, *T.mp);
        GBLA_CUDA_TRY(cudaGetLastError());
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
    return trsm_lower_rec(T, 0, T.npiv);
}

// ================================================================ echelon
// Blocked Gauss-Jordan of D over column panels of width <= 128.
//
// Panel step (one CTA): the rows that are not yet pivots are taken in order;
// each is reduced by the panel basis found so far (kept in reduced echelon
// form over the panel's columns) and, if something is left, becomes a new
// basis row (normalised at its leftmost nonzero, the other basis rows cleared
// at that column).  This is Alg. 3's "normalise, reduce by matching heads",
// restricted to the panel.  Each candidate carries the coefficients that
// express it in the chosen rows S, so at the end G satisfies
// G * D[S, panel] = U, U in reduced echelon form with pivot columns pc.
// The trailing update then applies, to every row outside S (earlier pivot
// rows included, which is what makes the result reduced):
//   row[c0:] <- row[c0:] - row[pc] * W,   W = G * D[S, c0:],
// and the rows S receive W.  Both products run on the tensor cores.
constexpr int PANEL = 128;

__global__ void __launch_bounds__(256) panel_kernel(const uint16_t *__restrict__ D, int64_t ldd, int64_t m, int64_t c0,
                                                    int bw, const int32_t *__restrict__ is_piv_row,
                                                    int32_t *__restrict__ t_out, int32_t *__restrict__ S_out,
                                                    int32_t *__restrict__ pc_out, uint16_t *__restrict__ G_out,
                                                    ModP mp)
{
    extern __shared__ uint32_t smem_u32[];
    uint32_t(*aug)[2 * PANEL] = reinterpret_cast<uint32_t(*)[2 * PANEL]>(smem_u32);  // [PANEL][256]
    __shared__ uint32_t cand[2 * PANEL];
    __shared__ uint32_t fk[PANEL];
    __shared__ int bcol[PANEL], S[PANEL], rnk[PANEL];
    __shared__ int cstar;
    __shared__ uint32_t inv_s;
    const int c = threadIdx.x;  // column of the augmented row: [panel | coefficients]
    const uint64_t P = mp.p;
    int t = 0;
    for (int64_t i = 0; i < m && t < bw; ++i) {
        if (is_piv_row[i]) continue;
        const uint32_t v = (c < bw) ? D[i * ldd + c0 + c] : ((c >= PANEL && c - PANEL == t) ? 1u : 0u);
        if (!__syncthreads_or(c < bw && v != 0)) continue;
        cand[c] = v;
        __syncthreads();
        // reduce by the basis (reduced echelon: coefficient = entry at its pivot)
        unsigned long long a = v;
        for (int k = 0; k < t; ++k) {
            const uint64_t coef = cand[bcol[k]];
            a += (P - coef) * aug[k][c];
        }
        const uint32_t nv = mod64(a, mp);
        __syncthreads();
        cand[c] = nv;
        if (c == 0) cstar = 1 << 30;
        __syncthreads();
        if (c < bw && nv != 0) atomicMin(&cstar, c);
        __syncthreads();
        const int cs = cstar;
        if (cs >= bw) continue;           // dependent on the rows taken so far
        if (c == 0) inv_s = invmod(cand[cs], mp);
        if (c < t) fk[c] = aug[c][cs];
        __syncthreads();
        const uint32_t nrm = mulmod(nv, inv_s, mp);
        for (int k = 0; k < t; ++k) {
            const uint32_t f = fk[k];
            if (f) aug[k][c] = mod64((uint64_t)aug[k][c] + (P - f) * nrm, mp);
        }
        aug[t][c] = nrm;
        if (c == 0) {
            bcol[t] = cs;
            S[t] = (int)i;
        }
        ++t;
        __syncthreads();
    }
    __syncthreads();
    // order the basis rows by pivot column
    if (c < t) {
        int r = 0;
        for (int k = 0; k < t; ++k) r += (bcol[k] < bcol[c]) ? 1 : 0;
        rnk[c] = r;
    }
    __syncthreads();
    if (c == 0) *t_out = t;
    if (c < t) {
        S_out[c] = S[c];
        pc_out[rnk[c]] = bcol[c];
    }
    for (int k = 0; k < t; ++k) {
        // G row rnk[k] = coefficient part of basis row k (columns = S order)
        if (c < PANEL) G_out[rnk[k] * PANEL + c] = (uint16_t)((c < t) ? aug[k][PANEL + c] : 0u);
    }
}

__global__ void zero_plane_rows_kernel(Planes H, const int32_t *__restrict__ rows, const int32_t *__restrict__ t_dev)
{
    const int t = *t_dev;
    const int j = blockIdx.x;
    if (j >= t) return;
    const size_t off = (size_t)rows[j] * H.kp;
    for (int k = threadIdx.x; k < H.kp; k += blockDim.x) {
        H.plane(0)[off + k] = __float2bfloat16_rn(0.f);
        H.plane(1)[off + k] = __float2bfloat16_rn(0.f);
    }
}

// D[S[k]][c0 + i] = W^T[i][k]; mark the rows as pivots; record pivots.
__global__ void write_pivots_kernel(uint16_t *D, int64_t ldd, int64_t c0, int64_t ncols, const uint16_t *__restrict__ WT,
                                    int64_t ldw, const int32_t *__restrict__ S, const int32_t *__restrict__ pc,
                                    const int32_t *__restrict__ t_dev, int32_t *__restrict__ is_piv_row,
                                    int32_t *__restrict__ prow, int32_t *__restrict__ pcol, int64_t rank0)
{
    const int t = *t_dev;
    const int k = blockIdx.y;
    if (k >= t) return;
    const int64_t r = S[k];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ncols; i += (int64_t)gridDim.x * blockDim.x)
        D[r * ldd + c0 + i] = WT[i * ldw + k];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        is_piv_row[r] = 1;
        prow[rank0 + k] = (int32_t)r;
        pcol[rank0 + k] = (int32_t)(c0 + pc[k]);
    }
}

int echelon_d(const EchelonD &E, int64_t *rank_out)
{
    *rank_out = 0;
    const int64_t m = E.m, n = E.n;
    if (m <= 0 || n <= 0) return GBLA_OK;
    cudaStream_t s = E.s;
    const ModP &mp = *E.mp;
    int32_t *t_dev = nullptr, *S = nullptr, *pc = nullptr;
    uint16_t *G = nullptr, *WT = nullptr;
    Planes Gp{}, DsT{}, Wp{}, H{};
    int rc = GBLA_OK;
    int64_t rank = 0;
    const int64_t ldw = PANEL;
    const size_t panel_smem = (size_t)PANEL * 2 * PANEL * sizeof(uint32_t);
    GBLA_CUDA_TRY(cudaMemsetAsync(E.is_piv_row, 0, sizeof(int32_t) * (size_t)m, s));
    GBLA_TRY(dalloc_t(&t_dev, 4, s));
    GBLA_TRY(dalloc_t(&S, PANEL, s));
    GBLA_TRY(dalloc_t(&pc, PANEL, s));
    GBLA_TRY(dalloc_t(&G, (size_t)PANEL * PANEL, s));
    GBLA_TRY(dalloc_t(&WT, (size_t)round_up(n, 128) * PANEL, s));
    GBLA_TRY(planes_alloc(&Gp, PANEL, PANEL, 4, s));
    GBLA_TRY(planes_alloc(&DsT, n, PANEL, 2, s));
    GBLA_TRY(planes_alloc(&Wp, n, PANEL, 4, s));
    GBLA_TRY(planes_alloc(&H, m, PANEL, 2, s));
    static bool attr = false;
    if (!attr) {
        GBLA_CUDA_TRY(cudaFuncSetAttribute(panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)panel_smem));
        attr = true;
    }
    for (int64_t c0 = 0; c0 < n && rank < m; c0 += PANEL) {
        const int bw = (int)((n - c0) < PANEL ? (n - c0) : PANEL);
        const int64_t nc = n - c0;   // trailing columns incl. the panel
        panel_kernel<<<1, 2 * PANEL, panel_smem, s>>>(E.D16, E.ldd, m, c0, bw, E.is_piv_row, t_dev, S, pc, G, mp);
        if (cudaGetLastError() != cudaSuccess) { rc = GBLA_E_CUDA; break; }
        int32_t t = 0;
        if (cudaMemcpyAsync(&t, t_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) { rc = GBLA_E_CUDA; break; }
        if (t == 0) continue;
        // G (rows: pivots in column order, cols: S order) as a B-operand: Bop[k][j] = G[k][j]
        if ((rc = to_planes(Gp, t, t, G, PANEL, 0, false, nullptr, nullptr, mp, s))) break;
        // D[S, c0:]^T as an A-operand: Aop[i][j] = D[S[j]][c0 + i]
        if ((rc = to_planes(DsT, nc, t, E.D16, E.ldd, c0, true, S, nullptr, mp, s))) break;
        // W^T = D[S, c0:]^T * G^T
        if (cudaMemsetAsync(WT, 0, sizeof(uint16_t) * (size_t)nc * ldw, s) != cudaSuccess) { rc = GBLA_E_CUDA; break; }
        if ((rc = modgemm(DsT, 0, 0, Gp, 0, 0, WT, ldw, nc, t, t, +1, mp, E.variant, E.err, s, E.ctr))) break;
        // W as a B-operand: Bop[i][k] = W^T[i][k]
        if ((rc = to_planes(Wp, nc, t, WT, ldw, 0, false, nullptr, nullptr, mp, s))) break;
        // H = D[:, c0 + pc] with the rows S zeroed
        if ((rc = to_planes(H, m, t, E.D16, E.ldd, c0, false, nullptr, pc, mp, s))) break;
        zero_plane_rows_kernel<<<t, 128, 0, s>>>(H, S, t_dev);
        if (cudaGetLastError() != cudaSuccess) { rc = GBLA_E_CUDA; break; }
        // every other row: row[c0:] -= row[pc] * W
        if ((rc = modgemm(H, 0, 0, Wp, 0, 0, E.D16 + c0, E.ldd, m, nc, t, -1, mp, E.variant, E.err, s, E.ctr))) break;
        dim3 grid((unsigned)((nc + 255) / 256 < 64 ? (nc + 255) / 256 : 64), (unsigned)t);
        write_pivots_kernel<<<grid, 256, 0, s>>>(E.D16, E.ldd, c0, nc, WT, ldw, S, pc, t_dev, E.is_piv_row, E.prow,
                                                 E.pcol, rank);
        if (cudaGetLastError() != cudaSuccess) { rc = GBLA_E_CUDA; break; }
        rank += t;
    }
    dfree(t_dev, s);
    dfree(S, s);
    dfree(pc, s);
    dfree(G, s);
    dfree(WT, s);
    planes_free(&Gp, s);
    planes_free(&DsT, s);
    planes_free(&Wp, s);
    planes_free(&H, s);
    *rank_out = rank;
    return rc;
}

}  // namespace gbla
