// split.cu -- FL step 1 (pivot analysis and splicing) and FL step 5 (output
// assembly) of the GBLA paper, Sec. 3.1 and Sec. 4.1, plus the 2-multiline
// layout of Definition 1 (Sec. 4.2).
//
// Step 1 on the GPU:
//   (a1) one warp per row validates the CSR and finds the row's pivoting
//        candidate = its leftmost nonzero column;
//   (a2) per column, the candidate rows compete through one 64-bit atomicMin
//        on the key (row weight << 32 | row index): the winner is the row
//        with the fewest nonzeros, ties to the smaller index.  A scan over
//        the column flags gives the column permutation: pivot columns first,
//        then the other columns, each group in input order;
//   (a3) a second warp-per-row pass scatters every entry into the blocks
//        A (pivot rows x pivot columns, rows normalised to a leading 1),
//        B (pivot rows x other columns), C and D (the other rows), directly
//        in the digit-plane layout the tensor-core product reads.
#include "common.cuh"
#include "internal.cuh"
#include "split.cuh"

namespace gbla {

// ------------------------------------------------------------------ scan
__global__ void scan_block_kernel(const int64_t *__restrict__ in, int64_t *__restrict__ out, int64_t n,
                                  int64_t *__restrict__ block_sums)
{
    __shared__ int64_t warp_tot[8];
    const int64_t base = (int64_t)blockIdx.x * 1024 + threadIdx.x * 4;
    int64_t v[4];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        s += v[i];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    int64_t woff = 0;
    for (int w = 0; w < warp; ++w) woff += warp_tot[w];
    int64_t run = woff + incl - s;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == 255 && block_sums) {
        int64_t tot = 0;
        for (int w = 0; w < 8; ++w) tot += warp_tot[w];
        block_sums[blockIdx.x] = tot;
    }
}

__global__ void scan_add_kernel(int64_t *__restrict__ out, int64_t n, const int64_t *__restrict__ offs)
{
    const int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    const int64_t o = offs[blockIdx.x];
    for (int k = 0; k < 4; ++k)
        if (i + k * 256 < n) out[i + k * 256] += o;
}

__global__ void copy_i64_kernel(int64_t *dst, const int64_t *src) { *dst = *src; }

int scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total_dev, cudaStream_t s)
{
    if (n <= 0) {
        if (total_dev) GBLA_CUDA_TRY(cudaMemsetAsync(total_dev, 0, sizeof(int64_t), s));
        return GBLA_OK;
    }
    const int64_t nb = (n + 1023) / 1024;
    DevTemp<int64_t> sums(s);
    GBLA_TRY(sums.alloc((size_t)nb + 1));
    scan_block_kernel<<<(unsigned)nb, 256, 0, s>>>(in, out, n, sums);
    GBLA_CUDA_TRY(launch_check());
    int rc = GBLA_OK;
    if (nb == 1) {
        // one block: its sum is the total
        if (total_dev) {
            copy_i64_kernel<<<1, 1, 0, s>>>(total_dev, sums);
            if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
        }
    } else {
        // scan the block sums (sums[nb] receives the grand total), add them back
        rc = scan_i64(sums, sums, nb, sums.p + nb, s);
        if (rc == GBLA_OK) {
            scan_add_kernel<<<(unsigned)nb, 256, 0, s>>>(out, n, sums);
            if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
        }
        if (rc == GBLA_OK && total_dev) {
            copy_i64_kernel<<<1, 1, 0, s>>>(total_dev, sums.p + nb);
            if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
        }
    }
    return rc;
}

// ---------------------------------------------------------- (a1) + (a2)
__global__ void scan_rows_kernel(int64_t m, int64_t n, int64_t nnz, const int64_t *__restrict__ row_ptr,
                                 const int32_t *__restrict__ col, const uint16_t *__restrict__ val, uint32_t p,
                                 int32_t *__restrict__ lead, unsigned long long *__restrict__ best, uint32_t *err)
{
    const int64_t warp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp_id >= m) return;
    const int64_t r = warp_id;
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
        if (lane == 0) {
            dev_fail(err, DEV_ERR_INVAL);
            lead[r] = -1;
        }
        return;
    }
    if (lane == 0) {
        if (e > b) {
            const int32_t c = col[b];
            lead[r] = c;
            const unsigned long long key = ((unsigned long long)(e - b) << 32) | (unsigned long long)r;
            atomicMin(&best[c], key);
        } else {
            lead[r] = -1;
        }
    }
}

__global__ void col_flags_kernel(int64_t n, const unsigned long long *__restrict__ best, int64_t *__restrict__ flag)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) flag[c] = (best[c] != ~0ull) ? 1 : 0;
}

// colmap[c] = permuted column index: pivot columns first (ascending), then the
// others (ascending).
__global__ void colmap_kernel(int64_t n, const unsigned long long *__restrict__ best, const int64_t *__restrict__ pos,
                              const int64_t *__restrict__ npiv_dev, int32_t *__restrict__ colmap,
                              int32_t *__restrict__ pivcol_orig, int32_t *__restrict__ npcol_orig,
                              int32_t *__restrict__ piv_row)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int64_t npiv = *npiv_dev;
    const unsigned long long bk = best[c];
    if (bk != ~0ull) {
        const int64_t k = pos[c];
        colmap[c] = (int32_t)k;
        pivcol_orig[k] = (int32_t)c;
        piv_row[k] = (int32_t)(bk & 0xFFFFFFFFull);
    } else {
        const int64_t k = c - pos[c];
        colmap[c] = (int32_t)(npiv + k);
        npcol_orig[k] = (int32_t)c;
    }
}

__global__ void row_flags_kernel(int64_t m, const int32_t *__restrict__ lead,
                                 const unsigned long long *__restrict__ best, int64_t *__restrict__ flag)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    const int32_t l = lead[r];
    flag[r] = (l >= 0 && (int64_t)(best[l] & 0xFFFFFFFFull) != r) ? 1 : 0;
}

// C/D rows are ordered by the permuted index of their leading column (a
// counting sort; rows with the same lead stay in input order).  X = C*A^-1 is
// zero left of a row's lead, so in this order the nonzeros of X, and of the
// Schur complement, form a staircase that the products and solves skip.
__global__ void cd_count_kernel(int64_t m, const int64_t *__restrict__ flag, const int32_t *__restrict__ lead,
                                const int32_t *__restrict__ colmap, int64_t *__restrict__ cnt)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < m && flag[r]) atomicAdd(reinterpret_cast<unsigned long long *>(&cnt[colmap[lead[r]]]), 1ull);
}

__global__ void cd_scatter_kernel(int64_t m, const int64_t *__restrict__ flag, const int32_t *__restrict__ lead,
                                  const int32_t *__restrict__ colmap, const int64_t *__restrict__ off,
                                  int32_t *__restrict__ fill, int32_t *__restrict__ cd_rows)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m || !flag[r]) return;
    const int64_t k = colmap[lead[r]];
    cd_rows[off[k] + atomicAdd(&fill[k], 1)] = (int32_t)r;
}

// Sort each bucket by input row index, then index.  Buckets are small in
// F4 matrices (a few rows share a lead); a bucket of more than 2048 rows keeps
// the arrival order, which changes which rows become pivots of D' but not
// the result, the reduced echelon form being unique.
__global__ void cd_finish_kernel(int64_t npiv, const int64_t *__restrict__ off, int32_t *__restrict__ cd_rows,
                                 int32_t *__restrict__ cd_index, int32_t *__restrict__ cd_lead)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npiv) return;
    const int64_t b = off[k], e = off[k + 1];
    for (int64_t i = b + 1; i < e && e - b <= 2048; ++i) {
        const int32_t v = cd_rows[i];
        int64_t j = i - 1;
        while (j >= b && cd_rows[j] > v) {
            cd_rows[j + 1] = cd_rows[j];
            --j;
        }
        cd_rows[j + 1] = v;
    }
    for (int64_t i = b; i < e; ++i) {
        cd_index[cd_rows[i]] = (int32_t)i;
        cd_lead[i] = (int32_t)k;
    }
}

__global__ void inv_lead_kernel(int64_t npiv, const int32_t *__restrict__ piv_row, const int64_t *__restrict__ row_ptr,
                                const uint16_t *__restrict__ val, uint32_t *__restrict__ inv, ModP mp)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npiv) return;
    inv[k] = invmod(val[row_ptr[piv_row[k]]], mp);
}

int pivot_analysis(const DevCSR &in, const ModP &mp, PivotInfo *pi, uint32_t *err, cudaStream_t s)
{
    const int64_t m = in.m, n = in.n;
    pi->m = m;
    pi->n = n;
    GBLA_TRY(dalloc_t(&pi->lead, (size_t)m + 1, s));
    GBLA_TRY(dalloc_t(&pi->best, (size_t)n + 1, s));
    GBLA_CUDA_TRY(cudaMemsetAsync(pi->best, 0xFF, sizeof(unsigned long long) * (size_t)(n + 1), s));
    if (m > 0) {
        const int64_t threads = m * 32;
        scan_rows_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(m, n, in.nnz, in.row_ptr, in.col, in.val,
                                                                           mp.p, pi->lead, pi->best, err);
        GBLA_CUDA_TRY(launch_check());
    }
    DevTemp<int64_t> cflag(s), rflag(s), rpos(s);
    GBLA_TRY(cflag.alloc((size_t)n + 1));
    GBLA_TRY(rflag.alloc((size_t)m + 1));
    GBLA_TRY(rpos.alloc((size_t)(m > n ? m : n) + 2));
    GBLA_TRY(dalloc_t(&pi->dev_counts, 2, s));
    if (n > 0) {
        col_flags_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, pi->best, cflag);
        GBLA_CUDA_TRY(launch_check());
    }
    GBLA_TRY(scan_i64(cflag, cflag, n, pi->dev_counts + 0, s));
    if (m > 0) {
        row_flags_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(m, pi->lead, pi->best, rflag);
        GBLA_CUDA_TRY(launch_check());
    }
    GBLA_TRY(scan_i64(rflag, rpos, m, pi->dev_counts + 1, s));
    int64_t host_counts[2] = {0, 0};
    GBLA_TRY(readback(host_counts, pi->dev_counts, sizeof(host_counts), s));
    uint32_t herr = 0;
    GBLA_TRY(readback(&herr, err, sizeof(herr), s));
    if (herr & DEV_ERR_INVAL) return GBLA_E_INVAL;
    pi->npiv = host_counts[0];
    pi->m_cd = host_counts[1];
    pi->n_d = n - pi->npiv;
    GBLA_TRY(dalloc_t(&pi->colmap, (size_t)n + 1, s));
    GBLA_TRY(dalloc_t(&pi->pivcol_orig, (size_t)pi->npiv + 1, s));
    GBLA_TRY(dalloc_t(&pi->npcol_orig, (size_t)pi->n_d + 1, s));
    GBLA_TRY(dalloc_t(&pi->piv_row, (size_t)pi->npiv + 1, s));
    GBLA_TRY(dalloc_t(&pi->cd_rows, (size_t)pi->m_cd + 1, s));
    GBLA_TRY(dalloc_t(&pi->cd_index, (size_t)m + 1, s));
    GBLA_TRY(dalloc_t(&pi->cd_lead, (size_t)pi->m_cd + 1, s));
    GBLA_TRY(dalloc_t(&pi->inv_lead, (size_t)pi->npiv + 1, s));
    if (n > 0) {
        colmap_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, pi->best, cflag, pi->dev_counts, pi->colmap,
                                                                  pi->pivcol_orig, pi->npcol_orig, pi->piv_row);
        GBLA_CUDA_TRY(launch_check());
    }
    if (m > 0) {
        // counting sort of the C/D rows by leading pivot column (rpos reused as counts/offsets)
        DevTemp<int32_t> fill(s);
        const int64_t nk = pi->npiv + 1;
        GBLA_TRY(fill.alloc((size_t)nk));
        GBLA_CUDA_TRY(cudaMemsetAsync(fill, 0, sizeof(int32_t) * (size_t)nk, s));
        GBLA_CUDA_TRY(cudaMemsetAsync(rpos, 0, sizeof(int64_t) * (size_t)(nk < m + 1 ? m + 1 : nk), s));
        GBLA_CUDA_TRY(cudaMemsetAsync(pi->cd_index, 0xFF, sizeof(int32_t) * (size_t)m, s));
        cd_count_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(m, rflag, pi->lead, pi->colmap, rpos);
        GBLA_CUDA_TRY(launch_check());
        GBLA_TRY(scan_i64(rpos, rpos, nk, nullptr, s));
        cd_scatter_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(m, rflag, pi->lead, pi->colmap, rpos, fill,
                                                                      pi->cd_rows);
        GBLA_CUDA_TRY(launch_check());
        if (pi->npiv > 0) {
            cd_finish_kernel<<<(unsigned)((pi->npiv + 255) / 256), 256, 0, s>>>(pi->npiv, rpos, pi->cd_rows,
                                                                                pi->cd_index, pi->cd_lead);
            GBLA_CUDA_TRY(launch_check());
        }
    }
    if (pi->npiv > 0) {
        inv_lead_kernel<<<(unsigned)((pi->npiv + 255) / 256), 256, 0, s>>>(pi->npiv, pi->piv_row, in.row_ptr, in.val,
                                                                          pi->inv_lead, mp);
        GBLA_CUDA_TRY(launch_check());
    }
    return GBLA_OK;
}

void pivot_free(PivotInfo *pi, cudaStream_t s)
{
    dfree(pi->lead, s);
    dfree(pi->best, s);
    dfree(pi->dev_counts, s);
    dfree(pi->colmap, s);
    dfree(pi->pivcol_orig, s);
    dfree(pi->npcol_orig, s);
    dfree(pi->piv_row, s);
    dfree(pi->cd_rows, s);
    dfree(pi->cd_index, s);
    dfree(pi->cd_lead, s);
    dfree(pi->inv_lead, s);
    *pi = PivotInfo();
}

// ---------------------------------------------------------------- (a3)
// One warp per input row.  Pivot rows are normalised by the inverse of their
// leading coefficient and go to A (pivot columns) and B (other columns),
// unless A16 is null (the sparse path keeps them sparse); other rows go to C
// and D.  All four blocks are dense uint16 row-major here;
// the digit planes the tensor-core product reads are made from A and B by a
// tiled transposing conversion (coalesced on both sides).
__global__ void split_scatter_kernel(int64_t m, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                     const uint16_t *__restrict__ val, const int32_t *__restrict__ lead,
                                     const unsigned long long *__restrict__ best, const int32_t *__restrict__ colmap,
                                     const int32_t *__restrict__ cd_index, const uint32_t *__restrict__ inv_lead,
                                     int64_t npiv, uint16_t *__restrict__ A16, int64_t lda, uint16_t *__restrict__ B16,
                                     int64_t ldb, uint16_t *__restrict__ C16, int64_t ldc, uint16_t *__restrict__ D16,
                                     int64_t ldd, ModP mp)
{
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= m) return;
    const int32_t l = lead[r];
    if (l < 0) return;
    const int64_t b = row_ptr[r], e = row_ptr[r + 1];
    const bool is_piv = (int64_t)(best[l] & 0xFFFFFFFFull) == r;
    if (is_piv) {
        if (!A16) return;   // sparse path: pivot rows go to sparse_build
        const int64_t k = colmap[l];
        const uint32_t inv = inv_lead[k];
        for (int64_t i = b + lane; i < e; i += 32) {
            const int64_t c = colmap[col[i]];
            const uint16_t v = (uint16_t)mulmod(val[i], inv, mp);
            if (c < npiv) A16[k * lda + c] = v;
            else B16[k * ldb + (c - npiv)] = v;
        }
    } else {
        const int64_t i_cd = cd_index[r];
        for (int64_t i = b + lane; i < e; i += 32) {
            const int64_t c = colmap[col[i]];
            if (c < npiv) C16[i_cd * ldc + c] = val[i];
            else D16[i_cd * ldd + (c - npiv)] = val[i];
        }
    }
}

int split_scatter(const DevCSR &in, const PivotInfo &pi, uint16_t *A16, int64_t lda, uint16_t *B16, int64_t ldb,
                  uint16_t *C16, int64_t ldc, uint16_t *D16, int64_t ldd, const ModP &mp, cudaStream_t s)
{
    if (in.m <= 0) return GBLA_OK;
    const int64_t threads = in.m * 32;
    split_scatter_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
        in.m, in.row_ptr, in.col, in.val, pi.lead, pi.best, pi.colmap, pi.cd_index, pi.inv_lead, pi.npiv, A16, lda,
        B16, ldb, C16, ldc, D16, ldd, mp);
    GBLA_CUDA_TRY(launch_check());
    return GBLA_OK;
}

// ------------------------------------------------------------ multiline
// Pair q holds pivot rows 2q and 2q+1 (A rows, permuted column indices).
// Entries exclude each row's own leading 1 (the unit diagonal of A).
// Row 2q+1 of an odd count is a virtual zero row.
__device__ __forceinline__ void a_row_range(int64_t k, int64_t npiv, const int32_t *piv_row, const int64_t *row_ptr,
                                            int64_t &b, int64_t &e)
{
    if (k >= npiv) { b = e = 0; return; }
    const int64_t r = piv_row[k];
    b = row_ptr[r] + 1;   // skip the lead
    e = row_ptr[r + 1];
}

template <bool FILL>
__global__ void multiline_kernel(int64_t npairs, int64_t npiv, const int32_t *__restrict__ piv_row,
                                 const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                 const uint16_t *__restrict__ val, const int32_t *__restrict__ colmap,
                                 const uint32_t *__restrict__ inv_lead, int64_t *__restrict__ cnt_or_ptr,
                                 int32_t *__restrict__ ml_pos, uint32_t *__restrict__ ml_val,
                                 int32_t *__restrict__ inblk, ModP mp)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= npairs) return;
    int64_t b1, e1, b2, e2;
    a_row_range(2 * q, npiv, piv_row, row_ptr, b1, e1);
    a_row_range(2 * q + 1, npiv, piv_row, row_ptr, b2, e2);
    const uint32_t inv1 = inv_lead[2 * q];
    const uint32_t inv2 = (2 * q + 1 < npiv) ? inv_lead[2 * q + 1] : 0;
    int64_t i1 = b1, i2 = b2, out = FILL ? cnt_or_ptr[q] : 0;
    const int64_t blk_end = (2 * q / LEAF_COLS + 1) * LEAF_COLS;
    int32_t n_in = 0;
    // Only entries in pivot columns inside the pair's own diagonal block of
    // A: the sparse solves apply exactly these; everything right of the block
    // goes through the dense products.  Both rows are sorted by column, and
    // the permuted pivot columns keep the input order.
    while (true) {
        int64_t c1 = INT64_MAX, c2 = INT64_MAX;
        while (i1 < e1) {
            int64_t c = colmap[col[i1]];
            if (c < npiv) { c1 = c; break; }
            ++i1;
        }
        while (i2 < e2) {
            int64_t c = colmap[col[i2]];
            if (c < npiv) { c2 = c; break; }
            ++i2;
        }
        if (c1 >= blk_end) c1 = INT64_MAX;
        if (c2 >= blk_end) c2 = INT64_MAX;
        if (c1 == INT64_MAX && c2 == INT64_MAX) break;
        const int64_t c = c1 < c2 ? c1 : c2;
        uint32_t v1 = 0, v2 = 0;
        if (c1 == c) { v1 = mulmod(val[i1], inv1, mp); ++i1; }
        if (c2 == c) { v2 = mulmod(val[i2], inv2, mp); ++i2; }
        if (FILL) {
            ml_pos[out] = (int32_t)c;
            ml_val[out] = v1 | (v2 << 16);
        }
        n_in += (c < blk_end) ? 1 : 0;
        ++out;
    }
    if (!FILL) cnt_or_ptr[q] = out;
    else inblk[q] = n_in;
}

int multiline_build(const DevCSR &in, const PivotInfo &pi, Multiline *ml, const ModP &mp, cudaStream_t s)
{
    const int64_t npairs = (pi.npiv + 1) / 2;
    ml->npairs = npairs;
    GBLA_TRY(dalloc_t(&ml->ptr, (size_t)npairs + 2, s));
    if (npairs == 0) {
        GBLA_CUDA_TRY(cudaMemsetAsync(ml->ptr, 0, sizeof(int64_t), s));
        ml->pos = nullptr;
        ml->val = nullptr;
        return GBLA_OK;
    }
    const unsigned nb = (unsigned)((npairs + 127) / 128);
    multiline_kernel<false><<<nb, 128, 0, s>>>(npairs, pi.npiv, pi.piv_row, in.row_ptr, in.col, in.val, pi.colmap,
                                               pi.inv_lead, ml->ptr, nullptr, nullptr, nullptr, mp);
    GBLA_CUDA_TRY(launch_check());
    GBLA_TRY(scan_i64(ml->ptr, ml->ptr, npairs, ml->ptr + npairs, s));
    int64_t total = 0;
    GBLA_TRY(readback(&total, ml->ptr + npairs, sizeof(int64_t), s));
    ml->total = total;
    GBLA_TRY(dalloc_t(&ml->pos, (size_t)total + 1, s));
    GBLA_TRY(dalloc_t(&ml->val, (size_t)total + 1, s));
    GBLA_TRY(dalloc_t(&ml->inblk, (size_t)npairs + 1, s));
    multiline_kernel<true><<<nb, 128, 0, s>>>(npairs, pi.npiv, pi.piv_row, in.row_ptr, in.col, in.val, pi.colmap,
                                              pi.inv_lead, ml->ptr, ml->pos, ml->val, ml->inblk, mp);
    GBLA_CUDA_TRY(launch_check());
    return GBLA_OK;
}

void multiline_free(Multiline *ml, cudaStream_t s)
{
    dfree(ml->ptr, s);
    dfree(ml->pos, s);
    dfree(ml->val, s);
    dfree(ml->inblk, s);
    *ml = Multiline();
}

// Generic multiline of consecutive row pairs of an arbitrary CSR (test entry).
__global__ void multiline_pairs_kernel(int64_t npairs, int64_t m, const int64_t *__restrict__ row_ptr,
                                       const int32_t *__restrict__ col, const uint16_t *__restrict__ val,
                                       int64_t *__restrict__ cnt_or_ptr, int32_t *__restrict__ ml_pos,
                                       uint16_t *__restrict__ ml_val, int fill)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= npairs) return;
    int64_t i1 = row_ptr[2 * q], e1 = row_ptr[2 * q + 1];
    int64_t i2 = (2 * q + 1 < m) ? row_ptr[2 * q + 1] : 0, e2 = (2 * q + 1 < m) ? row_ptr[2 * q + 2] : 0;
    int64_t out = fill ? cnt_or_ptr[q] : 0;
    while (i1 < e1 || i2 < e2) {
        const int64_t c1 = i1 < e1 ? col[i1] : INT64_MAX, c2 = i2 < e2 ? col[i2] : INT64_MAX;
        const int64_t c = c1 < c2 ? c1 : c2;
        uint16_t v1 = 0, v2 = 0;
        if (c1 == c) v1 = val[i1++];
        if (c2 == c) v2 = val[i2++];
        if (fill) {
            ml_pos[out] = (int32_t)c;
            ml_val[2 * out] = v1;
            ml_val[2 * out + 1] = v2;
        }
        ++out;
    }
    if (!fill) cnt_or_ptr[q] = out;
}

int multiline_pairs(int64_t m, const int64_t *row_ptr, const int32_t *col, const uint16_t *val, int64_t *ml_ptr_dev,
                    int32_t *ml_pos_dev, uint16_t *ml_val_dev, int64_t *total, cudaStream_t s)
{
    const int64_t npairs = (m + 1) / 2;
    if (npairs == 0) {
        *total = 0;
        GBLA_CUDA_TRY(cudaMemsetAsync(ml_ptr_dev, 0, sizeof(int64_t), s));
        return GBLA_OK;
    }
    const unsigned nb = (unsigned)((npairs + 127) / 128);
    multiline_pairs_kernel<<<nb, 128, 0, s>>>(npairs, m, row_ptr, col, val, ml_ptr_dev, nullptr, nullptr, 0);
    GBLA_CUDA_TRY(launch_check());
    GBLA_TRY(scan_i64(ml_ptr_dev, ml_ptr_dev, npairs, ml_ptr_dev + npairs, s));
    GBLA_TRY(readback(total, ml_ptr_dev + npairs, sizeof(int64_t), s));
    if (ml_pos_dev) {
        multiline_pairs_kernel<<<nb, 128, 0, s>>>(npairs, m, row_ptr, col, val, ml_ptr_dev, ml_pos_dev, ml_val_dev, 1);
        GBLA_CUDA_TRY(launch_check());
    }
    return GBLA_OK;
}

}  // namespace gbla
