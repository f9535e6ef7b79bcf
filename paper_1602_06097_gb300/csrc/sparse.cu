// sparse.cu -- the pivot rows of the split as sparse operands (FL step 1,
// GBLA paper Sec. 4.1; the block densities of Table 4: A and B are sparse).
//
// On the sparse path the normalised pivot rows are never materialised as
// dense npiv x npiv and npiv x n_d blocks.  Their entries go to
//   * Adiag: A's diagonal blocks of width L (the leaves of the triangular
//     solve), dense uint16, row k holding A[k][c] at column c % L for c in
//     k's own block -- the input of the leaf inverses;
//   * two K-compacted operands of the gathered product (Compact):
//       SA: A's entries A[k][c] whose column c lies in a later leaf than k
//           (the off-diagonal blocks), grouped by the 128-column tile of c;
//       SB: B's entries, grouped by the 128-column tile of their non-pivot
//           column.
//     For a tile t the rows k with a nonzero in the tile form the list
//     kidx[koff[t] .. koff[t + 1]) (ascending, padded with KIDX_PAD to a
//     multiple of 128), and the tile restricted to those rows is stored as
//     dense B-operand digit planes, chunk-major: list entries 32 q .. 32 q + 31
//     of all tiles' lists form chunk q, 128 rows (the tile's columns) of
//     64 bf16 (hi digits of the 32 values, then lo digits).
//     F4 rows come in runs of consecutive columns with vertical repetition
//     (Sec. 4.2), so a 128-column tile meets few rows and the compacted
//     tiles are far denser than the block.
//
// Steps (one warp per pivot row, or one CTA per tile):
//   1. mark: bit k of tile t's row bitmap is set when row k has an entry in
//      tile t (atomicOr); Adiag entries are written directly;
//   2. count: per tile, exclusive prefix of the bitmap words' popcounts;
//   3. offsets: koff = exclusive scan of the counts rounded up to 128;
//   4. list: the set bits in order;
//   5. values: the position of entry (k, c) in its tile's list is the tile's
//      word prefix plus the popcount of the lower bits of k's word.
#include "common.cuh"
#include "internal.cuh"
#include "split.cuh"

namespace gbla {

namespace {

constexpr int TILE = 128;

__device__ __forceinline__ void store_digit_planes(__nv_bfloat16 *rowp, int kin, uint32_t v, const ModP &mp) {
    int h, l;
    digits(v, mp.p, h, l);
    rowp[kin] = i2bf(h);
    rowp[32 + kin] = i2bf(l);
}

// Step 1 (one warp per pivot row k).
__global__ void sp_mark_kernel(int64_t npiv, int L, const int32_t *__restrict__ piv_row,
                               const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                               const uint16_t *__restrict__ val, const int32_t *__restrict__ colmap,
                               const uint32_t *__restrict__ inv_lead, uint16_t *__restrict__ Adiag, int64_t wpr,
                               uint32_t *__restrict__ bitsA, uint32_t *__restrict__ bitsB, ModP mp)
{
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= npiv) return;
    const int64_t r = piv_row[k];
    const int64_t b = row_ptr[r], e = row_ptr[r + 1];
    const uint32_t inv = inv_lead[k];
    const int64_t kleaf = k / L;
    const uint32_t bit = 1u << (k & 31);
    const int64_t w = k >> 5;
    for (int64_t i = b + lane; i < e; i += 32) {
        const int64_t c = colmap[col[i]];
        if (c < npiv) {
            if (c / L == kleaf) Adiag[k * L + (c % L)] = (uint16_t)mulmod(val[i], inv, mp);
            else atomicOr(&bitsA[(c / TILE) * wpr + w], bit);
        } else {
            atomicOr(&bitsB[((c - npiv) / TILE) * wpr + w], bit);
        }
    }
}

// Step 2 (one CTA of 256 threads per tile): wordoff[t][w] = set bits of the
// tile's words before w; padded[t] = the tile's count rounded up to 128.
__global__ void __launch_bounds__(256) sp_count_kernel(int64_t wpr, const uint32_t *__restrict__ bits,
                                                       int32_t *__restrict__ wordoff, int64_t *__restrict__ padded)
{
    __shared__ int32_t part[256];
    const int64_t t = blockIdx.x;
    const uint32_t *tb = bits + t * wpr;
    int32_t *to = wordoff + t * wpr;
    const int64_t per = (wpr + 255) / 256;
    const int64_t w0 = threadIdx.x * per, w1 = (w0 + per < wpr) ? w0 + per : wpr;
    int32_t s = 0;
    for (int64_t w = w0; w < w1; ++w) s += __popc(tb[w]);
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {   // 256 partial sums: a serial scan is cheap
        int32_t run = 0;
        for (int i = 0; i < 256; ++i) {
            const int32_t x = part[i];
            part[i] = run;
            run += x;
        }
        padded[t] = ((int64_t)run + TILE - 1) / TILE * TILE;
    }
    __syncthreads();
    int32_t run = part[threadIdx.x];
    for (int64_t w = w0; w < w1; ++w) {
        to[w] = run;
        run += __popc(tb[w]);
    }
}

// Step 4 (one CTA per tile): the list of the tile's rows.
__global__ void __launch_bounds__(256) sp_list_kernel(int64_t wpr, const uint32_t *__restrict__ bits,
                                                      const int32_t *__restrict__ wordoff,
                                                      const int64_t *__restrict__ koff, int32_t *__restrict__ kidx)
{
    const int64_t t = blockIdx.x;
    for (int64_t w = threadIdx.x; w < wpr; w += blockDim.x) {
        uint32_t x = bits[t * wpr + w];
        int64_t pos = koff[t] + wordoff[t * wpr + w];
        while (x) {
            const int b = __ffs(x) - 1;
            kidx[pos++] = (int32_t)(w * 32 + b);
            x &= x - 1u;
        }
    }
}

// Step 5 (one warp per pivot row k): values of the compacted tiles.
__global__ void sp_values_kernel(int64_t npiv, int L, const int32_t *__restrict__ piv_row,
                                 const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                 const uint16_t *__restrict__ val, const int32_t *__restrict__ colmap,
                                 const uint32_t *__restrict__ inv_lead, int64_t wpr,
                                 const uint32_t *__restrict__ bitsA, const int32_t *__restrict__ woffA,
                                 const int64_t *__restrict__ koffA, __nv_bfloat16 *__restrict__ planesA,
                                 const uint32_t *__restrict__ bitsB, const int32_t *__restrict__ woffB,
                                 const int64_t *__restrict__ koffB, __nv_bfloat16 *__restrict__ planesB, ModP mp)
{
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= npiv) return;
    const int64_t r = piv_row[k];
    const int64_t b = row_ptr[r], e = row_ptr[r + 1];
    const uint32_t inv = inv_lead[k];
    const int64_t kleaf = k / L;
    const int64_t w = k >> 5;
    const uint32_t below = (1u << (k & 31)) - 1u;
    for (int64_t i = b + lane; i < e; i += 32) {
        const int64_t c = colmap[col[i]];
        const uint32_t *bits;
        const int32_t *woff;
        const int64_t *koff;
        __nv_bfloat16 *planes;
        int64_t cc;
        if (c < npiv) {
            if (c / L == kleaf) continue;   // diagonal block: Adiag
            bits = bitsA, woff = woffA, koff = koffA, planes = planesA, cc = c;
        } else {
            bits = bitsB, woff = woffB, koff = koffB, planes = planesB, cc = c - npiv;
        }
        const int64_t t = cc / TILE;
        const int64_t kk = koff[t] + woff[t * wpr + w] + __popc(bits[t * wpr + w] & below);
        __nv_bfloat16 *rowp = planes + ((kk >> 5) * TILE + (cc % TILE)) * 64;
        store_digit_planes(rowp, (int)(kk & 31), mulmod(val[i], inv, mp), mp);
    }
}

}  // namespace

void compact_free(Compact *c, cudaStream_t s)
{
    dfree(c->kidx, s);
    dfree(c->koff, s);
    dfree(c->planes, s);
    *c = Compact();
}

int sparse_build(const DevCSR &in, const PivotInfo &pi, int L, uint16_t *Adiag, Compact *SA, Compact *SB,
                 const ModP &mp, cudaStream_t s)
{
    const int64_t npiv = pi.npiv, n_d = pi.n_d;
    if (npiv <= 0) return GBLA_OK;
    const int64_t wpr = (npiv + 31) / 32;
    Compact *cs[2] = {SA, SB};
    const int64_t ntiles[2] = {(npiv + TILE - 1) / TILE, (n_d + TILE - 1) / TILE};
    uint32_t *bits[2] = {nullptr, nullptr};
    int32_t *woff[2] = {nullptr, nullptr};
    int64_t *padded[2] = {nullptr, nullptr};
    int rc = GBLA_OK;
    for (int a = 0; a < 2 && rc == GBLA_OK; ++a) {
        cs[a]->ntiles = ntiles[a];
        const size_t words = (size_t)(ntiles[a] > 0 ? ntiles[a] : 1) * (size_t)wpr;
        if ((rc = dalloc_t(&bits[a], words, s)) != GBLA_OK) break;
        if ((rc = dalloc_t(&woff[a], words, s)) != GBLA_OK) break;
        if ((rc = dalloc_t(&padded[a], (size_t)ntiles[a] + 1, s)) != GBLA_OK) break;
        if ((rc = dalloc_t(&cs[a]->koff, (size_t)ntiles[a] + 2, s)) != GBLA_OK) break;
        if (cudaMemsetAsync(bits[a], 0, words * sizeof(uint32_t), s) != cudaSuccess) rc = GBLA_E_CUDA;
    }
    if (rc == GBLA_OK && Adiag &&
        cudaMemsetAsync(Adiag, 0, sizeof(uint16_t) * (size_t)round_up(npiv, L) * (size_t)L, s) != cudaSuccess)
        rc = GBLA_E_CUDA;
    const unsigned warps_grid = (unsigned)((npiv * 32 + 255) / 256);
    if (rc == GBLA_OK) {
        sp_mark_kernel<<<warps_grid, 256, 0, s>>>(npiv, L, pi.piv_row, in.row_ptr, in.col, in.val, pi.colmap,
                                                  pi.inv_lead, Adiag, wpr, bits[0], bits[1], mp);
        if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
    }
    int64_t totals[2] = {0, 0};
    for (int a = 0; a < 2 && rc == GBLA_OK; ++a) {
        if (ntiles[a] <= 0) {
            if (cudaMemsetAsync(cs[a]->koff, 0, sizeof(int64_t), s) != cudaSuccess) rc = GBLA_E_CUDA;
            continue;
        }
        sp_count_kernel<<<(unsigned)ntiles[a], 256, 0, s>>>(wpr, bits[a], woff[a], padded[a]);
        if (launch_check() != cudaSuccess) { rc = GBLA_E_CUDA; break; }
        rc = scan_i64(padded[a], cs[a]->koff, ntiles[a], cs[a]->koff + ntiles[a], s);
    }
    if (rc == GBLA_OK) {
        int64_t h[2] = {0, 0};
        for (int a = 0; a < 2 && rc == GBLA_OK; ++a)
            if (ntiles[a] > 0) rc = readback(&h[a], cs[a]->koff + ntiles[a], sizeof(int64_t), s);
        totals[0] = h[0];
        totals[1] = h[1];
    }
    for (int a = 0; a < 2 && rc == GBLA_OK; ++a) {
        cs[a]->total = totals[a];
        const size_t nk = (size_t)(totals[a] > 0 ? totals[a] : 1);
        if ((rc = dalloc_t(&cs[a]->kidx, nk, s)) != GBLA_OK) break;
        // chunk q (list entries 32 q .. 32 q + 31) is 128 rows of 64 bf16
        // (hi digits of the 32 entries, then lo): 256 plane elements per entry
        const size_t pe = (size_t)(totals[a] > 0 ? totals[a] : 32) * 256;
        if ((rc = dalloc(reinterpret_cast<void **>(&cs[a]->planes), pe * sizeof(__nv_bfloat16), s)) != GBLA_OK)
            break;
        if (cudaMemsetAsync(cs[a]->kidx, 0x7F, nk * sizeof(int32_t), s) != cudaSuccess ||
            cudaMemsetAsync(cs[a]->planes, 0, pe * sizeof(__nv_bfloat16), s) != cudaSuccess) {
            rc = GBLA_E_CUDA;
            break;
        }
        if (ntiles[a] > 0 && totals[a] > 0) {
            sp_list_kernel<<<(unsigned)ntiles[a], 256, 0, s>>>(wpr, bits[a], woff[a], cs[a]->koff, cs[a]->kidx);
            if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
        }
    }
    if (rc == GBLA_OK) {
        sp_values_kernel<<<warps_grid, 256, 0, s>>>(npiv, L, pi.piv_row, in.row_ptr, in.col, in.val, pi.colmap,
                                                    pi.inv_lead, wpr, bits[0], woff[0], SA->koff, SA->planes,
                                                    bits[1], woff[1], SB->koff, SB->planes, mp);
        if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
    }
    for (int a = 0; a < 2; ++a) {
        dfree(bits[a], s);
        dfree(woff[a], s);
        dfree(padded[a], s);
    }
    return rc;
}


namespace {
__global__ void sp_iota_kernel(int32_t *v, int64_t n, int64_t add)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (int32_t)(i + add);
}
__global__ void sp_ones_kernel(uint32_t *v, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = 1u;
}
// One warp per row: row_ptr monotone inside [0, nnz], columns strictly
// increasing in [0, n), values in [1, p).
__global__ void sp_validate_kernel(int64_t m, int64_t n, int64_t nnz, const int64_t *__restrict__ row_ptr,
                                   const int32_t *__restrict__ col, const uint16_t *__restrict__ val, uint32_t p,
                                   uint32_t *err)
{
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= m) return;
    const int64_t b = row_ptr[r], e = row_ptr[r + 1];
    bool bad = (b < 0) || (e < b) || (e > nnz) || (r == 0 && b != 0) || (r == m - 1 && e != nnz);
    if (!bad)
        for (int64_t i = b + lane; i < e; i += 32) {
            const int32_t c = col[i];
            const uint32_t v = val[i];
            if (c < 0 || c >= n || v == 0 || v >= p) bad = true;
            if (i > b && col[i - 1] >= c) bad = true;
        }
    if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) dev_fail(err, DEV_ERR_INVAL);
}
}  // namespace

int compact_from_csr(const DevCSR &S, Compact *out, const ModP &mp, uint32_t *err, cudaStream_t s)
{
    // S as the B block of a matrix whose K rows are all pivot rows with unit
    // leads: piv_row = identity, every column of S maps past the pivots,
    // leading coefficients 1.
    if (S.m > 0) {
        sp_validate_kernel<<<(unsigned)((S.m * 32 + 255) / 256), 256, 0, s>>>(S.m, S.n, S.nnz, S.row_ptr, S.col,
                                                                             S.val, mp.p, err);
        GBLA_CUDA_TRY(launch_check());
        uint32_t herr = 0;
        GBLA_TRY(readback(&herr, err, sizeof(herr), s));
        if (herr) return map_dev_err(herr);
    }
    PivotInfo pi;
    pi.m = S.m;
    pi.n = S.n;
    pi.npiv = S.m;
    pi.n_d = S.n;
    int rc = dalloc_t(&pi.piv_row, (size_t)S.m + 1, s);
    if (rc == GBLA_OK) rc = dalloc_t(&pi.colmap, (size_t)S.n + 1, s);
    if (rc == GBLA_OK) rc = dalloc_t(&pi.inv_lead, (size_t)S.m + 1, s);
    if (rc == GBLA_OK && S.m > 0) {
        sp_iota_kernel<<<(unsigned)((S.m + 255) / 256), 256, 0, s>>>(pi.piv_row, S.m, 0);
        sp_ones_kernel<<<(unsigned)((S.m + 255) / 256), 256, 0, s>>>(pi.inv_lead, S.m);
        if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
        ++g_launches;
    }
    if (rc == GBLA_OK && S.n > 0) {
        sp_iota_kernel<<<(unsigned)((S.n + 255) / 256), 256, 0, s>>>(pi.colmap, S.n, S.m);
        if (launch_check() != cudaSuccess) rc = GBLA_E_CUDA;
    }
    Compact unused;
    if (rc == GBLA_OK) rc = sparse_build(S, pi, 128, nullptr, &unused, out, mp, s);
    compact_free(&unused, s);
    dfree(pi.piv_row, s);
    dfree(pi.colmap, s);
    dfree(pi.inv_lead, s);
    pi = PivotInfo();
    return rc;
}

}  // namespace gbla
