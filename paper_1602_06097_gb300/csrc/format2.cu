// format2.cu -- the paper's Format 2 matrix files (GBLA paper Sec. 3.2,
// Table 2) decoded on the device into the reduction's CSR input.
//
// Layout (little-endian): u32 b (bits 0-2: coefficient type, b = u | v << 1,
// 8 * 2^v bits, u = 1 unsigned as in the section's worked example; higher bits
// a version, ignored), u32 m, u32 n, u64 p, u64 nnz, u32 rows[m] (row
// lengths), u32 polmap[m] (row i carries polynomial polmap[i]'s
// coefficients), u64 k, u64 colid[k] (the rows' columns, row after row: a run
// of s >= 2 consecutive columns from f is the pair f, s; a lone column f is
// f | 2^31), u32 pnb, u64 pnnz, u32 prow[pnb] (polynomial lengths), the
// polynomials' coefficients pdata[pnnz] one after the other.
//
// The host reads the fixed fields and the section offsets (each checked
// against the file size) and copies the five sections into aligned device
// buffers.  The rest runs in parallel:
//   1. row_ptr and the polynomial starts are exclusive scans of the row and
//      polynomial lengths;
//   2. every column entry is classified without a sequential pass: with g the
//      inclusive count of lone (masked) entries and last[e] the position of
//      the g[e]-th lone entry (scattered), an unmasked entry is a run start
//      when e - last[e] is odd and a run length when it is even;
//   3. entries emit 1 (lone), s (run start, s read from the next entry) or 0
//      columns; off = the exclusive scan of those counts;
//   4. entry e writes positions off[e] .. off[e] + count - 1: the lone
//      column, or the run start plus q - off[e] (a warp per 32 entries, the
//      lanes writing consecutive positions);
//   5. checks: a run stays inside the row of its first column (no row starts
//      strictly inside it), columns rise within a row and stay below n;
//   6. row i copies polynomial polmap[i]'s coefficients (one warp per row),
//      reduced mod p (signed types too); a zero residue is rejected.
// Violations set DEV_ERR_INVAL in a device status word: GBLA_E_INVAL.
#include <string.h>

#include "common.cuh"
#include "internal.cuh"

namespace gbla {
namespace {

enum : int8_t { F2_LONE = 0, F2_START = 1, F2_LEN = 2 };

__global__ void f2_widen_kernel(const uint32_t *__restrict__ in, int64_t *__restrict__ out, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i];
}

// masked flag of each column entry; bits 32-63 must be zero
__global__ void f2_mask_kernel(const uint64_t *__restrict__ colid, int64_t k, int64_t *__restrict__ g,
                               uint32_t *err)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= k) return;
    const uint64_t x = colid[e];
    if (x >> 32) dev_fail(err, DEV_ERR_INVAL);
    g[e] = (int64_t)((x >> 31) & 1u);
}

// gex = exclusive count of lone entries: lone entry e is the (gex[e]+1)-th
__global__ void f2_last_kernel(const uint64_t *__restrict__ colid, int64_t k, const int64_t *__restrict__ gex,
                               int64_t *__restrict__ lastm)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < k && ((colid[e] >> 31) & 1u)) lastm[gex[e] + 1] = e;
}

__global__ void f2_count_kernel(const uint64_t *__restrict__ colid, int64_t k, const int64_t *__restrict__ gex,
                                const int64_t *__restrict__ lastm, int64_t *__restrict__ cnt,
                                int8_t *__restrict__ role, uint32_t *err)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= k) return;
    const uint64_t x = colid[e];
    if ((x >> 31) & 1u) {
        role[e] = F2_LONE;
        cnt[e] = 1;
        return;
    }
    const int64_t incl = gex[e];   // lone entries before e (e itself is not one)
    const int64_t last = incl > 0 ? lastm[incl] : -1;
    if ((e - last) & 1) {
        role[e] = F2_START;
        cnt[e] = 0;
        if (e + 1 >= k || ((colid[e + 1] >> 31) & 1u)) {   // a run start without its length
            dev_fail(err, DEV_ERR_INVAL);
            return;
        }
        const uint64_t s = colid[e + 1];
        if (s < 2 || s >= (1ull << 31)) {
            dev_fail(err, DEV_ERR_INVAL);
            return;
        }
        cnt[e] = (int64_t)s;
    } else {
        role[e] = F2_LEN;
        cnt[e] = 0;
    }
}

__global__ void f2_total_check_kernel(const int64_t *__restrict__ total, int64_t nnz, const int64_t *__restrict__ ptot,
                                      int64_t pnnz, uint32_t *err)
{
    if (*total != nnz || (ptot && *ptot != pnnz)) dev_fail(err, DEV_ERR_INVAL);
}

// first position of every non-empty row (the lengths may not add up to nnz
// in a malformed file: that is reported elsewhere, here nothing past nnz)
__global__ void f2_row_flags_kernel(const int64_t *__restrict__ row_ptr, int64_t m, int64_t nnz,
                                    int8_t *__restrict__ flag)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < m && row_ptr[r + 1] > row_ptr[r] && row_ptr[r] < nnz) flag[row_ptr[r]] = 1;
}

// Columns of the rows: one warp per 32 consecutive column entries, which it
// expands one after the other, the lanes writing 32 consecutive positions of
// the entry's run at a time (coalesced).  An entry covers positions
// off[e] .. off[e] + cnt[e] (a lone column one, a run start s, a run length
// none).  A run must not cross into the next row (flag marks row starts) and
// no column may reach n.  Skipped when an earlier check already failed (the
// totals then need not match nnz).
__global__ void f2_expand_kernel(const uint64_t *__restrict__ colid, const int64_t *__restrict__ off,
                                 const int64_t *__restrict__ cnt, const int8_t *__restrict__ role, int64_t k,
                                 const int8_t *__restrict__ flag, int64_t nnz, int64_t n, int32_t *__restrict__ col,
                                 uint32_t *err)
{
    if (*(volatile uint32_t *)err) return;
    const int lane = threadIdx.x & 31;
    const int64_t e0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32;
    if (e0 >= k) return;
    const int64_t e = e0 + lane;
    const bool has = e < k;
    const uint64_t x_l = has ? colid[e] : 0;
    const int64_t o_l = has ? off[e] : 0, c_l = has ? cnt[e] : 0;
    const int r_l = has ? (int)role[e] : (int)F2_LEN;
    const int last = (int)min((int64_t)32, k - e0);
    for (int i = 0; i < last; ++i) {
        const uint64_t x = __shfl_sync(0xffffffffu, x_l, i);
        const int64_t o = __shfl_sync(0xffffffffu, o_l, i), c = __shfl_sync(0xffffffffu, c_l, i);
        const int r = __shfl_sync(0xffffffffu, r_l, i);
        if (r == F2_LEN || c == 0) continue;
        if (c < 0 || o < 0 || o + c > nnz) {
            if (lane == 0) dev_fail(err, DEV_ERR_INVAL);
            return;
        }
        const int64_t base = r == F2_LONE ? (int64_t)(x & 0x7FFFFFFFull) : (int64_t)x;
        if (base + c > n) {
            if (lane == 0) dev_fail(err, DEV_ERR_INVAL);
            return;
        }
        for (int64_t t = lane; t < c; t += 32) {
            const int64_t q = o + t;
            if (t > 0 && flag[q]) dev_fail(err, DEV_ERR_INVAL);   // the run crosses into the next row
            col[q] = (int32_t)(base + t);
        }
    }
}

__global__ void f2_order_kernel(const int32_t *__restrict__ col, const int8_t *__restrict__ flag, int64_t nnz,
                                uint32_t *err)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q + 1 < nnz && !flag[q + 1] && col[q + 1] <= col[q]) dev_fail(err, DEV_ERR_INVAL);
}

template <typename T>
__device__ __forceinline__ uint32_t f2_residue(T x, uint32_t p)
{
    if (T(-1) < T(0)) {   // signed
        int64_t v = (int64_t)x % (int64_t)p;
        return (uint32_t)(v < 0 ? v + p : v);
    }
    return (uint32_t)((uint64_t)x % p);
}

// one warp per row
template <typename T>
__global__ void f2_values_kernel(const int64_t *__restrict__ row_ptr, const uint32_t *__restrict__ polmap,
                                 int64_t m, int64_t nnz, const uint32_t *__restrict__ prow,
                                 const int64_t *__restrict__ pstart, int64_t pnb, int64_t pnnz,
                                 const T *__restrict__ pdata, uint32_t p, uint16_t *__restrict__ val, uint32_t *err)
{
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= m) return;
    const int64_t j = polmap[r];
    const int64_t len = row_ptr[r + 1] - row_ptr[r];
    // lengths that disagree with nnz or pnnz (reported elsewhere) touch nothing
    if (j >= pnb || (int64_t)prow[j] != len || row_ptr[r + 1] > nnz || pstart[j] + len > pnnz) {
        if (lane == 0) dev_fail(err, DEV_ERR_INVAL);
        return;
    }
    const T *src = pdata + pstart[j];
    uint16_t *dst = val + row_ptr[r];
    for (int64_t t = lane; t < len; t += 32) {
        const uint32_t v = f2_residue(src[t], p);
        if (v == 0) dev_fail(err, DEV_ERR_INVAL);
        dst[t] = (uint16_t)v;
    }
}

struct F2Rows {
    const int64_t *row_ptr;
    const uint32_t *polmap;
    int64_t m, nnz;
    const uint32_t *prow;
    const int64_t *pstart;
    int64_t pnb, pnnz;
};

template <typename T>
int f2_values(const F2Rows &R, const void *pdata, uint32_t p, uint16_t *val, uint32_t *err, cudaStream_t s)
{
    if (R.m <= 0) return GBLA_OK;
    f2_values_kernel<T><<<(unsigned)((R.m * 32 + 255) / 256), 256, 0, s>>>(
        R.row_ptr, R.polmap, R.m, R.nnz, R.prow, R.pstart, R.pnb, R.pnnz, static_cast<const T *>(pdata), p, val, err);
    GBLA_CUDA_TRY(launch_check());
    return GBLA_OK;
}

bool read_field(const uint8_t *f, size_t bytes, size_t off, void *dst, size_t size)
{
    if (off > bytes || size > bytes - off) return false;
    memcpy(dst, f + off, size);
    return true;
}

unsigned blocks(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace
}  // namespace gbla

using namespace gbla;

extern "C" int gbla_decode_format2(const void *file, size_t bytes, void *stream, gbla_csr_out *out, uint32_t *p_out)
{
    return gbla_decode_format2_ex(file, bytes, stream, out, p_out, nullptr);
}

extern "C" int gbla_decode_format2_ex(const void *file, size_t bytes, void *stream, gbla_csr_out *out,
                                      uint32_t *p_out, double *decode_ms)
{
    if (decode_ms) *decode_ms = -1.0;
    if (!out) return GBLA_E_INVAL;
    memset(out, 0, sizeof(*out));
    if (!file || !p_out) return GBLA_E_INVAL;
    const uint8_t *f = static_cast<const uint8_t *>(file);
    // ---- fixed fields and section offsets, each checked against the size
    uint32_t b = 0, m32 = 0, n32 = 0, pnb32 = 0;
    uint64_t p64 = 0, nnz64 = 0, k64 = 0, pnnz64 = 0;
    if (!read_field(f, bytes, 0, &b, 4) || !read_field(f, bytes, 4, &m32, 4) || !read_field(f, bytes, 8, &n32, 4) ||
        !read_field(f, bytes, 12, &p64, 8) || !read_field(f, bytes, 20, &nnz64, 8))
        return GBLA_E_INVAL;
    const size_t m = m32, rows_off = 28, polmap_off = rows_off + 4 * m, k_off = polmap_off + 4 * m;
    if (m >= (1u << 31) || n32 >= (1u << 31) || p64 < 2 || p64 >= 65536u || nnz64 >= (1ull << 40))
        return GBLA_E_INVAL;
    if (!read_field(f, bytes, k_off, &k64, 8) || k64 > bytes / 8) return GBLA_E_INVAL;
    const size_t colid_off = k_off + 8, pnb_off = colid_off + 8 * (size_t)k64;
    if (!read_field(f, bytes, pnb_off, &pnb32, 4) || !read_field(f, bytes, pnb_off + 4, &pnnz64, 8))
        return GBLA_E_INVAL;
    const size_t prow_off = pnb_off + 12, pdata_off = prow_off + 4 * (size_t)pnb32;
    const int v = (b >> 1) & 3;
    const size_t tsize = (size_t)1 << v;
    if (pdata_off > bytes || pnnz64 > (bytes - pdata_off) / tsize || pdata_off + tsize * pnnz64 != bytes)
        return GBLA_E_INVAL;
    GBLA_TRY(check_device());
    const int64_t n = n32, nnz = (int64_t)nnz64, k = (int64_t)k64, pnb = pnb32, pnnz = (int64_t)pnnz64;
    const uint32_t p = (uint32_t)p64;
    cudaStream_t s = (cudaStream_t)stream;

    uint32_t *rows32 = nullptr, *polmap32 = nullptr, *prow32 = nullptr, *err = nullptr;
    uint64_t *colid = nullptr;
    void *pdata = nullptr;
    int64_t *row_ptr = nullptr, *pstart = nullptr, *g = nullptr, *lastm = nullptr, *cnt = nullptr, *off = nullptr;
    int64_t *total = nullptr;
    int8_t *role = nullptr, *flag = nullptr;
    int32_t *col = nullptr;
    uint16_t *val = nullptr;
    uint32_t err_h = 0;
    int rc = GBLA_OK;
#define F2STEP(expr)                         \
    do {                                     \
        if (rc == GBLA_OK) rc = (expr);      \
    } while (0)
#define F2CUDA(expr)                                                                \
    do {                                                                            \
        if (rc == GBLA_OK) {                                                        \
            const cudaError_t _e = (expr);                                          \
            if (_e != cudaSuccess) rc = _e == cudaErrorMemoryAllocation ? GBLA_E_NOMEM : GBLA_E_CUDA; \
        }                                                                           \
    } while (0)
    F2STEP(dalloc_t(&rows32, m + 1, s));
    F2STEP(dalloc_t(&polmap32, m + 1, s));
    F2STEP(dalloc_t(&colid, (size_t)k + 1, s));
    F2STEP(dalloc_t(&prow32, (size_t)pnb + 1, s));
    F2STEP(dalloc(&pdata, tsize * (size_t)pnnz + 16, s));
    F2STEP(dalloc_t(&pstart, (size_t)pnb + 1, s));
    F2STEP(dalloc_t(&g, (size_t)k + 1, s));
    F2STEP(dalloc_t(&lastm, (size_t)k + 2, s));
    F2STEP(dalloc_t(&cnt, (size_t)k + 1, s));
    F2STEP(dalloc_t(&off, (size_t)k + 1, s));
    F2STEP(dalloc_t(&total, 2, s));
    F2STEP(dalloc_t(&role, (size_t)k + 1, s));
    F2STEP(dalloc_t(&flag, (size_t)nnz + 1, s));
    F2STEP(dalloc_t(&err, 1, s));
    F2CUDA(out_malloc((void **)&row_ptr, sizeof(int64_t) * (m + 1)));
    F2CUDA(out_malloc((void **)&col, sizeof(int32_t) * (size_t)(nnz + 1)));
    F2CUDA(out_malloc((void **)&val, sizeof(uint16_t) * (size_t)(nnz + 1)));
    F2CUDA(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
    F2CUDA(cudaMemsetAsync(flag, 0, (size_t)nnz + 1, s));
    F2CUDA(cudaMemsetAsync(total, 0, 2 * sizeof(int64_t), s));
    // the sections
    if (m) F2CUDA(cudaMemcpyAsync(rows32, f + rows_off, 4 * m, cudaMemcpyHostToDevice, s));
    if (m) F2CUDA(cudaMemcpyAsync(polmap32, f + polmap_off, 4 * m, cudaMemcpyHostToDevice, s));
    if (k) F2CUDA(cudaMemcpyAsync(colid, f + colid_off, 8 * (size_t)k, cudaMemcpyHostToDevice, s));
    if (pnb) F2CUDA(cudaMemcpyAsync(prow32, f + prow_off, 4 * (size_t)pnb, cudaMemcpyHostToDevice, s));
    if (pnnz) F2CUDA(cudaMemcpyAsync(pdata, f + pdata_off, tsize * (size_t)pnnz, cudaMemcpyHostToDevice, s));
    // the decode proper (device work after the copies) is event-timed on request
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (decode_ms && rc == GBLA_OK) {
        F2CUDA(cudaEventCreate(&ev[0]));
        F2CUDA(cudaEventCreate(&ev[1]));
        F2CUDA(cudaEventRecord(ev[0], s));
    }
    // 1. scans of the lengths
    if (m && rc == GBLA_OK) {
        f2_widen_kernel<<<blocks((int64_t)m), 256, 0, s>>>(rows32, row_ptr, (int64_t)m);
        F2CUDA(launch_check());
    }
    F2STEP(scan_i64(row_ptr, row_ptr, (int64_t)m, row_ptr + m, s));
    if (pnb && rc == GBLA_OK) {
        f2_widen_kernel<<<blocks(pnb), 256, 0, s>>>(prow32, pstart, pnb);
        F2CUDA(launch_check());
    }
    F2STEP(scan_i64(pstart, pstart, pnb, pstart + pnb, s));
    // 2.-3. roles, counts and offsets of the column entries
    if (k && rc == GBLA_OK) {
        f2_mask_kernel<<<blocks(k), 256, 0, s>>>(colid, k, g, err);
        F2CUDA(launch_check());
    }
    F2STEP(scan_i64(g, g, k, nullptr, s));
    if (k && rc == GBLA_OK) {
        f2_last_kernel<<<blocks(k), 256, 0, s>>>(colid, k, g, lastm);
        F2CUDA(launch_check());
    }
    if (k && rc == GBLA_OK) {
        f2_count_kernel<<<blocks(k), 256, 0, s>>>(colid, k, g, lastm, cnt, role, err);
        F2CUDA(launch_check());
    }
    F2STEP(scan_i64(cnt, off, k, total, s));
    if (rc == GBLA_OK) {
        f2_total_check_kernel<<<1, 1, 0, s>>>(total, nnz, pstart + pnb, pnnz, err);
        F2CUDA(launch_check());
    }
    if (rc == GBLA_OK) {
        f2_total_check_kernel<<<1, 1, 0, s>>>(row_ptr + m, nnz, nullptr, 0, err);
        F2CUDA(launch_check());
    }
    // 4.-5. columns and their checks
    if (m && rc == GBLA_OK) {
        f2_row_flags_kernel<<<blocks((int64_t)m), 256, 0, s>>>(row_ptr, (int64_t)m, nnz, flag);
        F2CUDA(launch_check());
    }
    if (nnz && k && rc == GBLA_OK) {
        f2_expand_kernel<<<(unsigned)((k + 255) / 256), 256, 0, s>>>(colid, off, cnt, role, k, flag, nnz, n, col,
                                                                     err);
        F2CUDA(launch_check());
    }
    if (nnz && rc == GBLA_OK) {
        f2_order_kernel<<<blocks(nnz), 256, 0, s>>>(col, flag, nnz, err);
        F2CUDA(launch_check());
    }
    // 6. coefficients
    if (rc == GBLA_OK) {
        const F2Rows R{row_ptr, polmap32, (int64_t)m, nnz, prow32, pstart, pnb, pnnz};
        const bool sgn = (b & 1) == 0;
        switch (v) {
        case 0: rc = sgn ? f2_values<int8_t>(R, pdata, p, val, err, s) : f2_values<uint8_t>(R, pdata, p, val, err, s); break;
        case 1: rc = sgn ? f2_values<int16_t>(R, pdata, p, val, err, s) : f2_values<uint16_t>(R, pdata, p, val, err, s); break;
        case 2: rc = sgn ? f2_values<int32_t>(R, pdata, p, val, err, s) : f2_values<uint32_t>(R, pdata, p, val, err, s); break;
        default: rc = sgn ? f2_values<int64_t>(R, pdata, p, val, err, s) : f2_values<uint64_t>(R, pdata, p, val, err, s); break;
        }
    }
    if (ev[1] && rc == GBLA_OK) F2CUDA(cudaEventRecord(ev[1], s));
    F2STEP(readback(&err_h, err, sizeof(uint32_t), s));
    if (rc == GBLA_OK) rc = map_dev_err(err_h);
    if (ev[1] && rc == GBLA_OK) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess) *decode_ms = ms;
    }
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    dfree(rows32, s);
    dfree(polmap32, s);
    dfree(colid, s);
    dfree(prow32, s);
    dfree(pdata, s);
    dfree(pstart, s);
    dfree(g, s);
    dfree(lastm, s);
    dfree(cnt, s);
    dfree(off, s);
    dfree(total, s);
    dfree(role, s);
    dfree(flag, s);
    dfree(err, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == GBLA_OK) rc = GBLA_E_CUDA;
    if (rc != GBLA_OK) {
        cudaGetLastError();
        if (row_ptr) cudaFree(row_ptr);
        if (col) cudaFree(col);
        if (val) cudaFree(val);
        return rc;
    }
    out->nrows = (int64_t)m;
    out->ncols = n;
    out->nnz = nnz;
    out->row_ptr = row_ptr;
    out->col = col;
    out->val = val;
    out->on_device = 1;
    *p_out = p;
    return GBLA_OK;
#undef F2STEP
#undef F2CUDA
}
