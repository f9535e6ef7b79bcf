// internal.cuh -- host-side interfaces between the library's translation units.
#pragma once

#include "common.cuh"

namespace gbla {

struct GemmCounters {
    double mod_ops = 0;      // algorithmic modular multiply-adds of the products
    double last_ops = 0;     // the same for the last product
    long launches = 0;
    long tc_launches = 0;
};

int device_sm_count();

// Raster group of the gathered product: a per-thread override (0 = none) and
// the default (environment switch GBLA_GATHER_GROUP_M, else the dense
// product's).
extern thread_local int g_gather_group_m_override;
int gather_group_m_default();

// One problem of a grouped product: rows a_row0.. of the A plane set times
// rows b_row0.. of the B plane set (the same K for all problems), into C
// rows c_rows[0..M) at columns c_col0 .. c_col0 + N.  tile_off = exclusive
// prefix of the problems' tile counts (ceil(M/128) * ceil(N/128)); entry
// [nprob] holds the total.
struct GroupProb {
    int32_t a_row0, b_row0, M, N;
    int64_t c_col0;
    const int32_t *c_rows;
    int64_t tile_off;
};

// Per-launch timing of the tensor-core kernels on the calling thread (kind 0:
// the dense product modgemm_tc_kernel, 1: the gathered product), opt-in per
// reduction: between begin and end every launch is bracketed by events on its
// stream, and the dense product adds valid rows x valid columns x K run of
// each tile to *tc_work_dev (device counter, may be null).  end() needs the
// stream synchronised.
struct KernelTimeTotals {
    double ms[2] = {0, 0};
    int64_t launches[2] = {0, 0};
};
void kernel_times_begin(unsigned long long *tc_work_dev);
void kernel_times_end(KernelTimeTotals *t);

// True on a device with the tcgen05 tensor-core path (compute capability 10.3).
bool tc_supported();

// GBLA_OK on a compute capability 10.3 device (and the memory pool set up),
// else GBLA_E_UNSUPPORTED.
int check_device();

// GBLA_* code of a device status word (DEV_ERR_* bits).
int map_dev_err(uint32_t e);

// Device-to-host copy of `bytes` into pageable host memory `dst` through a
// page-locked scratch buffer of the calling thread; synchronises stream s.
int readback(void *dst, const void *src, size_t bytes, cudaStream_t s);

// Releases what the reductions keep per host thread (a side stream and its
// events, the page-locked readback buffer); for worker threads about to exit.
void release_thread_resources();

// Product written as A-operand digit planes: Out[out_row0 + m, out_col0 + n] <-
// (A*B)[m, n] mod p (tensor-core variant only).  A may be a 4-plane set, read
// as its first two planes.
int modgemm_to_planes(const Planes &A, int64_t a_row0, const Planes &B, int64_t b_row0, const Planes &Out,
                      int64_t out_col0, int64_t M, int64_t N, int64_t K, const ModP &mp, uint32_t *err,
                      cudaStream_t s, GemmCounters *ctr, int64_t out_row0 = 0);

// K-compacted sparse operand S (npiv rows) of the gathered product, built by
// sparse_build (sparse.cu): for 128-column tile t, the rows with a nonzero in
// the tile are kidx[koff[t] .. koff[t+1]) (ascending, padded with KIDX_PAD to
// a multiple of 128), and the tile restricted to them is stored as B-operand
// digit planes, chunk-major (list entries 32 q .. 32 q + 31: 128 rows of 64
// bf16, hi digits then lo, at planes + 128 * 64 * q).
constexpr int32_t KIDX_PAD = 0x7F7F7F7F;
struct Compact {
    int64_t ntiles = 0;        // column tiles
    int64_t total = 0;         // list entries of all tiles (multiple of 128)
    int32_t *kidx = nullptr;   // [total]
    int64_t *koff = nullptr;   // [ntiles + 1]
    __nv_bfloat16 *planes = nullptr;   // [total / 32 chunks][128 rows][128 bf16] = total * 512
};
void compact_free(Compact *c, cudaStream_t s);

// Gathered product C[r, c] <- (C[r, c] + sign * sum_j X[r, j] * S[j, c]) mod p
// for rows r < M and columns c < N of C, c in tile nt0 + c / 128 of S; X is
// read from the A-operand plane set XT of its transpose (row j = column j of
// X, K = r).  Every list entry j >= xt_rows must be padding (KIDX_PAD, whose
// rows of S are zero): such entries read row 0 of XT.  With row_lead (device,
// ascending absolute lead of each row of X) a row tile skips the list entries
// left of its first row's lead.  Tensor-core variant only (p >= 8).
// With exec (device, optional), adds the list entries times row tiles the
// launch runs through (executed multiply-adds = exec * 128 * 128).
int modgemm_gather(const Compact &S, int64_t nt0, const Planes &XT, int64_t xt_rows, uint16_t *C, int64_t ldc,
                   int64_t M, int64_t N, int sign, const int32_t *row_lead, const ModP &mp, uint32_t *err,
                   cudaStream_t s, GemmCounters *ctr, unsigned long long *exec = nullptr);
// Panel application of one echelon wave (solve.cu), fused: for every job q
// (a panel with pivot rows S, t of them) and every 128-column block of D from
// the job's first column, D[rows_q] += A_q * D[S]_old restricted to the block,
// where A_q (M rows, K = 128, zero past t) is the job's stacked multipliers
// (G - I for the new pivot rows, then -H G for the dependent candidates) as a
// 2-plane A-operand set and rows_q = rowmap[a_row0 .. a_row0 + M) the rows of
// D they update (the pivot rows S, then the candidates).  D[S] is read in its
// u16 form, once per block, and turned into digit planes on chip; both updates
// of a block read it before either writes (rows of different jobs are
// disjoint).  jobs[q].item_off: prefix of the jobs' work items (column blocks
// of jobs with M > 0); jobs[njobs].item_off = the total.
struct PaJob {
    int64_t a_row0;       // first row of the job's block of A (and of rowmap)
    int64_t col0;         // first column of D the job updates
    int64_t item_off;     // work items of the jobs before
    const int32_t *srows; // the job's pivot rows of D (K of the product)
    int32_t M;            // rows of the job's block
    int32_t t;            // pivot rows (K used, <= 128)
    int32_t nc;           // columns of D from col0
    int32_t pad;
};
int panel_apply(const Planes &A, const PaJob *jobs, int njobs, const int32_t *rowmap, uint16_t *D, int64_t ldd,
                int64_t n, const ModP &mp, uint32_t *err, cudaStream_t s);

// Grouped product C[c_rows, c_col0:] += sign * A_p * B_p^T for every problem
// p, one launch (see GroupProb).
int modgemm_grouped(const Planes &A, const Planes &B, const GroupProb *probs, int nprob, int64_t K, uint16_t *C,
                    int64_t ldc, int sign, const ModP &mp, int variant, uint32_t *err, cudaStream_t s,
                    GemmCounters *ctr);

// One whole reduction on stream s (the body of gbla_reduce_ex; arguments
// already checked for null pointers and p).  Thread-safe: calls from
// different host threads on different streams run concurrently.
int reduce_impl(const gbla_csr_in *in, uint32_t p, const gbla_options *opt, cudaStream_t s, gbla_csr_out *out,
                int64_t *rank_out, gbla_stats *stats);
bool is_prime(uint32_t p);

// C <- (C + sign * A * B^T) mod p, A an A-operand plane set (2 planes,
// rows a_row0.., K from a_k0), B a B-operand plane set (4 planes, rows
// b_row0.., K from b_k0).  With c_rows, product row r updates C row
// c_rows[r] (a negative entry skips the row).
// With row_lead (ascending, absolute K index of each A row's first nonzero;
// a_row0 must be 0), each 128-row tile starts at its first row's lead.  K
// beyond the logical range must read zeros (zero padding) when K is not a
// multiple of 64.
int modgemm(const Planes &A, int64_t a_row0, int64_t a_k0, const Planes &B, int64_t b_row0, int64_t b_k0,
            uint16_t *C, int64_t ldc, int64_t M, int64_t N, int64_t K, int sign, const ModP &mp, int variant,
            uint32_t *err, cudaStream_t s, GemmCounters *ctr, const int32_t *c_rows = nullptr,
            const int32_t *row_lead = nullptr, const int32_t *row_lead_host = nullptr);

// The same product on the legacy warp-level tensor-core instructions
// (modgemm_alt.cu): variant GBLA_GEMM_FP64 (mma.sync f64, exact over k-blocks
// of 2^23) or GBLA_GEMM_U8 (mma.sync u8 -> s32 on the bytes of the residues,
// exact over k-blocks of 2^14).  Reads planes 0 and 1 of both sets; a_k0 and
// b_k0 multiples of 32; with row_lead (ascending, product-row indexed) each
// 64-row tile starts at its first row's lead.
int modgemm_alt(const Planes &A, int64_t a_row0, int64_t a_k0, const Planes &B, int64_t b_row0, int64_t b_k0,
                uint16_t *C, int64_t ldc, int64_t M, int64_t N, int64_t K, int sign, const ModP &mp, int variant,
                cudaStream_t s, const int32_t *c_rows, const int32_t *row_lead);

// C <- (C + sign * A * B) mod p for residues of a prime p < 2^31 (uint32,
// row-major, device): four balanced 8-bit digits per residue in bf16 and
// seven fp32 TMEM accumulators (modgemm.cu); synchronises s.
int modmatmul32(int64_t M, int64_t N, int64_t K, const uint32_t *A, int64_t lda, const uint32_t *B, int64_t ldb,
                uint32_t *C, int64_t ldc, uint32_t p, int sign, cudaStream_t s);

// Issue-rate microbenchmark of the FP64 or U8 mma.sync pipe (ops of the
// instruction per second, in units of 1e12), timed with events on s.
int pipe_peak(int variant, double *tops, cudaStream_t s);

// Test hook: a product whose loads are withheld, so that its bounded waits
// expire; sets DEV_ERR_TIMEOUT in *err (see modgemm.cu).
int modgemm_withheld_loads(uint32_t *err, cudaStream_t s);

// u16 -> digit planes (see modgemm.cu).
int to_planes(const Planes &dst, int64_t R, int64_t Kc, const uint16_t *src, int64_t lds, int64_t col_off,
              bool transposed, const int32_t *rgather, const int32_t *cgather, const ModP &mp, cudaStream_t s,
              const int32_t *zero_if = nullptr, bool k_le_r_only = false, int64_t dst_col0 = 0);

// One-shot allocation fault injection (see gbla.cu): true when this
// allocation is to fail.
bool inject_alloc_fault();
// cudaMalloc for memory that leaves the library (results), with fault
// injection.
cudaError_t out_malloc(void **ptr, size_t bytes);

// Stream-ordered device allocation helpers (memory pool of the device).
int dalloc(void **ptr, size_t bytes, cudaStream_t s);
void dfree(void *ptr, cudaStream_t s);

template <typename T>
inline int dalloc_t(T **ptr, size_t count, cudaStream_t s) {
    return dalloc(reinterpret_cast<void **>(ptr), count * sizeof(T) + 16, s);
}

// A scratch device array owned by one scope: released (stream-ordered on s)
// on every exit from it, early error returns included.
template <typename T>
struct DevTemp {
    T *p = nullptr;
    cudaStream_t s = nullptr;
    explicit DevTemp(cudaStream_t st) : s(st) {}
    DevTemp(const DevTemp &) = delete;
    DevTemp &operator=(const DevTemp &) = delete;
    ~DevTemp() { dfree(p, s); }
    int alloc(size_t count) { return dalloc_t(&p, count, s); }
    operator T *() const { return p; }
};

int planes_alloc(Planes *pl, int64_t rows, int64_t k, int nplanes, cudaStream_t s);
void planes_free(Planes *pl, cudaStream_t s);

// Exclusive prefix sum of n int64 values (in may equal out); *total_dev (a
// device pointer, may be null) receives the sum.
int scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total_dev, cudaStream_t s);

}  // namespace gbla
