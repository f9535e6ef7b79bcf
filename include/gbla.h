/*
 * gbla.h -- C ABI of the GB300 (sm_103a) Faugere-Lachartre reduction.
 *
 * Problem (GBLA paper, arXiv 1602.06097, Sec. 3.1 and Sec. 4.1): M is an
 * m x n matrix over GF(p), p a prime < 2^16, stored as CSR with uint16
 * coefficients and int32 column indices, rows = polynomials, columns =
 * monomials in decreasing monomial order (the layout of the paper's binary
 * Format 1, Table 2).  The library returns either
 *   - want_reduced = 1: the reduced row echelon form RREF(M) (FL steps 1-5 and
 *     the second FL pass on the right block, Sec. 4.1), or
 *   - want_reduced = 0: the echelon form of the new order of operations
 *     (Alg. 2, Sec. 4.3): the chosen pivot rows of M normalised to a leading
 *     1, plus the reduced echelon form of the Schur complement D - C A^-1 B.
 * In both cases rows are sorted by pivot column (leftmost nonzero, always 1),
 * zero rows are dropped, and columns are back in the input (monomial) order
 * (FL step 5).  rank(M) = number of rows returned.  Pivot rows are chosen per
 * leading column as the row with the fewest nonzeros, ties to the smaller row
 * index (the paper's "keep A as sparse as possible", Sec. 3.1).
 *
 * All arithmetic is exact modular integer arithmetic.
 *
 * Threading: calls are independent and thread-safe; calls on different
 * streams run their device work concurrently (GBLA_SERIALIZE=1 in the
 * environment makes them follow one another).  Errors are returned as codes,
 * never thrown.
 */
#ifndef GBLA_H
#define GBLA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---------------------------------------------------- */
#define GBLA_OK 0
#define GBLA_E_INVAL 1       /* bad argument or malformed matrix (see gbla_csr_in) */
#define GBLA_E_NOMEM 2       /* device or host allocation failed */
#define GBLA_E_CUDA 3        /* a CUDA runtime/driver call failed */
#define GBLA_E_TIMEOUT 4     /* a bounded device-side wait expired; the context stays usable */
#define GBLA_E_INTERNAL 5    /* internal consistency check failed */
#define GBLA_E_UNSUPPORTED 6 /* no sm_103a device, or an option this build cannot honour */
#define GBLA_E_CANCELLED 7   /* a server request was cancelled before it ran */

/* ---- matrix types ---------------------------------------------------- */
/* Input matrix, borrowed (never modified, never freed by the library).
 * row_ptr[nrows+1] with row_ptr[0] = 0 and row_ptr[nrows] = nnz, monotone;
 * col[nnz] strictly increasing inside each row, 0 <= col < ncols;
 * val[nnz] in [1, p) (no explicit zeros).  Violations give GBLA_E_INVAL.
 * The pointers are host pointers, or device pointers when
 * gbla_options.device_ptrs = 1. */
typedef struct {
    int64_t nrows, ncols, nnz;
    const int64_t *row_ptr;
    const int32_t *col;
    const uint16_t *val;
} gbla_csr_in;

/* Result matrix, owned by the library; release with gbla_free().  nrows is
 * the rank.  on_device = 1 when the arrays are device memory (requested with
 * gbla_options.device_ptrs = 1), else host memory.  Host results are
 * page-locked; gbla_free returns them to a library cache (at most
 * GBLA_HOST_CACHE_MB megabytes, default 8192) that later results reuse. */
typedef struct {
    int64_t nrows, ncols, nnz;
    int64_t *row_ptr;
    int32_t *col;
    uint16_t *val;
    int on_device;
} gbla_csr_out;

#define GBLA_GEMM_AUTO 0     /* tensor-core path where it applies */
#define GBLA_GEMM_TCGEN05 1  /* bf16 8-bit digits on tcgen05.mma, fp32 TMEM accumulators */
#define GBLA_GEMM_SIMT 2     /* exact int64 CUDA-core kernel (reference variant) */
/* Measured alternatives of the Schur update D <- D - X*B (Sec. 4.3) on the
 * legacy warp-level tensor-core instructions.  In gbla_options they select the
 * dense path with the Schur update on that pipe (every other product on
 * tcgen05; needs p >= 8); gbla_modmatmul runs the whole product on it. */
#define GBLA_GEMM_FP64 3     /* mma.sync m8n8k4 f64 on balanced residues: exact while
                                k-blocks of 2^23 keep sums below 2^53 (delayed reduction) */
#define GBLA_GEMM_U8 4       /* mma.sync m16n8k32 u8 x u8 -> s32 on the residues' bytes,
                                three accumulators, exact over k-blocks of 2^14 */

/* How C*A^-1 and the Schur update treat the pivot rows (Sec. 4.1, Table 4's
 * block densities). */
#define GBLA_PATH_AUTO 0    /* sparse where the tensor-core path applies, else dense */
#define GBLA_PATH_DENSE 1   /* A and B materialised densely, dense tensor-core products */
#define GBLA_PATH_SPARSE 2  /* A and B kept sparse: products with K compacted per
                               128-column tile to the rows that meet it (needs
                               the tensor-core variant, p >= 8) */

typedef struct {
    int want_reduced;  /* 1: RREF(M); 0: echelon form of the new order */
    int gemm_variant;  /* GBLA_GEMM_AUTO, _TCGEN05 or _SIMT: every dense modular product;
                          GBLA_GEMM_FP64 or _U8: the Schur update only (dense path) */
    int device_ptrs;   /* 1: input and output arrays live on the device */
    int panel_width;   /* column panel of the D echelonisation, 0 = default (128) */
    int path;          /* GBLA_PATH_* */
    int leaf_width;    /* leaf columns of the triangular solve: 0 = chosen per matrix,
                          else 128, 256, 512 or 1024 */
    int kernel_times;  /* 1: time every launch of the two tensor-core kernels with events
                          and count the dense product's tile work (gbla_stats.tc_*,
                          gather_*); needs stats */
    int fl_order;      /* GBLA_ORDER_*: order of the FL steps */
    int autotune;      /* 1: the choices left open here (path on GBLA_PATH_AUTO, leaf_width
                          0, the gathered product's raster group) are made per shape
                          bucket by measurement: the first calls of a bucket (rows, columns
                          and density rounded to powers of two, tensor-core paths only) try
                          the candidates in turn, later calls take the fastest.  Every
                          candidate gives the same exact result. */
    int echelon;       /* GBLA_ECHELON_*: forward pass of the echelon step of D' */
} gbla_options;

/* Forward pass of the echelon step of the Schur complement D'.  Column panels
 * eliminate 128 columns at a time with tensor-core updates; SGE is the
 * paper's structured Gaussian elimination with sparse pivot rows (Alg. 3,
 * its parallel form in Sec. 5.1), for a D' that stays sparse: each warp
 * reduces one row at a time by the sparse pivots found so far and claims the
 * row's leading column when it has none.  If its pivot pool (about four times
 * the nonzeros of D') fills up, the panels finish the pass.  AUTO samples the
 * rows of D' and takes SGE when at most 30% of its entries are nonzero
 * (measured 1.6-2.1x faster than the panels there), else the panels.  The
 * result is the same either way. */
#define GBLA_ECHELON_AUTO 0
#define GBLA_ECHELON_PANELS 1
#define GBLA_ECHELON_SGE 2

/* Order of the FL steps.  The new order (Sec. 4.3) computes X = C*A^-1 and
 * D <- D - X*B, and A^-1*B only for the reduced form.  The original order
 * (Sec. 4.1 steps 2-3) computes B <- A^-1*B first and D <- D - C*B, so the
 * reduced form needs one triangular solve instead of two; it runs on the
 * dense path (GBLA_PATH_SPARSE with it gives GBLA_E_UNSUPPORTED). */
#define GBLA_ORDER_NEW 0
#define GBLA_ORDER_TRSM_FIRST 1

/* Per-call statistics (optional out-parameter). */
typedef struct {
    int64_t npiv;      /* pivots known from the input (rows of A) */
    int64_t m_cd;      /* non-pivot, non-empty rows (rows of C and D) */
    int64_t n_d;       /* non-pivot columns (columns of B and D) */
    int64_t rank_d;    /* rank of the Schur complement D' */
    double ms_split, ms_trsm, ms_schur, ms_echelon, ms_backsub, ms_output, ms_total;
    double mod_ops;    /* modular multiply-adds of the dense products (zero staircase excluded) */
    int64_t launches;  /* CUDA kernels launched by the call */
    double schur_mod_ops; /* the same for the Schur update D <- D - X*B alone */
    double ms_echelon_back; /* part of ms_echelon: the backward pass (RREF rows from the echelon form) */
    int64_t path;      /* GBLA_PATH_DENSE or GBLA_PATH_SPARSE: the path taken */
    int64_t list_a, list_b; /* sparse path: compacted K entries (all tiles) of A's
                               off-diagonal blocks and of B */
    int64_t leaf_width;     /* leaf columns of the triangular solve */
    double schur_exec_mod_ops; /* sparse path: multiply-adds the Schur launch runs on the tensor
                                  cores (its compacted tiles, zeros included) */
    /* with gbla_options.kernel_times: the dense tensor-core product (all its
     * launches: leaf solves, echelon waves, back-substitution) and the gathered
     * product (triangular-solve updates and the Schur update) */
    int64_t tc_launches, gather_launches;
    double tc_ms, gather_ms;     /* sums of the event-timed launch durations */
    double tc_mod_ops;           /* dense product: valid rows x columns x K run of its tiles */
    int64_t tc_pair_launches;    /* dense product launches that ran on CTA pairs (cta_group::2,
                                    enabled by the environment switch GBLA_GEMM_PAIR=1) */
    int64_t gather_group_m;      /* row tiles per raster group of the gathered product */
    int64_t tune_state;          /* with autotune: 1 = a trial of one candidate, 2 = the bucket's
                                    fastest candidate, 3 = default while trials are in flight;
                                    0 without autotune */
    int64_t echelon_method;      /* GBLA_ECHELON_PANELS or GBLA_ECHELON_SGE: the forward pass that
                                    finished the echelon step */
    double d_density;            /* with GBLA_ECHELON_SGE or _AUTO: nonzero share of D' on at most
                                    4,096 evenly spaced rows (else -1) */
} gbla_stats;

/* ---- whole reduction -------------------------------------------------- */
/* Synchronous: host input, host output.  *rank receives the rank.  On error
 * *out is zeroed. */
int gbla_reduce(const gbla_csr_in *in, uint32_t p, int want_reduced,
                gbla_csr_out *out, int64_t *rank);

/* Extended form.  `stream` is a cudaStream_t (NULL = default stream).  The
 * call enqueues its work on `stream` and synchronises it a few times to read
 * sizes (pivot count, rank of D'); it returns once the result is complete.
 * opt may be NULL (defaults).  stats may be NULL. */
int gbla_reduce_ex(const gbla_csr_in *in, uint32_t p, const gbla_options *opt,
                   void *stream, gbla_csr_out *out, int64_t *rank, gbla_stats *stats);

/* ---- many matrices ----------------------------------------------------- */
/* Batch: reduce n independent matrices (in[i] over GF(p[i]), options opt for
 * all, NULL = defaults).  `workers` host threads (0 = 8), each with its own
 * CUDA stream on the current device, take the matrices largest first; their
 * reductions overlap on the device.  outs[i], ranks[i],
 * codes[i] receive each result (release outs with gbla_free).  Returns
 * GBLA_OK, or the first failing code (the other results are still valid
 * where codes[i] == 0). */
int gbla_reduce_batch(int n, const gbla_csr_in *in, const uint32_t *p, const gbla_options *opt,
                      int workers, gbla_csr_out *outs, int64_t *ranks, int *codes);

/* Server: a request queue with continuous batching.  Requests (host CSR,
 * copied at submit) are admitted in arrival order whenever a worker is free
 * and the request's estimated device footprint fits in mem_budget next to
 * the requests already running; a request larger than the budget runs alone.
 * Admitted requests run on the workers' streams and overlap on the device
 * with the requests already running.  Latency is measured from submit to
 * result ready. */
typedef struct gbla_server gbla_server;
typedef struct {
    int64_t submitted, completed, failed, cancelled, queued, running;
    double p50_ms, p99_ms, mean_ms;   /* submit-to-ready latency of completed requests */
    size_t mem_budget, mem_in_use;    /* bytes, estimated footprints of running requests */
    int64_t peak_running;             /* most requests running at once so far */
} gbla_server_stats;

/* One request's timeline (gbla_server_wait_ex).  The device times come from
 * CUDA events recorded on the worker's stream right before and right after
 * the reduction, in ms since a reference event recorded when the server was
 * created; two requests whose [device_start_ms, device_end_ms] intervals
 * intersect had device work in flight at the same time.  -1 where events
 * were not available. */
typedef struct {
    double latency_ms;        /* submit to result ready (host clock) */
    double queue_ms;          /* submit to the start of the reduction */
    double device_start_ms, device_end_ms;
    int64_t running_at_start; /* requests running when this one started, itself included */
} gbla_request_info;

#define GBLA_REQ_QUEUED 0
#define GBLA_REQ_RUNNING 1
#define GBLA_REQ_DONE 2
#define GBLA_REQ_CANCELLED 3

/* mem_budget 0 = 80% of the device memory free now; workers 0 = 8. */
int gbla_server_create(size_t mem_budget, int workers, gbla_server **srv);
/* opt->device_ptrs must be 0.  *ticket identifies the request. */
int gbla_server_submit(gbla_server *srv, const gbla_csr_in *in_host, uint32_t p,
                       const gbla_options *opt, int64_t *ticket);
/* Wait up to timeout_s seconds (< 0: forever).  Returns the request's code
 * and fills *out (host arrays, release with gbla_free) and *rank; the ticket
 * is consumed.  GBLA_E_TIMEOUT if not done in time (the ticket stays valid),
 * GBLA_E_CANCELLED if it was cancelled. */
int gbla_server_wait(gbla_server *srv, int64_t ticket, double timeout_s,
                     gbla_csr_out *out, int64_t *rank, double *latency_ms);
/* The same, filling *info (may be NULL) with the request's timeline. */
int gbla_server_wait_ex(gbla_server *srv, int64_t ticket, double timeout_s,
                        gbla_csr_out *out, int64_t *rank, gbla_request_info *info);
/* State of a request without waiting: *state = GBLA_REQ_*.  The ticket stays
 * valid.  GBLA_E_INVAL for an unknown (or already consumed) ticket. */
int gbla_server_poll(gbla_server *srv, int64_t ticket, int *state);
/* Cancel a request that is still queued (GBLA_E_INVAL if running or done). */
int gbla_server_cancel(gbla_server *srv, int64_t ticket);
int gbla_server_get_stats(gbla_server *srv, gbla_server_stats *st);
/* Drop queued requests, wait for running ones, release everything.  Call it
 * after all waits have returned. */
void gbla_server_destroy(gbla_server *srv);

/* Release a result (host or device arrays); zeroes *out.  NULL-safe. */
void gbla_free(gbla_csr_out *out);

/* Human-readable error text for a GBLA_* code (static storage). */
const char *gbla_strerror(int code);

/* ABI version (major*100 + minor). */
int gbla_version(void);

/* Environment switches read once per process: GBLA_LOG=1 prints one line per
 * reduction on stderr (path, order, variant, leaf width, block shapes, list
 * sizes, phase times); GBLA_FAULT_ALLOC_AFTER=n arms the allocation fault
 * below at the first allocation. */

/* Fault injection for tests (host side, no device fault): every device and
 * host allocation of the library counts against one process-wide counter;
 * the allocation that follows the next n fails once (the call returns
 * GBLA_E_NOMEM, or the batch member / server request does), after which
 * allocations succeed again.  n < 0 disarms. */
int gbla_selftest_fail_alloc_after(int64_t n);

/* Bytes of the device's stream-ordered memory pool currently allocated (the
 * library's scratch; 0 when no call is in flight and nothing leaked).
 * Synchronises the device. */
int gbla_device_bytes_in_use(int64_t *bytes);

/* ---- building blocks, exposed for testing ----------------------------- */
/* Modular matrix product on device memory (FL steps 2-3, the dense Schur
 * update D <- D - C*A^-1*B of Sec. 4.1, done as an exact GEMM):
 *     C <- (C + sign * A * B) mod p
 * A: M x K, B: K x N, C: M x N, all row-major uint16 device arrays with
 * leading dimensions lda, ldb, ldc (in elements), entries in [0, p).
 * sign is +1 or -1.  variant is GBLA_GEMM_*.  Scratch is allocated on
 * `stream` and released before return; the call synchronises `stream`. */
int gbla_modmatmul(int64_t M, int64_t N, int64_t K, const uint16_t *A, int64_t lda,
                   const uint16_t *B, int64_t ldb, uint16_t *C, int64_t ldc,
                   uint32_t p, int sign, int variant, void *stream);

/* The exact modular product for 32-bit coefficients (wider limbs): C <- (C +
 * sign * A * B) mod p for a prime 2 < p < 2^31, A: M x K, B: K x N, C: M x N
 * row-major uint32 device arrays (leading dimensions in elements), entries in
 * [0, p).  Each residue, in balanced form, is split into four 8-bit digits
 * exact in bf16 (the coefficient representations of Sec. 2: uint16 for 16-bit
 * primes, uint32 for 32-bit ones); the sixteen digit products of a pair land
 * in seven fp32 tensor-memory accumulators by digit position, exact over
 * k-blocks of 256, and are reduced mod p in 64-bit integers.  tcgen05 only
 * (GBLA_E_UNSUPPORTED elsewhere).  Scratch on `stream`; synchronises it. */
int gbla_modmatmul32(int64_t M, int64_t N, int64_t K, const uint32_t *A, int64_t lda,
                     const uint32_t *B, int64_t ldb, uint32_t *C, int64_t ldc,
                     uint32_t p, int sign, void *stream);

/* Issue-rate microbenchmark of a legacy tensor-core pipe: variant
 * GBLA_GEMM_FP64 (mma.sync m8n8k4 f64) or GBLA_GEMM_U8 (mma.sync m16n8k32
 * u8).  Every warp runs eight independent accumulator chains on operands held
 * in registers; the loop grows until one launch lasts at least 20 ms, timed
 * with CUDA events on `stream`.  *tops receives the instruction's operations
 * (2*M*N*K per instruction) per second in units of 1e12.  Synchronises
 * `stream`.  GBLA_E_INVAL for another variant or a null tops. */
int gbla_pipe_peak(int variant, double *tops, void *stream);

/* Sparse-path product (the Schur update D <- D - X*B of the new order,
 * Sec. 4.3, with B kept sparse as in Table 4):
 *     C <- (C + sign * X * S) mod p
 * X: M x K dense row-major uint16 (device, leading dimension ldx), entries in
 * [0, p); S: K x N sparse CSR on the device (int64 row_ptr[K+1], int32 col
 * strictly increasing per row, uint16 val in [1, p)); C: M x N dense
 * row-major uint16 (device, ldc).  x_lead (device, may be NULL): ascending
 * index of each X row's first nonzero column (X must be zero left of it); a
 * 128-row tile then skips the rows of S left of its first row's lead.  S is
 * compacted per 128-column tile to the rows that meet the tile, and the
 * product runs on the tensor cores with that compacted K.  A malformed S
 * gives GBLA_E_INVAL (C untouched); p < 8 gives GBLA_E_UNSUPPORTED.  Scratch
 * is allocated on `stream` and released before return; synchronises
 * `stream`. */
int gbla_spmm(int64_t M, int64_t N, int64_t K, const uint16_t *X, int64_t ldx, const gbla_csr_in *S_dev,
              const int32_t *x_lead, uint16_t *C, int64_t ldc, uint32_t p, int sign, void *stream);

/* FL step 1 pivot analysis on device memory (Sec. 3.1, Sec. 4.1 step 1):
 * validates the CSR (device pointers), and writes for every column c
 * piv_row[c] = the input row chosen as pivot for c (-1 if no row leads at c).
 * *npiv receives the number of pivots.  piv_row is a device array of ncols
 * int64.  Synchronises `stream`. */
int gbla_pivots(const gbla_csr_in *in_dev, uint32_t p, int64_t *piv_row_dev,
                int64_t *npiv, void *stream);

/* 2-multiline vector of pairs of pivot rows (Definition 1, Sec. 4.2), the
 * layout the sparse reduction C <- C*A^-1 reads.  For a device CSR of 2*q
 * rows (host pointers here, small inputs), fills for each pair of rows
 * (2i, 2i+1): pos = union of their columns, ascending; val[2e], val[2e+1] =
 * the two rows' values at pos[e] (0 where a row has none).  Output arrays are
 * host arrays sized by the caller: ml_ptr[q+1], ml_pos[total], ml_val[2*total]
 * where total <= nnz.  Returns GBLA_OK or an error. */
int gbla_multiline(const gbla_csr_in *pairs_host, int64_t *ml_ptr, int32_t *ml_pos,
                   uint16_t *ml_val, void *stream);

/* Failure-path self test (the paper has no counterpart).  Every wait of the
 * library's kernels on an mbarrier is bounded (about one second of device
 * clock); when one expires the kernel stops its other roles, waits for its own
 * copies, frees tensor memory, records the timeout and returns, so the CUDA
 * context stays usable.  This runs one product tile whose loads are withheld
 * and returns the resulting code: GBLA_E_TIMEOUT after about a second.
 * Synchronises `stream`. */
int gbla_selftest_wait_timeout(void *stream);

/* Pivot analysis that allocates no memory.  The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory
 * during a call -- an application that reserves all device memory up front
 * for its own pool, or a latency-sensitive loop where an allocation may
 * synchronise the device.  Same arguments and result as gbla_pivots (device
 * CSR in, device piv_row[ncols] out, *npiv on the host), but its only scratch
 * is a fixed 8 MiB device array inside the library, held by every GPU that
 * loads the library until the process exits.  ncols above 1,048,576 (2^20)
 * is rejected with GBLA_E_INVAL; so is a malformed CSR, in which case
 * piv_row is left unwritten.  The first call on a device (and the first after
 * its context was recreated, e.g. by cudaDeviceReset) looks up that array's
 * device address; make that first call before any stream capture.  All calls
 * share the array (each clears what it uses), so calls that overlap on the
 * GPU race: serialise them.  GBLA_E_UNSUPPORTED without a compute capability
 * 10.3 device.  Synchronises `stream`. */
int gbla_pivots_noalloc(const gbla_csr_in *in_dev, uint32_t p, int64_t *piv_row_dev,
                        int64_t *npiv, void *stream);

/* Format 2 matrix file (Sec. 3.2, Table 2) -> device CSR input.  `file` is
 * the whole file in host memory (borrowed, `bytes` long, little-endian):
 * u32 b (bits 0-2: coefficient type u | v << 1, 8 * 2^v bits, u = 1 unsigned;
 * the higher bits are a version and are ignored), u32 m, u32 n, u64 p,
 * u64 nnz, u32 rows[m] (row lengths), u32 polmap[m] (row i carries the
 * coefficients of polynomial polmap[i]), u64 k, u64 colid[k] (the rows'
 * columns in order: a run of s >= 2 consecutive columns from f is the pair
 * f, s, a lone column f is f | 2^31, runs never cross a row), u32 pnb,
 * u64 pnnz, u32 prow[pnb] (polynomial lengths), pdata[pnnz] (the
 * polynomials' coefficients in that type, signed ones taken mod p).  On
 * success *out holds device arrays (on_device = 1, nrows = m; release with
 * gbla_free) in the form gbla_reduce_ex takes, and *p the prime.  A file that
 * breaks any of these rules, a column >= n, columns not increasing within a
 * row, a coefficient that is 0 mod p, p outside [2, 2^16) or bytes after the
 * last field gives GBLA_E_INVAL and *out zeroed.  Synchronises `stream`. */
int gbla_decode_format2(const void *file, size_t bytes, void *stream, gbla_csr_out *out, uint32_t *p);
/* The same; *decode_ms (may be NULL) receives the event-timed duration of the
 * decode's device work on `stream` after the file's sections are on the
 * device (host-to-device copies excluded), or -1 on failure. */
int gbla_decode_format2_ex(const void *file, size_t bytes, void *stream, gbla_csr_out *out, uint32_t *p,
                           double *decode_ms);

#ifdef __cplusplus
}
#endif
#endif /* GBLA_H */
