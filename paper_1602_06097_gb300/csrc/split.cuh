// split.cuh -- device data of FL step 1 (pivot analysis and splicing).
#pragma once

#include "common.cuh"
#include "internal.cuh"

namespace gbla {

// A CSR matrix in device memory.
struct DevCSR {
    int64_t m = 0, n = 0, nnz = 0;
    const int64_t *row_ptr = nullptr;
    const int32_t *col = nullptr;
    const uint16_t *val = nullptr;
};

// Result of the pivot analysis.  Permuted column order: the npiv pivot
// columns ascending, then the n_d other columns ascending.  Row k of A/B is
// input row piv_row[k]; row i of C/D is input row cd_rows[i], C/D rows
// ordered by leading column (cd_lead ascending), ties in input order.
struct PivotInfo {
    int64_t m = 0, n = 0, npiv = 0, m_cd = 0, n_d = 0;
    int32_t *lead = nullptr;                 // [m] leading column or -1
    unsigned long long *best = nullptr;      // [n] (weight << 32 | row) of the chosen pivot, or ~0
    int64_t *dev_counts = nullptr;           // [2] npiv, m_cd on the device
    int32_t *colmap = nullptr;               // [n] input column -> permuted index
    int32_t *pivcol_orig = nullptr;          // [npiv] permuted pivot column -> input column
    int32_t *npcol_orig = nullptr;           // [n_d] permuted other column -> input column
    int32_t *piv_row = nullptr;              // [npiv] row of A -> input row
    int32_t *cd_rows = nullptr;              // [m_cd] row of C/D -> input row
    int32_t *cd_index = nullptr;             // [m] input row -> row of C/D or -1
    int32_t *cd_lead = nullptr;              // [m_cd] permuted leading column of each C/D row (ascending)
    uint32_t *inv_lead = nullptr;            // [npiv] inverse of the pivot row's leading coefficient
};

// 2-multiline storage of the diagonal blocks of A (Definition 1): pair q =
// A rows 2q, 2q+1, entries at permuted pivot columns inside the pair's own
// block of LEAF_COLS columns, excluding each row's unit diagonal.  val packs
// row 2q's value in the low 16 bits and row 2q+1's in the high 16 bits.
// Column blocks of the blocked triangular solves.
constexpr int LEAF_COLS = 128;

struct Multiline {
    int64_t npairs = 0, total = 0;
    int64_t *ptr = nullptr;    // [npairs + 1]
    int32_t *pos = nullptr;    // [total]
    uint32_t *val = nullptr;   // [total]
    int32_t *inblk = nullptr;  // [npairs] entries of pair q inside its own column block of LEAF_COLS
};

int pivot_analysis(const DevCSR &in, const ModP &mp, PivotInfo *pi, uint32_t *err, cudaStream_t s);
void pivot_free(PivotInfo *pi, cudaStream_t s);

int split_scatter(const DevCSR &in, const PivotInfo &pi, uint16_t *A16, int64_t lda, uint16_t *B16, int64_t ldb,
                  uint16_t *C16, int64_t ldc, uint16_t *D16, int64_t ldd, const ModP &mp, cudaStream_t s);

int multiline_build(const DevCSR &in, const PivotInfo &pi, Multiline *ml, const ModP &mp, cudaStream_t s);

// The pivot rows as sparse operands (sparse.cu): Adiag (round_up(npiv, L) x L
// uint16, zeroed here) <- A's diagonal blocks of width L; SA <- A's
// off-diagonal blocks and SB <- B, K-compacted per 128-column tile.
int sparse_build(const DevCSR &in, const PivotInfo &pi, int L, uint16_t *Adiag, Compact *SA, Compact *SB,
                 const ModP &mp, cudaStream_t s);

// A sparse K x N matrix S (device CSR, validated here: GBLA_E_INVAL on a
// malformed one) as a compacted operand (rows = K).
int compact_from_csr(const DevCSR &S, Compact *out, const ModP &mp, uint32_t *err, cudaStream_t s);
void multiline_free(Multiline *ml, cudaStream_t s);

int multiline_pairs(int64_t m, const int64_t *row_ptr, const int32_t *col, const uint16_t *val, int64_t *ml_ptr_dev,
                    int32_t *ml_pos_dev, uint16_t *ml_val_dev, int64_t *total, cudaStream_t s);

}  // namespace gbla
