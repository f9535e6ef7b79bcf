// solve.cuh -- triangular solves and the echelonisation of D.
#pragma once

#include "common.cuh"
#include "internal.cuh"
#include "split.cuh"

#include <vector>

namespace gbla {

// X * A = C (A unit upper triangular, npiv x npiv), X overwrites C.
struct TrsmUpper {
    int64_t mrows, npiv;
    uint16_t *C16;
    int64_t ldc;
    const Multiline *ml;   // A rows, 2-multiline
    const Planes *Xp;      // A-operand planes of X (mrows x npiv), written here
    const Planes *At;      // B-operand planes of A^T (npiv x npiv)
    const ModP *mp;
    int variant;
    uint32_t *err;
    cudaStream_t s;
    GemmCounters *ctr;
    const int32_t *lead_dev;                 // optional: ascending lead of each row (device)
    const std::vector<int32_t> *lead_host;   // the same on the host
    // Optional (tensor-core variant): B-operand planes of the inverses of A's
    // diagonal blocks of width tc_leaf (upper_leaf_inverses) and an A-operand
    // scratch set of mrows x tc_leaf.  With both, a diagonal block is solved as
    // X_J = C_J * A_JJ^-1 on the tensor cores instead of by the multiline kernel.
    const Planes *Zt;
    const Planes *Ct;
    int tc_leaf;
};
int trsm_upper(const TrsmUpper &T);

// B-operand planes (4 planes, L * ceil(npiv / L) rows x L) of the inverses of
// the unit upper triangular diagonal blocks A[J, J] of width L (a power of two,
// multiple of 128) of A (dense uint16, lda): row L q + j, column k of Zt holds
// (A_JJ^-1)[k][j] for block J = [L q, L q + L), zero outside A.  For L >= 512
// the wider levels of the inverses are tensor-core products (err: their
// device status word).
// With Zr (optional), the same inverses also as B-operand planes of Z_J
// itself: Zr row J L + k, column j = Z_J[k][j] (the lower solve's leaves).
int upper_leaf_inverses(const uint16_t *A16, int64_t lda, int64_t npiv, int L, const Planes &Zt, const ModP &mp,
                        uint32_t *err, cudaStream_t s, const Planes *Zr = nullptr);

// Leaf inverses as upper_leaf_inverses, from A's diagonal blocks alone:
// Adiag (round_up(npiv, L) x L uint16) row k holds A[k][c] at column c % L for
// the columns c of k's own block (sparse_build).
int upper_leaf_inverses_diag(const uint16_t *Adiag, int64_t npiv, int L, const Planes &Zt, const ModP &mp,
                             uint32_t *err, cudaStream_t s, const Planes *Zr = nullptr);

// X * A = C on the sparse path (tensor-core variant): the transposed solution
// X^T is written to the A-operand planes XT (rows = pivots, K = rows of C).
// Left-looking over leaves J of width L:
//   C_J -= X_{<J} * A_{<J,J}   gathered product over SA (K-compacted A),
//   X_J^T = Z_J^T * C_J^T      one product with Z_J = A_JJ^-1 (Zt),
// only for the rows whose lead is left of the leaf's end (rows ascending by
// lead).  C16 is modified; XT must be zero on entry.
struct TrsmSparse {
    int64_t mrows, npiv;
    uint16_t *C16;
    int64_t ldc;
    const Compact *SA;
    const Planes *Zt;     // B-operand planes of the leaf inverses (rows npiv, K = L)
    const Planes *Ct;     // 4-plane scratch of mrows x L: C_J as B-operand
    const Planes *XT;     // out
    int L;
    const ModP *mp;
    uint32_t *err;
    cudaStream_t s;
    GemmCounters *ctr;
    const int32_t *lead_dev;
    const std::vector<int32_t> *lead_host;
};
int trsm_sparse(const TrsmSparse &T);

// X' * A^T = C' (A^T unit lower triangular), X' overwrites C'.  Right-
// looking from the last columns: a leaf J solves X'_J A'_JJ = C'_J, then
// C'_{<J} -= X'_J A'_{J,<J} for the columns left of it.  With Zr and Ct a
// leaf of width tc_leaf is X'_J = C'_J Z_J^T (Z_J = A_JJ^-1) on the tensor
// cores, else the multiline leaf kernel solves it.
struct TrsmLower {
    int64_t mrows, npiv;
    uint16_t *C16;
    int64_t ldc;
    const Multiline *ml;
    const Planes *Xp;      // A-operand planes of X' (mrows x npiv), written here
    const Planes *Arow;    // B-operand planes of A (npiv x npiv, row-major A)
    const ModP *mp;
    int variant;
    uint32_t *err;
    cudaStream_t s;
    GemmCounters *ctr;
    const Planes *Zr = nullptr;   // B-operand planes of the leaf inverses Z_J (rows npiv, K = tc_leaf)
    const Planes *Ct = nullptr;   // A-operand scratch of mrows x tc_leaf
    int tc_leaf = 0;
};
int trsm_lower(const TrsmLower &T);

// Reduced echelon form of D (m x n, uint16, modified in place).  On return
// *R (allocated here, rank x ldd, release with dfree) holds the RREF rows in
// pivot-column order, with pivot columns pcol[0..rank) ascending.
struct EchelonD {
    int64_t m, n;
    uint16_t *D16;
    int64_t ldd;
    int32_t *is_piv_row;   // [m] scratch
    int32_t *prow, *pcol;  // [m] outputs (prow: row of D each pivot came from)
    uint16_t **R;          // out: RREF rows, rank x ldd
    const ModP *mp;
    int variant;
    uint32_t *err;
    cudaStream_t s;
    GemmCounters *ctr;
    cudaEvent_t back_start = nullptr;   // optional: recorded when the backward pass begins
    int back_leaf = 0;                  // leaf rows of the back-substitution (power of two >= 128; 0: 128)
    int method = 0;                     // forward pass: 0 column panels, 1 sparse SGE (sge.cu), 2 SGE when
                                        // D' has at most SGE_MAX_DENSITY nonzeros, else panels
    double *density = nullptr;          // out (methods 1, 2): nonzero share of D' before the pass
    int *sge_completed = nullptr;       // out (methods 1, 2): 1 if SGE finished the forward pass
    // With np_out set, *R is not formed: the caller receives the reduced rows
    // at the non-pivot columns only (row k = RREF row k, whose pivot column is
    // pcol[k] with value 1 and whose other pivot columns are 0), and owns the
    // buffers (device, stream-ordered).
    struct NonPivot {
        uint16_t *Rnp = nullptr;   // rank x ldnp
        int64_t ldnp = 0;
        int32_t *npc = nullptr;    // [nnp] column of D of each non-pivot column, ascending
        int64_t nnp = 0;
    } *np_out = nullptr;
};
int echelon_d(const EchelonD &E, int64_t *rank_out);

// Forward pass of the echelon step by structured Gaussian elimination with
// sparse pivot rows (Alg. 3, parallel form of Sec. 5.1): on success prow,
// pcol hold the pivots in ascending column order, their rows of D16 are
// normalised and zero left of the lead, *rank their number.  *overflow: the
// sparse pivot pool filled up; D16 then holds valid row combinations of D'
// and the caller continues with the panel method.  *density: nonzero share
// of D' on entry (dprime_density: counted on at most 4,096 evenly spaced rows).
int sge_forward(const EchelonD &E, double density, int64_t *rank, bool *overflow);
int dprime_density(const EchelonD &E, double *density);

// Largest nonzero share of D' for which the automatic choice takes SGE
// (measured: SGE 1.6-2.1x faster than the panels up to a share of 0.30).
constexpr double SGE_MAX_DENSITY = 0.3;

}  // namespace gbla
