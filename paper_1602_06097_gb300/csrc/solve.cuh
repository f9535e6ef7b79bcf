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
};
int trsm_upper(const TrsmUpper &T);

// X' * A^T = C' (A^T unit lower triangular), X' overwrites C'.
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
};
int echelon_d(const EchelonD &E, int64_t *rank_out);

}  // namespace gbla
