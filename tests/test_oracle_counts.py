"""Pins for the oracle's work counters (modular multiply-adds per phase).

``oracle.echelon(..., ops=[...])`` reports
  ops_b -- Alg. 2 (Sec. 4.3): a non-pivot row reduced by pivot row j
           (multiplier x_j != 0) costs one multiply-add per entry of that row
           at the other pivot columns (the sparse C <- C*A^-1);
  ops_c -- ... and one per entry at the non-pivot columns (D <- D - X*B);
  ops_d -- the Gauss-Jordan pass on the Schur complement (Sec. 4.1 step 4
           and the reduced-echelon remark): nnz(P) - 1 per subtraction of a
           multiple of row P, forward and backward;
  ops_e -- back-substitution of the top block (0 in the echelon form).

Each matrix below is built so that the counts follow in closed form from its
construction (a pivot chain whose multipliers are known, A = I so that
X = C, a Schur complement of rank one, pairs whose backward step is known).
A counter that also counts zero multipliers, counts nnz(P) instead of
nnz(P) - 1, swaps the A and B parts or skips the backward pass fails one of
them.
"""
import numpy as np
import pytest

import oracle
from paper_1602_06097_gb300 import synth


def _ops(dense, p):
    dense = np.asarray(dense, dtype=np.int64) % p
    m, n = dense.shape
    rp, c, v = synth.dense_to_csr(dense)
    ops = []
    oracle.echelon(m, n, p, rp, c, v, ops=ops)
    return ops


@pytest.mark.parametrize("k", [3, 5, 17])
def test_chain_counts_only_nonzero_multipliers(k):
    """Pivot rows e_j + e_{j+1} (j < k-1) and e_{k-1}; one extra row
    e_0 + e_1 + e_2.  Its multipliers are X = (1, 0, 1, -1, 1, -1, ...): pivot
    row 1 is skipped, every other row j < k-1 costs its one off-diagonal
    entry, so ops_b = k - 2."""
    p = 65521
    M = np.zeros((k + 1, k), np.int64)
    for j in range(k):
        M[j, j] = 1
        if j + 1 < k:
            M[j, j + 1] = 1
    M[k, 0] = M[k, 1] = M[k, 2] = 1
    ops = _ops(M, p)
    assert ops == [k - 2, 0, 0, 0]


@pytest.mark.parametrize("seed", range(4))
def test_identity_a_block_gives_x_equal_c(seed):
    """A = I (pivot rows e_j + B_j with B_j on the non-pivot columns), so
    X = C and ops_c = sum over non-pivot rows of sum_{j in supp C_r} nnz(B_j);
    ops_b = 0."""
    rng = np.random.default_rng(300 + seed)
    p = [65521, 32003, 7, 11][seed]
    npv, nq, mnp = 12, 20, 9
    n = npv + nq
    M = np.zeros((npv + mnp, n), np.int64)
    nb = np.zeros(npv, np.int64)
    for j in range(npv):
        M[j, j] = 1
        q = rng.choice(nq, size=int(rng.integers(0, 4)), replace=False)
        M[j, npv + q] = rng.integers(1, p, size=len(q))
        nb[j] = len(q)
    expect_c = 0
    for r in range(mnp):
        # at least 4 entries: a pivot row (at most 4 entries, smaller index)
        # keeps every leading column
        s = np.sort(rng.choice(npv, size=int(rng.integers(4, 8)), replace=False))
        M[npv + r, s] = rng.integers(1, p, size=len(s))
        q = rng.choice(nq, size=int(rng.integers(0, 5)), replace=False)
        M[npv + r, npv + q] = rng.integers(1, p, size=len(q))
        expect_c += int(nb[s].sum())
    ops = _ops(M, p)
    assert ops[0] == 0
    assert ops[1] == expect_c
    assert ops[3] == 0


@pytest.mark.parametrize("mnp,t", [(2, 5), (7, 1), (30, 12)])
def test_rank_one_schur_complement_forward_count(mnp, t):
    """Pivot rows are unit vectors, so the Schur complement is the non-pivot
    rows' tails lambda_r * v (nnz(v) = t): the first becomes a pivot, each
    other one is cancelled by one subtraction, ops_d = (mnp - 1)(t - 1)."""
    rng = np.random.default_rng(mnp * 31 + t)
    p = 65521
    npv, nq = 6, 40
    n = npv + nq
    v = np.zeros(nq, np.int64)
    v[np.sort(rng.choice(nq, size=t, replace=False))] = rng.integers(1, p, size=t)
    M = np.zeros((npv + mnp, n), np.int64)
    for j in range(npv):
        M[j, j] = 1
    for r in range(mnp):
        M[npv + r, int(rng.integers(0, npv))] = int(rng.integers(1, p))
        M[npv + r, npv:] = v * int(rng.integers(1, p)) % p
    ops = _ops(M, p)
    assert ops == [0, 0, (mnp - 1) * (t - 1), 0]


def test_backward_pass_count_on_pairs():
    """Pairs of Schur rows e_a + e_b + v_i, e_b + v_i on disjoint columns
    (a < b < supp v_i): the forward pass makes both pivots without any
    subtraction; the backward pass clears column b of the first row with one
    subtraction of the final e_b + v_i, costing nnz(v_i).  ops_d = sum t_i."""
    rng = np.random.default_rng(9)
    p = 32003
    npv = 3
    ts = [1, 4, 9, 2]
    width = sum(2 + t for t in ts)
    n = npv + width
    rows = []
    col = npv
    for t in ts:
        a, b = col, col + 1
        vcols = list(range(col + 2, col + 2 + t))
        col += 2 + t
        vals = rng.integers(1, p, size=t)
        r1 = np.zeros(n, np.int64)
        r2 = np.zeros(n, np.int64)
        r1[a] = r1[b] = r2[b] = 1
        r1[vcols] = vals
        r2[vcols] = vals
        rows += [r1, r2]
    M = np.zeros((npv + len(rows), n), np.int64)
    for j in range(npv):
        M[j, j] = 1
    for i, r in enumerate(rows):
        M[npv + i] = r
        M[npv + i, i % npv] = 5   # lead at a pivot column (X = 5 e_j)
    ops = _ops(M, p)
    assert ops == [0, 0, sum(ts), 0]


def test_counts_of_a_generated_matrix_are_consistent():
    """On an F4-shaped matrix the counters are integers, the Schur part is
    bounded by its dense size, and reducing twice gives the same counts."""
    spec = synth.FLSpec(m=300, n=420, npiv=180, density=0.05, run_len=(3, 12), seed=501)
    rp, c, v = synth.fl_matrix(spec)
    a, b = [], []
    oracle.echelon(spec.m, spec.n, spec.p, rp, c, v, ops=a)
    oracle.echelon(spec.m, spec.n, spec.p, rp, c, v, ops=b)
    assert a == b
    assert all(float(x).is_integer() and x >= 0 for x in a)
    assert a[0] > 0 and a[1] > 0 and a[3] == 0


@pytest.mark.parametrize("seed", range(3))
def test_row_counts_equal_the_echelon_counters(seed):
    """The counts-only entry point reduces the same rows in the same order as
    oracle.echelon (whose counters are pinned above)."""
    spec = synth.FLSpec(m=400, n=600, npiv=250, density=0.04, run_len=(3, 16), seed=900 + seed,
                        p=[65521, 32003, 11][seed])
    rp, c, v = synth.fl_matrix(spec)
    ops = []
    _, _, _, _, npiv = oracle.echelon(spec.m, spec.n, spec.p, rp, c, v, ops=ops)
    b, cc, npiv2, secs = oracle.row_counts(spec.m, spec.n, spec.p, rp, c, v)
    assert (b, cc, npiv2) == (ops[0], ops[1], npiv)
    assert secs >= 0
