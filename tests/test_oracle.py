"""Pins for the CPU oracle, checked against what the mathematics fixes.

Nothing here re-types the oracle's formulas.  The oracle's RREF is pinned by:

* brute force over GF(7): the whole row space is enumerated and the RREF is
  read off it (for each pivot column, the unique vector of the space with a 1
  there and 0 at every other pivot column);
* determinant ranks over GF(65521): Leibniz expansion of every minor;
* closed forms: a matrix built as G * R0 from a chosen RREF R0 and a full
  column rank G has RREF exactly R0 (any size);
* special cases (identity, zero, permutations, duplicates, rank one, p = 2, 3);
* the defining properties of an RREF (unit pivots, zeros elsewhere in pivot
  columns, strictly increasing pivot columns) plus span equality checked with
  a separately written column-wise elimination.

The multiline encoder is pinned by the paper's Example 1, and planted
mistakes (compiled-in mutants of oracle.c) are shown to fail these pins.
"""
import itertools
import json
import os
import random

import numpy as np
import pytest

import oracle
from paper_1602_06097_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- helpers
def to_csr(dense):
    return synth.dense_to_csr(np.asarray(dense, dtype=np.int64))


def run_rref(dense, p, mutant=0):
    dense = np.asarray(dense, dtype=np.int64) % p
    m, n = dense.shape
    rp, c, v = to_csr(dense)
    r, orp, oc, ov = oracle.rref(m, n, p, rp, c, v, mutant=mutant)
    return synth.csr_to_dense(r, n, orp, oc, ov)


def run_echelon(dense, p, mutant=0):
    dense = np.asarray(dense, dtype=np.int64) % p
    m, n = dense.shape
    rp, c, v = to_csr(dense)
    r, orp, oc, ov, npiv = oracle.echelon(m, n, p, rp, c, v, mutant=mutant)
    return synth.csr_to_dense(r, n, orp, oc, ov), npiv


def brute_rref(dense, p):
    """RREF read off the enumerated row space (tiny m only)."""
    dense = np.asarray(dense, dtype=np.int64) % p
    m, n = dense.shape
    space = set()
    for coeffs in itertools.product(range(p), repeat=m):
        v = tuple(int(x) for x in (np.array(coeffs, dtype=np.int64) @ dense) % p) if m else tuple([0] * n)
        space.add(v)
    def lead(v):
        for j, x in enumerate(v):
            if x:
                return j
        return None
    pivots = sorted({lead(v) for v in space if lead(v) is not None})
    rows = []
    for c in pivots:
        cands = [v for v in space if lead(v) == c and v[c] == 1 and all(v[d] == 0 for d in pivots if d != c)]
        assert len(cands) == 1, "RREF row must be unique"
        rows.append(cands[0])
    out = np.array(rows, dtype=np.int64).reshape(len(rows), n)
    # |space| = p^rank is itself a check of the rank
    assert len(space) == p ** len(rows)
    return out


def det_mod(a, p):
    """Leibniz determinant mod p (tiny matrices)."""
    k = len(a)
    tot = 0
    for perm in itertools.permutations(range(k)):
        inv = sum(1 for i in range(k) for j in range(i + 1, k) if perm[i] > perm[j])
        prod = 1
        for i in range(k):
            prod = prod * int(a[i][perm[i]]) % p
        tot += -prod if inv % 2 else prod
    return tot % p


def rank_by_minors(dense, p):
    dense = np.asarray(dense, dtype=np.int64) % p
    m, n = dense.shape
    for k in range(min(m, n), 0, -1):
        for rs in itertools.combinations(range(m), k):
            for cs in itertools.combinations(range(n), k):
                if det_mod(dense[np.ix_(rs, cs)], p):
                    return k
    return 0


def rank_colwise(dense, p):
    """Rank by column-wise elimination with row swaps (written independently
    of the oracle: columns outer, explicit swaps, Python big ints)."""
    a = [[int(x) % p for x in row] for row in np.asarray(dense)]
    m = len(a)
    n = len(a[0]) if m else 0
    r = 0
    for c in range(n):
        piv = next((i for i in range(r, m) if a[i][c]), None)
        if piv is None:
            continue
        a[r], a[piv] = a[piv], a[r]
        inv = pow(a[r][c], p - 2, p)
        for i in range(r + 1, m):
            if a[i][c]:
                f = a[i][c] * inv % p
                a[i] = [(x - f * y) % p for x, y in zip(a[i], a[r])]
        r += 1
    return r


def assert_rref_shape(R, p):
    R = np.asarray(R, dtype=np.int64)
    prev = -1
    for i in range(R.shape[0]):
        nz = np.nonzero(R[i])[0]
        assert len(nz), "zero row in output"
        c = nz[0]
        assert c > prev, "pivot columns must strictly increase"
        prev = c
        assert R[i, c] == 1, "pivot must be 1"
        col = R[:, c].copy()
        col[i] = 0
        assert not col.any(), "pivot column must be zero elsewhere"
        assert (R[i] >= 0).all() and (R[i] < p).all()


def assert_span_equal(M, R, p):
    """Every row of M reduces to zero against R (R in RREF), and stacking R
    onto M does not raise the rank."""
    M = np.asarray(M, dtype=np.int64) % p
    R = np.asarray(R, dtype=np.int64)
    if R.shape[0]:
        pc = [int(np.nonzero(R[i])[0][0]) for i in range(R.shape[0])]
        resid = (M - M[:, pc] @ R) % p
        assert not resid.any(), "an input row is not in the span of the output"
    rk = rank_colwise(M, p)
    assert rk == R.shape[0]
    assert rank_colwise(np.vstack([M, R]) if R.shape[0] else M, p) == rk


def random_rref(rng, r, n, p, density=1.0):
    """A random r x n RREF matrix with chosen pivot columns."""
    pcs = np.sort(rng.choice(n, size=r, replace=False))
    R = np.zeros((r, n), np.int64)
    for i, c in enumerate(pcs):
        R[i, c] = 1
        for j in range(c + 1, n):
            if j in pcs:
                continue
            if rng.random() < density:
                R[i, j] = rng.integers(0, p)
    return R, pcs


def full_col_rank(rng, m, r, p):
    T = np.tril(rng.integers(0, p, size=(r, r)), -1) + np.eye(r, dtype=np.int64)
    Z = rng.integers(0, p, size=(m - r, r))
    G = np.vstack([T, Z])
    return G[rng.permutation(m)]


# ----------------------------------------------------------------- pins
@pytest.mark.parametrize("seed", range(120))
def test_rref_matches_brute_force_gf7(seed):
    rng = np.random.default_rng(seed)
    m = int(rng.integers(1, 5))
    n = int(rng.integers(1, 6))
    dense = np.where(rng.random((m, n)) < 0.6, rng.integers(1, 7, size=(m, n)), 0)
    if seed % 5 == 0 and m > 1:
        dense[1] = dense[0] * 3 % 7           # a multiple of another row
    if seed % 7 == 0:
        dense[0] = 0                          # an empty row
    R = run_rref(dense, 7)
    B = brute_rref(dense, 7)
    assert R.shape == B.shape
    assert (R == B).all()


@pytest.mark.parametrize("seed", range(40))
def test_rref_rank_by_minors_gf65521(seed):
    p = 65521
    rng = np.random.default_rng(1000 + seed)
    m = int(rng.integers(1, 5))
    n = int(rng.integers(1, 5))
    dense = np.where(rng.random((m, n)) < 0.7, rng.integers(1, p, size=(m, n)), 0)
    if seed % 3 == 0 and m > 2:
        dense[2] = (dense[0] * 5 + dense[1] * (p - 2)) % p   # dependent row
    R = run_rref(dense, p)
    assert R.shape[0] == rank_by_minors(dense, p)
    assert_rref_shape(R, p)
    assert_span_equal(dense, R, p)


@pytest.mark.parametrize("p", [2, 3, 7, 251, 32003, 65521])
@pytest.mark.parametrize("seed", range(4))
def test_rref_closed_form_G_times_R0(p, seed):
    """RREF(G * R0) == R0 when G has full column rank: a closed form at any size."""
    rng = np.random.default_rng(seed * 31 + p)
    m, n, r = 24, 30, 11
    R0, _ = random_rref(rng, r, n, p, density=0.7)
    G = full_col_rank(rng, m, r, p)
    M = (G @ R0) % p
    R = run_rref(M, p)
    assert R.shape == R0.shape and (R == R0).all()


def test_special_cases():
    p = 65521
    I = np.eye(7, dtype=np.int64)
    assert (run_rref(I, p) == I).all()
    perm = np.random.default_rng(3).permutation(7)
    assert (run_rref(I[perm] * 5, p) == I).all()
    Z = np.zeros((4, 6), np.int64)
    assert run_rref(Z, p).shape == (0, 6)
    u = np.array([3, 0, 9, 1], np.int64)
    v = np.array([0, 0, 4, 7, 0, 2], np.int64)
    R = run_rref(np.outer(u, v) % p, p)
    inv4 = pow(4, p - 2, p)
    assert R.shape == (1, 6) and (R[0] == v * inv4 % p).all()
    D = np.array([[0, 2, 3], [0, 2, 3], [0, 4, 6]], np.int64)
    R = run_rref(D, p)
    inv2 = pow(2, p - 2, p)
    assert R.shape == (1, 3) and (R[0] == np.array([0, 1, 3 * inv2 % p])).all()
    # p = 2: xor algebra
    X = np.array([[1, 1, 0], [0, 1, 1], [1, 0, 1]], np.int64)
    R = run_rref(X, 2)
    assert (R == np.array([[1, 0, 1], [0, 1, 1]])).all()
    # m = 0, n = 0 and all-empty rows
    r, rp, c, v = oracle.rref(0, 5, p, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.uint16))
    assert r == 0
    r, rp, c, v = oracle.rref(3, 0, p, np.zeros(4, np.int64), np.zeros(0, np.int32), np.zeros(0, np.uint16))
    assert r == 0


def test_vandermonde_full_rank():
    """A Vandermonde matrix with distinct nodes has full row rank, and any m
    leading columns are independent, so the RREF is [I | V1^-1 V2]."""
    p = 65521
    m, n = 9, 14
    nodes = np.arange(2, 2 + m)
    V = np.array([[pow(int(x), j, p) for j in range(n)] for x in nodes], np.int64)
    R = run_rref(V, p)
    assert R.shape == (m, n)
    assert (R[:, :m] == np.eye(m, dtype=np.int64)).all()
    assert_span_equal(V, R, p)


@pytest.mark.parametrize("seed", range(6))
def test_rref_invariants_on_fl_shaped(seed):
    p = 65521 if seed % 2 == 0 else 32003
    spec = synth.FLSpec(m=70, n=90, npiv=40, p=p, density=0.08, run_len=(2, 6), seed=seed)
    rp, c, v = synth.fl_matrix(spec)
    M = synth.csr_to_dense(spec.m, spec.n, rp, c, v)
    R = run_rref(M, p)
    assert_rref_shape(R, p)
    assert_span_equal(M, R, p)


def test_invalid_inputs_rejected():
    p = 65521
    rp = np.array([0, 2], np.int64)
    with pytest.raises(oracle.OracleError):
        oracle.rref(1, 4, p, rp, np.array([2, 1], np.int32), np.array([1, 1], np.uint16))  # unsorted
    with pytest.raises(oracle.OracleError):
        oracle.rref(1, 4, p, rp, np.array([1, 4], np.int32), np.array([1, 1], np.uint16))  # out of range
    with pytest.raises(oracle.OracleError):
        oracle.rref(1, 4, p, rp, np.array([1, 2], np.int32), np.array([0, 1], np.uint16))  # explicit zero
    with pytest.raises(oracle.OracleError):
        oracle.rref(1, 4, 65535, rp, np.array([1, 2], np.int32), np.array([1, 1], np.uint16))  # not prime


# ------------------------------------------------------------ echelon form
def test_pivot_choice_golden():
    g = json.load(open(os.path.join(GOLDEN, "pivot_choice.json")))
    m, n = g["m"], g["n"]
    dense = np.zeros((m, n), np.int64)
    for i, row in enumerate(g["rows"]):
        for c, v in row:
            dense[i, c] = v
    rp, c, v = to_csr(dense)
    piv = oracle.pivots(m, n, rp, c)
    assert list(piv) == g["expected_piv_row"]
    r, orp, oc, ov, npiv = oracle.echelon(m, n, 11, rp, c, v)
    assert npiv == g["expected_npiv"]


@pytest.mark.parametrize("seed", range(8))
def test_echelon_bottom_block_is_rref_rows(seed):
    """Bottom block = rows of RREF(M) whose pivot column is not a leading
    column of any input row; top block = chosen input rows, normalised."""
    p = [65521, 32003, 7, 65521][seed % 4]
    rng = np.random.default_rng(77 + seed)
    m, n, r = 40, 50, 25
    R0, pcs = random_rref(rng, r, n, p, density=0.3)
    G = full_col_rank(rng, m, r, p)
    # sparsify G so that several rows keep distinct leading columns
    G = np.where(rng.random(G.shape) < 0.25, G, 0)
    M = (G @ R0) % p
    E, npiv = run_echelon(M, p)
    leads = {int(np.nonzero(row)[0][0]) for row in M if row.any()}
    assert npiv == len(leads)
    # rank agrees with the closed form (G may have lost rank after sparsifying)
    R = run_rref(M, p)
    assert E.shape[0] == R.shape[0] == rank_colwise(M, p)
    e_piv = [int(np.nonzero(row)[0][0]) for row in E]
    assert e_piv == sorted(e_piv)
    for i, c in enumerate(e_piv):
        if c in leads:
            cands = [row for row in M if row.any() and int(np.nonzero(row)[0][0]) == c]
            w = min(int(np.count_nonzero(x)) for x in cands)
            first = next(x for x in cands if np.count_nonzero(x) == w)
            expect = first * pow(int(first[c]), p - 2, p) % p
            assert (E[i] == expect).all()
        else:
            j = [int(np.nonzero(row)[0][0]) for row in R].index(c)
            assert (E[i] == R[j]).all()
    assert_span_equal(M, R, p)


@pytest.mark.parametrize("seed", range(3))
def test_echelon_matches_rref_on_fl_shaped(seed):
    spec = synth.FLSpec(m=300, n=420, npiv=180, density=0.05, run_len=(3, 12), seed=500 + seed)
    rp, c, v = synth.fl_matrix(spec)
    r1, rp1, c1, v1 = oracle.rref(spec.m, spec.n, spec.p, rp, c, v)
    r2, rp2, c2, v2, npiv = oracle.echelon(spec.m, spec.n, spec.p, rp, c, v)
    assert r1 == r2
    R = synth.csr_to_dense(r1, spec.n, rp1, c1, v1)
    E = synth.csr_to_dense(r2, spec.n, rp2, c2, v2)
    M = synth.csr_to_dense(spec.m, spec.n, rp, c, v)
    leads = {int(c[rp[i]]) for i in range(spec.m) if rp[i + 1] > rp[i]}
    Rp = [int(np.nonzero(row)[0][0]) for row in R]
    for i, row in enumerate(E):
        c0 = int(np.nonzero(row)[0][0])
        if c0 not in leads:
            assert (row == R[Rp.index(c0)]).all()
    assert_rref_shape(R, spec.p)
    pc = Rp
    assert not ((M - M[:, pc] @ R) % spec.p).any()


# -------------------------------------------------------------- multiline
def test_multiline_example1_golden():
    g = json.load(open(os.path.join(GOLDEN, "multiline_example1.json")))
    r1, r2 = np.array(g["r1"]), np.array(g["r2"])
    p1, p2 = np.nonzero(r1)[0], np.nonzero(r2)[0]
    assert list(p1) == g["p1"] and list(r1[p1]) == g["v1"]
    assert list(p2) == g["p2"] and list(r2[p2]) == g["v2"]
    pos, val = oracle.multiline(p1, r1[p1], p2, r2[p2])
    assert list(pos) == g["ml_pos"]
    assert list(val) == g["ml_val"]
    assert int((val == 0).sum()) == g["padding_zeros"]


# -------------------------------------------------------------- mutants
def _pins_pass(mutant):
    try:
        for seed in range(25):
            rng = np.random.default_rng(seed)
            m = int(rng.integers(2, 5))
            n = int(rng.integers(2, 6))
            dense = np.where(rng.random((m, n)) < 0.7, rng.integers(1, 7, size=(m, n)), 0)
            if not (run_rref(dense, 7, mutant) == brute_rref(dense, 7)).all():
                return False
        g = json.load(open(os.path.join(GOLDEN, "pivot_choice.json")))
        dense = np.zeros((g["m"], g["n"]), np.int64)
        for i, row in enumerate(g["rows"]):
            for c, v in row:
                dense[i, c] = v
        rp, c, v = to_csr(dense)
        if list(oracle.pivots(g["m"], g["n"], rp, c, mutant=mutant)) != g["expected_piv_row"]:
            return False
    except (AssertionError, ValueError):
        return False
    return True


@pytest.mark.parametrize("mutant", [1, 2, 3])
def test_planted_mistakes_fail_the_pins(mutant):
    assert _pins_pass(0)
    assert not _pins_pass(mutant)
