"""Pins of the oracle's 32-bit functions (oracle.rref32, oracle.echelon32:
primes p < 2^31, uint32 values, the paper's 32-bit coefficient type, Sec. 2).

What fixes the expected results, independently of the oracle:
1. sympy's reduced row echelon form over GF(p) (DomainMatrix over GF(p)), a
   library routine, on random and rank-deficient matrices at primes on both
   sides of 2^16 and up to 2^31 - 1;
2. closed forms at p = 2^31 - 1: identity, scaled permutation, rank one, zero;
3. invariants of an RREF on larger inputs: unit leads strictly increasing,
   pivot columns zero elsewhere, every input row the combination of the
   output rows given by its entries at the pivot columns;
4. below 2^16 the 32-bit entry point agrees with oracle.rref (pinned in
   tests/test_oracle.py);
5. malformed input is rejected;
6. the planted mistakes of the mutant builds (wrong sign, dropped term) fail
   pin 1;
7. the new-order echelon form: its top block is the FL step-1 pivot rows
   normalised, its bottom block sympy's RREF of the Schur complement
   D - C A^-1 B over GF(p) (inverse and RREF by sympy), and below 2^16 it
   agrees with oracle.echelon.
"""
import numpy as np
import pytest

import oracle

sympy = pytest.importorskip("sympy")
from sympy.polys.matrices import DomainMatrix  # noqa: E402

P31 = 2**31 - 1
PRIMES = [13, 65521, 65537, 1_000_000_007, P31]


def to_csr(d):
    d = np.asarray(d, dtype=np.int64)
    m, n = d.shape
    rp, col, val = [0], [], []
    for i in range(m):
        nz = np.nonzero(d[i])[0]
        col.extend(nz.tolist())
        val.extend(d[i, nz].tolist())
        rp.append(len(col))
    return (np.array(rp, np.int64), np.array(col, np.int32), np.array(val, np.uint32), m, n)


def dense_out(res, n):
    r, rp, col, val = res
    out = np.zeros((r, n), dtype=np.int64)
    for i in range(r):
        out[i, col[rp[i]:rp[i + 1]]] = val[rp[i]:rp[i + 1]]
    return out


def sympy_rref(d, p):
    m, n = d.shape
    F = sympy.GF(p)
    M = DomainMatrix([[F(int(x)) for x in row] for row in d], (m, n), F)
    R, pivots = M.rref()
    rows = [[int(F.to_sympy(x)) % p for x in R.to_list()[i]] for i in range(len(pivots))]
    return np.array(rows, dtype=np.int64).reshape(len(pivots), n)


def random_matrix(rng, m, n, p, density):
    d = rng.integers(1, p, size=(m, n), dtype=np.int64)
    return np.where(rng.random((m, n)) < density, d, 0)


def rank_deficient(rng, m, n, k, p):
    # rows = (m x k) @ (k x n) mod p with a sparse right factor
    g = rng.integers(0, p, size=(m, k), dtype=np.int64)
    b = random_matrix(rng, k, n, p, 0.4)
    out = np.zeros((m, n), dtype=object)
    for i in range(m):
        acc = [0] * n
        for t in range(k):
            if g[i, t]:
                for j in np.nonzero(b[t])[0]:
                    acc[j] = (acc[j] + int(g[i, t]) * int(b[t, j])) % p
        out[i] = acc
    return out.astype(np.int64)


@pytest.mark.parametrize("p", PRIMES)
@pytest.mark.parametrize("seed", range(3))
def test_rref32_equals_sympy_gf_p(p, seed):
    rng = np.random.default_rng(seed * 1000 + p % 997)
    for d in (random_matrix(rng, 12, 18, p, 0.5), rank_deficient(rng, 14, 16, 5, p)):
        rp, col, val, m, n = to_csr(d)
        got = dense_out(oracle.rref32(m, n, p, rp, col, val), n)
        assert np.array_equal(got, sympy_rref(d, p))


def test_rref32_closed_forms_at_2_31_minus_1():
    p, n = P31, 40
    rp, col, val, m, _ = to_csr(np.eye(n, dtype=np.int64))
    assert np.array_equal(dense_out(oracle.rref32(m, n, p, rp, col, val), n), np.eye(n, dtype=np.int64))
    rng = np.random.default_rng(5)
    perm = rng.permutation(n)
    scale = rng.integers(1, p, size=n, dtype=np.int64)
    d = np.zeros((n, n), dtype=np.int64)
    d[np.arange(n), perm] = scale
    rp, col, val, m, _ = to_csr(d)
    assert np.array_equal(dense_out(oracle.rref32(m, n, p, rp, col, val), n), np.eye(n, dtype=np.int64))
    # rank one: u w^T gives the single row w / w[lead]
    u = rng.integers(1, p, size=7, dtype=np.int64)
    w = np.where(rng.random(30) < 0.5, rng.integers(1, p, size=30, dtype=np.int64), 0)
    w[4] = 12345
    d = np.array([[int(a) * int(b) % p for b in w] for a in u], dtype=np.int64)
    rp, col, val, m, n1 = to_csr(d)
    lead = int(np.nonzero(w)[0][0])
    inv = pow(int(w[lead]), p - 2, p)
    expect = np.array([[int(x) * inv % p for x in w]], dtype=np.int64)
    assert np.array_equal(dense_out(oracle.rref32(m, n1, p, rp, col, val), n1), expect)
    # zero matrix: rank 0
    rp, col, val, m, n2 = to_csr(np.zeros((5, 9), dtype=np.int64))
    assert oracle.rref32(m, n2, p, rp, col, val)[0] == 0


@pytest.mark.parametrize("p", [65537, P31])
def test_rref32_invariants_on_larger_inputs(p):
    rng = np.random.default_rng(p % 1009)
    d = random_matrix(rng, 60, 90, p, 0.08)
    d[30:40] = d[0:10]                                  # dependent rows
    rp, col, val, m, n = to_csr(d)
    r, orp, ocol, oval = oracle.rref32(m, n, p, rp, col, val)
    R = dense_out((r, orp, ocol, oval), n)
    leads = [int(np.nonzero(R[i])[0][0]) for i in range(r)]
    assert all(R[i, leads[i]] == 1 for i in range(r))
    assert all(a < b for a, b in zip(leads, leads[1:]))
    for i, c in enumerate(leads):                       # pivot columns zero elsewhere
        assert np.count_nonzero(R[:, c]) == 1 and R[i, c] == 1
    for x in d:                                         # input rows lie in the span
        comb = np.zeros(n, dtype=object)
        for i, c in enumerate(leads):
            if x[c]:
                comb = (comb + int(x[c]) * R[i].astype(object)) % p
        assert np.array_equal(np.asarray(comb, dtype=np.int64), x % p)
    assert r == len(sympy_rref(d, p))


def test_rref32_agrees_with_the_16_bit_oracle():
    p = 65521
    rng = np.random.default_rng(7)
    d = random_matrix(rng, 40, 70, p, 0.15)
    rp, col, val, m, n = to_csr(d)
    r32 = oracle.rref32(m, n, p, rp, col, val)
    r16 = oracle.rref(m, n, p, rp, col, val.astype(np.uint16))
    assert r32[0] == r16[0]
    for a, b in zip(r32[1:], r16[1:]):
        assert np.array_equal(np.asarray(a, np.int64), np.asarray(b, np.int64))


@pytest.mark.parametrize("case", ["p not prime", "p too large", "value >= p", "explicit zero"])
def test_rref32_rejects_malformed_input(case):
    p = {"p not prime": 2**31 - 3, "p too large": 2**31 + 11}.get(case, P31)
    rp = np.array([0, 2], np.int64)
    col = np.array([0, 3], np.int32)
    val = np.array({"value >= p": [1, P31], "explicit zero": [1, 0]}.get(case, [1, 2]), np.uint32)
    with pytest.raises(oracle.OracleError):
        oracle.rref32(1, 5, p, rp, col, val)


@pytest.mark.parametrize("mutant", [1, 2])
def test_planted_mistakes_fail_the_sympy_pin(mutant):
    p = P31
    rng = np.random.default_rng(11)
    d = random_matrix(rng, 12, 16, p, 0.6)
    rp, col, val, m, n = to_csr(d)
    got = dense_out(oracle.rref32(m, n, p, rp, col, val, mutant=mutant), n)
    assert not np.array_equal(got, sympy_rref(d, p))


# ------------------------------------------------ new-order echelon, 32 bits
def split_expected(d, p):
    """The echelon form fixed by the mathematics: the FL step-1 pivot rows
    (leftmost nonzero; fewest nonzeros, then smallest index) normalised to a
    leading 1, and RREF(D - C A^-1 B) over GF(p) by sympy, placed at the
    non-pivot columns; rows ordered by pivot column."""
    m, n = d.shape
    F = sympy.GF(p)
    best = {}
    for i in range(m):
        nz = np.nonzero(d[i])[0]
        if len(nz) == 0:
            continue
        c, w = int(nz[0]), len(nz)
        if c not in best or w < best[c][1]:
            best[c] = (i, w)
    pcols = sorted(best)
    prows = [best[c][0] for c in pcols]
    others = [i for i in range(m) if i not in set(prows) and np.any(d[i])]
    npc = [c for c in range(n) if c not in best]
    rows = {}
    for c, i in zip(pcols, prows):
        inv = pow(int(d[i, c]), p - 2, p)
        rows[c] = [int(x) * inv % p for x in d[i]]
    if others and npc:
        def dm(sub):
            return DomainMatrix([[F(int(x)) for x in r] for r in sub], (len(sub), len(sub[0]) if sub else 0), F)
        A = dm([[d[i, c] for c in pcols] for i in prows]) if pcols else None
        Bm = dm([[d[i, c] for c in npc] for i in prows]) if pcols else None
        Cm = dm([[d[i, c] for c in pcols] for i in others]) if pcols else None
        Dm = dm([[d[i, c] for c in npc] for i in others])
        S = Dm - Cm * A.inv() * Bm if pcols else Dm
        R, piv = S.rref()
        Rl = R.to_list()
        for t, pc in enumerate(piv):
            row = [0] * n
            for j, c in enumerate(npc):
                row[c] = int(F.to_sympy(Rl[t][j])) % p
            rows[npc[pc]] = row
    order = sorted(rows)
    return np.array([rows[c] for c in order], dtype=np.int64).reshape(len(order), n), len(pcols)


@pytest.mark.parametrize("p", PRIMES)
@pytest.mark.parametrize("seed", range(3))
def test_echelon32_equals_the_split_through_sympy(p, seed):
    rng = np.random.default_rng(seed * 7919 + p % 991)
    # a nearly triangular matrix: staircase pivot rows plus dense-ish others
    m, n = 16, 22
    d = np.zeros((m, n), dtype=np.int64)
    for i in range(8):
        d[i, 2 * i] = rng.integers(1, p)
        extra = rng.random(n) < 0.3
        extra[:2 * i + 1] = False
        d[i, extra] = rng.integers(1, p, size=int(extra.sum()))
    d[8:] = random_matrix(rng, m - 8, n, p, 0.4)
    d[14] = d[9]                                         # a dependent row
    rp, col, val, mm, nn = to_csr(d)
    r, orp, ocol, oval, npiv = oracle.echelon32(mm, nn, p, rp, col, val)
    expect, enpiv = split_expected(d, p)
    assert npiv == enpiv and r == len(expect)
    assert np.array_equal(dense_out((r, orp, ocol, oval), nn), expect)


def test_echelon32_agrees_with_the_16_bit_oracle():
    p = 65521
    rng = np.random.default_rng(17)
    d = random_matrix(rng, 50, 80, p, 0.1)
    rp, col, val, m, n = to_csr(d)
    a = oracle.echelon32(m, n, p, rp, col, val)
    b = oracle.echelon(m, n, p, rp, col, val.astype(np.uint16))
    assert a[0] == b[0] and a[4] == b[4]
    for x, y in zip(a[1:4], b[1:4]):
        assert np.array_equal(np.asarray(x, np.int64), np.asarray(y, np.int64))


def test_echelon32_rejects_a_composite_modulus():
    rp, col, val, m, n = to_csr(np.eye(3, dtype=np.int64))
    with pytest.raises(oracle.OracleError):
        oracle.echelon32(m, n, 2**31 - 3, rp, col, val)
