"""Full-size checks on the 40,000 x 60,000 grouped workload, in the
configuration the benchmark times (input resident on the device, echelon
form of the new order).

The oracle needs about ten minutes of CPU for this matrix, so its result was
computed once by ``tests/golden/make_oracle_digest.py`` (which calls only the
oracle and the input generator) and stored as a SHA-256 digest of its CSR
arrays in ``tests/golden/oracle_fl_40000x60000.json``: the GPU result must
hash to the same digest (bit-exact, both paths).  Beside that exact check the
result is checked against what the oracle computes exactly at this size and
against properties that hold at any size:

1. The top block is exactly the oracle's choice of pivot rows (FL step 1,
   Sec. 3.1: fewest nonzeros, then smallest row index), each row multiplied by
   the inverse of its leading coefficient.
2. Every row has a unit leading entry and the leading columns strictly
   increase.
3. Every bottom row (one whose lead is not a top pivot column) vanishes at
   every other pivot column: the Schur block is in reduced echelon form and
   zero on the top pivot columns.
4. rowspace(input) is contained in rowspace(output): vectors of the output's
   null space (free columns random, pivot columns solved from the last row
   up) are annihilated by every input row.  An input row outside the span
   passes one such vector with probability 1/p.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from paper_1602_06097_gb300 import gbla, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def modpow(a, e, p):
    """Elementwise a^e mod p for an int64 array."""
    a = np.asarray(a, np.int64) % p
    r = np.ones_like(a)
    while e:
        if e & 1:
            r = r * a % p
        a = a * a % p
        e >>= 1
    return r


def segments(ptr, rows):
    """Concatenated element indices of the CSR rows `rows`."""
    starts, ends = ptr[rows], ptr[rows + 1]
    lens = ends - starts
    base = np.repeat(starts - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens)
    return base + np.arange(int(lens.sum()), dtype=np.int64), lens


@pytest.fixture(scope="module")
def full():
    spec = synth.workload("fl_40000x60000")
    rp, c, v = synth.fl_matrix(spec)
    d_rp = torch.from_numpy(rp).cuda()
    d_c = torch.from_numpy(c).cuda()
    d_v = torch.from_numpy(v.view(np.int16)).cuda()
    res = gbla.reduce_device(d_rp, d_c, d_v, (spec.m, spec.n), spec.p, want_reduced=False)
    try:
        rank, orp, oc, ov = res.to_host()
        stats = res.stats
    finally:
        res.free()
    out = (int(rank), orp.astype(np.int64), oc.astype(np.int64), ov.astype(np.int64))
    return spec, (rp, c.astype(np.int64), v.astype(np.int64)), out, stats


GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_fl_40000x60000.json")


def sha256_csr(row_ptr, col, val):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(row_ptr, dtype="<i8").tobytes())
    h.update(np.ascontiguousarray(col, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(val, dtype="<u2").tobytes())
    return h.hexdigest()


def test_fullsize_equals_the_oracle_bit_for_bit(full):
    spec, (rp, c, v), (rank, orp, oc, ov), st = full
    g = json.load(open(GOLDEN))
    assert sha256_csr(rp, c, v) == g["input_sha256"], "the generated input is not the one the oracle reduced"
    assert rank == g["rank"] and st["npiv"] == g["npiv"] and len(oc) == g["nnz"]
    assert sha256_csr(orp, oc, ov) == g["result_sha256"]


def test_fullsize_dense_path_equals_the_oracle_bit_for_bit(full):
    spec, (rp, c, v), _, _ = full
    g = json.load(open(GOLDEN))
    d = (torch.from_numpy(rp).cuda(), torch.from_numpy(c.astype(np.int32)).cuda(),
         torch.from_numpy(v.astype(np.uint16).view(np.int16)).cuda())
    res = gbla.reduce_device(*d, (spec.m, spec.n), spec.p, path=gbla.PATH_DENSE)
    try:
        rank, orp, oc, ov = res.to_host()
        assert res.stats["path"] == gbla.PATH_DENSE
    finally:
        res.free()
    assert rank == g["rank"]
    assert sha256_csr(orp, oc, ov) == g["result_sha256"]


def test_fullsize_counts(full):
    spec, _, (rank, orp, oc, ov), st = full
    assert rank == st["npiv"] + st["rank_d"]
    assert len(orp) == rank + 1 and orp[0] == 0 and orp[-1] == len(oc) == len(ov)
    assert np.all(np.diff(orp) > 0)
    assert np.all((ov > 0) & (ov < spec.p))
    assert np.all((oc >= 0) & (oc < spec.n))


def test_fullsize_top_block_is_the_normalised_pivot_rows(full):
    spec, (rp, c, v), (rank, orp, oc, ov), st = full
    p = spec.p
    piv = oracle.pivots(spec.m, spec.n, rp, c)
    pcols = np.nonzero(piv >= 0)[0]
    assert len(pcols) == st["npiv"]
    lead = oc[orp[:-1]]
    k = np.searchsorted(lead, pcols)
    assert np.all(k < rank) and np.all(lead[k] == pcols)
    rows_in = piv[pcols]
    idx_in, len_in = segments(rp, rows_in)
    idx_out, len_out = segments(orp, k)
    assert np.array_equal(len_in, len_out)
    assert np.array_equal(c[idx_in], oc[idx_out])
    inv = modpow(v[rp[rows_in]], p - 2, p)
    assert np.array_equal(v[idx_in] * np.repeat(inv, len_in) % p, ov[idx_out])


def test_fullsize_echelon_structure(full):
    spec, _, (rank, orp, oc, ov), st = full
    lead = oc[orp[:-1]]
    assert np.all(ov[orp[:-1]] == 1)
    assert np.all(np.diff(lead) > 0)
    top = np.zeros(spec.n, bool)
    top[np.nonzero(oracle.pivots(spec.m, spec.n, *full[1][:2]) >= 0)[0]] = True
    pivcol = np.zeros(spec.n, bool)
    pivcol[lead] = True
    bottom = np.nonzero(~top[lead])[0]
    assert len(bottom) == st["rank_d"]
    idx, lens = segments(orp, bottom)
    first = np.zeros(len(idx), bool)
    first[np.concatenate([[0], np.cumsum(lens)[:-1]])] = True
    assert not np.any(pivcol[oc[idx]] & ~first), "a bottom row has a nonzero at another pivot column"


def test_fullsize_input_rows_lie_in_the_output_span(full):
    spec, (rp, c, v), (rank, orp, oc, ov), _ = full
    p, n = spec.p, spec.n
    lead = oc[orp[:-1]]
    pivcol = np.zeros(n, bool)
    pivcol[lead] = True
    row_of = np.repeat(np.arange(spec.m), np.diff(rp))
    rng = np.random.default_rng(1602)
    for _ in range(2):
        z = rng.integers(0, p, size=n).astype(np.int64)
        z[pivcol] = 0
        for k in range(rank - 1, -1, -1):
            a, b = orp[k], orp[k + 1]
            s = int(np.dot(ov[a + 1:b], z[oc[a + 1:b]]) % p)
            z[lead[k]] = (p - s) % p
        # every output row annihilates z (its construction) ...
        prod_out = ov * z[oc]
        sums_out = np.bincount(np.repeat(np.arange(rank), np.diff(orp)), weights=prod_out, minlength=rank)
        assert np.all(np.mod(sums_out.astype(np.int64), p) == 0)
        # ... and so must every input row
        sums_in = np.bincount(row_of, weights=v * z[c], minlength=spec.m)
        assert np.all(np.mod(sums_in.astype(np.int64), p) == 0), "an input row is not in the output span"
