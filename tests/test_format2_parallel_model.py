"""The data-parallel decoding of Format 2 (Sec. 3.2) checked against the oracle
reader on the CPU, step for step as the device decoder runs it:

1. row_ptr and the polynomial starts are exclusive scans of rows[] and prow[];
2. every column entry is classified without a sequential pass: g = inclusive
   count of masked (lone) entries, last[e] = the position of the g[e]-th
   masked entry (scattered), and an unmasked entry is a run start when its
   distance to `last` is odd, a run length when it is even;
3. entries emit 1 (lone), s (start, s read from the next entry) or 0 columns;
   off = exclusive scan of those counts;
4. output position q belongs to the last entry with off <= q (binary search),
   its column is the lone column or the run start plus q - off;
5. a run must stay inside the row its first column falls in, columns rise
   within a row and stay below n;
6. row i takes polynomial polmap[i]'s coefficients (same length), mod p,
   nonzero.
"""
import numpy as np
import pytest

from oracle import formats as F
from paper_1602_06097_gb300 import synth

M31 = 1 << 31


class ModelError(ValueError):
    pass


def parse(buf):
    """Header and sections of a Format 2 file (the host side of the decoder)."""
    b, m, n = np.frombuffer(buf, "<u4", 3, 0)
    p, nnz = np.frombuffer(buf, "<u8", 2, 12)
    m, n, p, nnz = int(m), int(n), int(p), int(nnz)
    o = 28
    rows = np.frombuffer(buf, "<u4", m, o).astype(np.int64); o += 4 * m
    polmap = np.frombuffer(buf, "<u4", m, o).astype(np.int64); o += 4 * m
    k = int(np.frombuffer(buf, "<u8", 1, o)[0]); o += 8
    colid = np.frombuffer(buf, "<u8", k, o).astype(np.uint64); o += 8 * k
    pnb = int(np.frombuffer(buf, "<u4", 1, o)[0]); o += 4
    pnnz = int(np.frombuffer(buf, "<u8", 1, o)[0]); o += 8
    prow = np.frombuffer(buf, "<u4", pnb, o).astype(np.int64); o += 4 * pnb
    vt = F.value_type(int(b))
    pdata = np.frombuffer(buf, "<" + vt, pnnz, o)
    if o + pdata.nbytes != len(buf):
        raise ModelError("size")
    return m, n, p, nnz, rows, polmap, colid, prow, pdata


def model_decode(buf):
    m, n, p, nnz, rows, polmap, colid, prow, pdata = parse(buf)
    if p < 2 or p >= 1 << 16:
        raise ModelError("p")
    k = len(colid)
    # 1. scans
    row_ptr = np.concatenate([[0], np.cumsum(rows)]).astype(np.int64)
    pstart = np.concatenate([[0], np.cumsum(prow)]).astype(np.int64)
    if row_ptr[-1] != nnz or pstart[-1] != len(pdata):
        raise ModelError("totals")
    # 2. roles
    if np.any(colid >> np.uint64(32)):
        raise ModelError("high bits")
    masked = ((colid >> np.uint64(31)) & np.uint64(1)).astype(np.int64)
    g = np.cumsum(masked)
    lastm = np.full(int(g[-1]) + 1 if k else 1, -1, np.int64)
    mpos = np.nonzero(masked)[0]
    lastm[g[mpos]] = mpos
    e = np.arange(k)
    last = np.where(g > 0, lastm[g], -1)
    dist = e - last
    lone = masked == 1
    start = ~lone & (dist % 2 == 1)
    # 3. counts
    nxt_ok = np.zeros(k, bool)
    nxt_ok[:-1] = ~lone[1:]
    if np.any(start & ~nxt_ok):
        raise ModelError("start without length")
    cnt = np.where(lone, 1, 0).astype(np.int64)
    s_idx = np.nonzero(start)[0]
    cnt[s_idx] = colid[s_idx + 1].astype(np.int64)
    if np.any(cnt[s_idx] < 2):
        raise ModelError("short run")
    off = np.concatenate([[0], np.cumsum(cnt)[:-1]]) if k else np.zeros(0, np.int64)
    if int(cnt.sum()) != nnz:
        raise ModelError("count")
    # 4. expand
    q = np.arange(nnz)
    eq = np.searchsorted(off, q, side="right") - 1
    col = np.where(lone[eq], (colid[eq] & np.uint64(M31 - 1)).astype(np.int64),
                   colid[eq].astype(np.int64) + (q - off[eq]))
    # 5. checks
    row_of = lambda x: np.searchsorted(row_ptr, x, side="right") - 1
    if len(s_idx) and np.any(row_of(off[s_idx]) != row_of(off[s_idx] + cnt[s_idx] - 1)):
        raise ModelError("run crosses a row")
    if nnz and (col.min() < 0 or col.max() >= n):
        raise ModelError("column range")
    same_row = row_of(q[:-1]) == row_of(q[1:]) if nnz > 1 else np.zeros(0, bool)
    if np.any(same_row & (col[1:] <= col[:-1])):
        raise ModelError("order")
    # 6. values
    if np.any(polmap >= len(prow)) or np.any(prow[np.minimum(polmap, len(prow) - 1)] != rows):
        raise ModelError("polynomials")
    val = np.zeros(nnz, np.int64)
    for i in range(m):
        j = polmap[i]
        val[row_ptr[i]:row_ptr[i + 1]] = pdata[pstart[j]:pstart[j] + rows[i]].astype(np.int64) % p
    if np.any(val == 0):
        raise ModelError("zero")
    return m, n, p, row_ptr, col, val


def same(a, b):
    assert a[:3] == b[:3]
    for x, y in zip(a[3:], b[3:]):
        assert np.array_equal(np.asarray(x, np.int64), np.asarray(y, np.int64))


@pytest.mark.parametrize("seed", range(6))
def test_model_equals_oracle_reader(seed):
    rng = np.random.default_rng(seed)
    for _ in range(4):
        m, n = int(rng.integers(1, 60)), int(rng.integers(1, 90))
        p = int(rng.choice([2, 13, 251, 32003, 65521]))
        rp, c, v = synth.random_csr(rng, m, n, p, float(rng.uniform(0.0, 0.6)))
        vt = rng.choice([None, "i1", "i2", "u4", "i8"]) if p < 128 else rng.choice([None, "u4", "i4", "i8"])
        buf = synth.encode_format2(m, n, p, rp, c, v, vt)
        same(model_decode(buf), F.decode_format2(buf))


def test_model_on_fl_workload():
    spec = synth.workload("fl_2000x3000")
    rp, c, v = synth.fl_matrix(spec)
    buf = synth.encode_format2(spec.m, spec.n, spec.p, rp, c, v)
    same(model_decode(buf), F.decode_format2(buf))


def test_model_rejects_what_the_oracle_rejects():
    from test_formats import hand_format2, corrupt, OFF_COLID, OFF_POLMAP, OFF_PDATA
    good = hand_format2(1, 251, "B", [5, 6, 7, 9, 3, 250])
    same(model_decode(good), F.decode_format2(good))
    bad = [corrupt(good, OFF_COLID + 8, "<Q", 5), corrupt(good, OFF_COLID + 8, "<Q", 1),
           corrupt(good, OFF_COLID + 16, "<Q", 10 | M31), corrupt(good, OFF_COLID + 16, "<Q", 2 | M31),
           corrupt(good, OFF_COLID + 24, "<Q", (1 << 40) | 4 | M31), corrupt(good, OFF_POLMAP + 4, "<I", 2),
           corrupt(good, OFF_POLMAP + 4, "<I", 0), corrupt(good, OFF_PDATA + 2, "<B", 0),
           corrupt(good, OFF_COLID + 48, "<Q", 4 | M31),     # the last run loses its length
           corrupt(good, 12, "<Q", 1 << 17)]
    for buf in bad:
        with pytest.raises(F.FormatError):
            F.decode_format2(buf)
        with pytest.raises((ModelError, IndexError)):
            model_decode(buf)
