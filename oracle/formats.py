"""Plain CPU decoders of the paper's binary matrix files (Sec. 3.2, Table 2).

TEST INFRASTRUCTURE ONLY, like the rest of this package: only ``tests/`` may
import it.  It is the reference for decoding a file into the CSR input of the
reduction (row pointers int64, columns int32 strictly increasing per row,
values uint16 in [1, p)), written field by field from the table's order and
the section's rules, with every check spelt out.  The files' encoder used in
the tests lives with the input generators (``paper_1602_06097_gb300.synth``);
the two share no code.

Format 1 (Table 2, left): u32 m, u32 n, u32 p, u64 nnz, u16 data[nnz],
u32 cols[nnz], u32 rows[m] -- rows[i] is the length of row i, and row i's
entries are the next rows[i] (cols, data) pairs.

Format 2 (Table 2, right; Sec. 3.2):
  u32 b        -- bits 0-2: value type, b = u | (v << 1), 8 * 2^v bits;
                  the higher bits hold a version and are ignored here
  u32 m, u32 n, u64 p, u64 nnz
  u32 rows[m]  -- row lengths
  u32 polmap[m]-- row i carries the coefficients of polynomial polmap[i]
  u64 k, u64 colid[k]
                -- the rows' columns, row after row, compressed: a run of
                   s > 1 consecutive columns starting at f is the pair f, s;
                   a single column f is one entry f | 2^31
  u32 pnb, u64 pnnz, u32 prow[pnb]
                -- prow[j] = number of coefficients of polynomial j
  pdata[pnnz]  -- the polynomials' coefficients one after the other, in the
                  type given by b

Readings where the section is silent or garbled (listed in the design notes):
the mask of a single column is written with AND, which would erase f, so it is
read as OR; the type bit u is described as "1 iff signed" while the worked
example gives b = 0b011 for uint16, so the example is followed (u = 1:
unsigned); byte order is little-endian; a run never crosses the end of a row;
polynomial polmap[i] must have exactly rows[i] coefficients; a signed
coefficient is taken mod p; a coefficient that is 0 mod p is an explicit zero
and is rejected, as is anything left over after the last field.
"""
from __future__ import annotations

import numpy as np

MASK31 = 1 << 31


class FormatError(ValueError):
    """A file that does not follow the format."""


class _Reader:
    def __init__(self, buf: bytes):
        self.buf = memoryview(buf)
        self.pos = 0

    def take(self, dtype, count: int):
        dt = np.dtype(dtype).newbyteorder("<")
        nbytes = dt.itemsize * int(count)
        if count < 0 or self.pos + nbytes > len(self.buf):
            raise FormatError("file ends inside a field")
        out = np.frombuffer(self.buf[self.pos:self.pos + nbytes], dtype=dt).astype(dt.newbyteorder("="))
        self.pos += nbytes
        return out

    def one(self, dtype) -> int:
        return int(self.take(dtype, 1)[0])

    def finish(self):
        if self.pos != len(self.buf):
            raise FormatError("bytes left after the last field")


def _check_p(p):
    if p < 2 or p >= 1 << 16:
        raise FormatError("p must lie in [2, 2^16) for the reduction's input")


def _csr(m, n, p, lengths, cols, vals):
    """Checks of the CSR the reduction accepts (vals already reduced mod p),
    then the arrays."""
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(np.asarray(lengths, dtype=np.int64))
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.int64)
    if len(cols) != row_ptr[-1] or len(vals) != row_ptr[-1]:
        raise FormatError("row lengths and entries disagree")
    for i in range(m):
        c = cols[row_ptr[i]:row_ptr[i + 1]]
        if len(c) and (c[0] < 0 or c[-1] >= n or np.any(np.diff(c) <= 0)):
            raise FormatError(f"row {i}: columns out of range or not increasing")
    if np.any(vals == 0):
        raise FormatError("an explicit zero coefficient")
    return row_ptr, cols.astype(np.int32), vals.astype(np.uint16)


def decode_format1(buf: bytes):
    """Format 1 file -> (m, n, p, row_ptr, col, val)."""
    r = _Reader(buf)
    m = r.one("u4")
    n = r.one("u4")
    p = r.one("u4")
    nnz = r.one("u8")
    data = r.take("u2", nnz)
    cols = r.take("u4", nnz)
    rows = r.take("u4", m)
    r.finish()
    _check_p(p)
    if int(rows.astype(np.int64).sum()) != nnz:
        raise FormatError("row lengths do not add up to nnz")
    row_ptr, col, val = _csr(m, n, p, rows, cols, data.astype(np.int64) % p)
    return m, n, p, row_ptr, col, val


_TYPES = {(1, 0): "u1", (1, 1): "u2", (1, 2): "u4", (1, 3): "u8",
          (0, 0): "i1", (0, 1): "i2", (0, 2): "i4", (0, 3): "i8"}


def value_type(b: int) -> str:
    """numpy type code of the coefficients from the low three bits of b."""
    u, v = b & 1, (b >> 1) & 3
    return _TYPES[(u, v)]


def decode_columns(colid, rows, n):
    """The run-compressed column stream -> the columns of every row, in order."""
    out = []
    e = 0
    k = len(colid)
    for i, length in enumerate(rows):
        left = int(length)
        while left > 0:
            if e >= k:
                raise FormatError("column stream ends early")
            x = int(colid[e])
            if x >> 32:
                raise FormatError("column entry above 32 bits")
            if x & MASK31:
                out.append(x & (MASK31 - 1))
                left -= 1
                e += 1
            else:
                if e + 1 >= k:
                    raise FormatError("run without its length")
                s = int(colid[e + 1])
                if s < 2 or s > left:
                    raise FormatError(f"row {i}: run length {s} invalid or crossing the row's end")
                if x + s > n:
                    raise FormatError(f"row {i}: run past the last column")
                out.extend(range(x, x + s))
                left -= s
                e += 2
    if e != k:
        raise FormatError("column entries left after the last row")
    return out


def decode_format2(buf: bytes):
    """Format 2 file -> (m, n, p, row_ptr, col, val)."""
    r = _Reader(buf)
    b = r.one("u4")
    m = r.one("u4")
    n = r.one("u4")
    p = r.one("u8")
    nnz = r.one("u8")
    rows = r.take("u4", m).astype(np.int64)
    polmap = r.take("u4", m).astype(np.int64)
    k = r.one("u8")
    colid = r.take("u8", k)
    pnb = r.one("u4")
    pnnz = r.one("u8")
    prow = r.take("u4", pnb).astype(np.int64)
    pdata = r.take(value_type(b), pnnz)
    r.finish()
    _check_p(p)
    if m >= MASK31:
        raise FormatError("m must be below 2^31")
    if int(rows.sum()) != nnz:
        raise FormatError("row lengths do not add up to nnz")
    if int(prow.sum()) != pnnz:
        raise FormatError("polynomial lengths do not add up to pnnz")
    start = np.zeros(pnb + 1, dtype=np.int64)
    start[1:] = np.cumsum(prow)
    vals = []
    for i in range(m):
        j = int(polmap[i])
        if j >= pnb:
            raise FormatError(f"row {i}: polynomial {j} does not exist")
        if prow[j] != rows[i]:
            raise FormatError(f"row {i}: {rows[i]} columns but polynomial {j} has {prow[j]} coefficients")
        vals.extend(int(x) % p for x in pdata[start[j]:start[j + 1]])
    cols = decode_columns(colid, rows, n)
    row_ptr, col, val = _csr(m, n, p, rows, cols, vals)
    return m, n, p, row_ptr, col, val
