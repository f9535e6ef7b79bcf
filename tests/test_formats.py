"""The binary matrix files of Sec. 3.2 (Table 2): the oracle's readers pinned by
files assembled by hand, field by field in the table's order, then round trips
through the writers of the input generators, and malformed files.

The hand-worked Format 2 file is a 3 x 10 matrix over GF(251):
  row 0: columns 1, 2, 3, 7 with the coefficients of polynomial 0 (5, 6, 7, 9)
  row 1: columns 4, 9 with the coefficients of polynomial 1 (3, 250)
  row 2: columns 2, 3, 4, 5 with the coefficients of polynomial 0 again
so the column stream is 1, 3 (a run of 3 from column 1), 7|2^31 (a lone
column), 4|2^31, 9|2^31, 2, 4 (a run of 4 from column 2): k = 7 entries; the
coefficients are stored once per polynomial, in the unsigned 8-bit type
(b = 1 | 0 << 1 = 1).  A reader that takes the lone-column mask as AND, maps
coefficients by row instead of through polmap, or reads the type bit the
other way round fails one of these files.
"""
import struct

import numpy as np
import pytest

from oracle import formats as F
from paper_1602_06097_gb300 import synth

M31 = 1 << 31


def hand_format2(b, p, pdata_fmt, pdata):
    """The 3 x 10 example above, with its coefficients in the given type."""
    out = struct.pack("<I", b)
    out += struct.pack("<II", 3, 10)                       # m, n
    out += struct.pack("<QQ", p, 10)                       # p, nnz
    out += struct.pack("<III", 4, 2, 4)                    # rows
    out += struct.pack("<III", 0, 1, 0)                    # polmap
    out += struct.pack("<Q", 7)                            # k
    out += struct.pack("<7Q", 1, 3, 7 | M31, 4 | M31, 9 | M31, 2, 4)
    out += struct.pack("<I", 2)                            # pnb
    out += struct.pack("<Q", 6)                            # pnnz
    out += struct.pack("<II", 4, 2)                        # prow
    out += struct.pack("<" + pdata_fmt * 6, *pdata)        # pdata
    return out


def test_format2_hand_worked_example():
    m, n, p, rp, c, v = F.decode_format2(hand_format2(1, 251, "B", [5, 6, 7, 9, 3, 250]))
    assert (m, n, p) == (3, 10, 251)
    assert rp.tolist() == [0, 4, 6, 10]
    assert c.tolist() == [1, 2, 3, 7, 4, 9, 2, 3, 4, 5]
    assert v.tolist() == [5, 6, 7, 9, 3, 250, 5, 6, 7, 9]


def test_format2_signed_16_bit_coefficients():
    # b = 0 | 1 << 1: signed 16-bit; over GF(7) the coefficients -1, -3 are 6, 4
    _, _, p, _, _, v = F.decode_format2(hand_format2(2, 7, "h", [1, -1, 2, 3, -3, 5]))
    assert p == 7
    assert v.tolist() == [1, 6, 2, 3, 4, 5, 1, 6, 2, 3]


def test_format2_version_bits_are_ignored():
    _, _, _, _, c, v = F.decode_format2(hand_format2(1 | (2 << 28), 251, "B", [5, 6, 7, 9, 3, 250]))
    assert c.tolist()[:4] == [1, 2, 3, 7] and v.tolist()[4:6] == [3, 250]


def test_format1_hand_worked_example():
    # 2 x 5 over GF(13): row 0 = (0, 4, 0, 0, 12), row 1 = (7, 0, 0, 1, 0)
    buf = struct.pack("<III", 2, 5, 13) + struct.pack("<Q", 4)
    buf += struct.pack("<4H", 4, 12, 7, 1) + struct.pack("<4I", 1, 4, 0, 3) + struct.pack("<2I", 2, 2)
    m, n, p, rp, c, v = F.decode_format1(buf)
    assert (m, n, p) == (2, 5, 13)
    assert rp.tolist() == [0, 2, 4] and c.tolist() == [1, 4, 0, 3] and v.tolist() == [4, 12, 7, 1]


def same(a, b):
    assert a[:3] == b[:3]
    for x, y in zip(a[3:], b[3:]):
        assert np.array_equal(np.asarray(x, np.int64), np.asarray(y, np.int64))


@pytest.mark.parametrize("vtype", [None, "u2", "u4", "u8", "i2", "i4", "i8"])
def test_round_trip_fl_workload(vtype):
    spec = synth.workload("fl_2000x3000")
    rp, c, v = synth.fl_matrix(spec)
    ref = (spec.m, spec.n, spec.p, rp, c, v)
    same(F.decode_format2(synth.encode_format2(spec.m, spec.n, spec.p, rp, c, v, vtype)), ref)
    same(F.decode_format1(synth.encode_format1(spec.m, spec.n, spec.p, rp, c, v)), ref)


def test_round_trip_small_primes_and_byte_types():
    rng = np.random.default_rng(7)
    for p in (2, 3, 13, 127, 251):
        for vtype in ("u1", "i1", "i2"):
            m, n = 40, 70
            rp, c, v = synth.random_csr(rng, m, n, p, 0.2)
            buf = synth.encode_format2(m, n, p, rp, c, v, vtype)
            same(F.decode_format2(buf), (m, n, p, rp, c, v))


def test_round_trip_edge_shapes():
    rng = np.random.default_rng(8)
    cases = [np.zeros((3, 4), np.int64),                       # no entries
             np.array([[0, 0, 5]]),                             # one lone column at the end
             np.array([[1, 2, 3, 4]]),                          # one run over the whole row
             np.eye(6, dtype=np.int64) * 3,                     # lone columns only
             rng.integers(0, 2, (30, 50)) * rng.integers(1, 65521, (30, 50))]
    for d in cases:
        m, n = d.shape
        rp, c, v = synth.dense_to_csr(d)
        same(F.decode_format2(synth.encode_format2(m, n, 65521, rp, c, v)), (m, n, 65521, rp, c, v))


def test_shared_polynomials_are_stored_once():
    """Rows that are monomial shifts of one polynomial (the same coefficients
    at shifted columns) share one polynomial in Format 2."""
    f = np.array([3, 1, 4, 1, 5], np.int64)
    supp = np.array([0, 1, 2, 6, 7])
    rows = []
    for shift in (0, 3, 9, 11):
        rows.append((supp + shift, f))
    rows.append((np.array([1, 5]), np.array([2, 7])))
    m, n, p = len(rows), 20, 65521
    d = np.zeros((m, n), np.int64)
    for i, (cc, vv) in enumerate(rows):
        d[i, cc] = vv
    rp, c, v = synth.dense_to_csr(d)
    buf = synth.encode_format2(m, n, p, rp, c, v)
    k_at = 4 + 8 + 16 + 8 * m                          # after b, m, n, p, nnz, rows, polmap
    k = struct.unpack_from("<Q", buf, k_at)[0]
    pnb, pnnz = struct.unpack_from("<IQ", buf, k_at + 8 + 8 * k)
    assert pnb == 2 and pnnz == len(f) + 2 < len(v)   # coefficients stored once per polynomial
    same(F.decode_format2(buf), (m, n, p, rp, c, v))


def corrupt(buf, offset, fmt, value):
    b = bytearray(buf)
    struct.pack_into(fmt, b, offset, value)
    return bytes(b)


# offsets in the hand-worked file
OFF_ROWS = 4 + 8 + 16
OFF_POLMAP = OFF_ROWS + 12
OFF_COLID = OFF_POLMAP + 12 + 8
OFF_PDATA = OFF_COLID + 56 + 4 + 8 + 8


@pytest.mark.parametrize("name,make", [
    ("truncated", lambda g: g[:-1]),
    ("trailing byte", lambda g: g + b"\0"),
    ("run crossing the row's end", lambda g: corrupt(g, OFF_COLID + 8, "<Q", 5)),
    ("run length 1", lambda g: corrupt(g, OFF_COLID + 8, "<Q", 1)),
    ("lone column past n", lambda g: corrupt(g, OFF_COLID + 16, "<Q", 10 | M31)),
    ("columns not increasing", lambda g: corrupt(g, OFF_COLID + 16, "<Q", 2 | M31)),
    ("entry above 32 bits", lambda g: corrupt(g, OFF_COLID + 24, "<Q", (1 << 40) | 4 | M31)),
    ("polynomial out of range", lambda g: corrupt(g, OFF_POLMAP + 4, "<I", 2)),
    ("polynomial of another length", lambda g: corrupt(g, OFF_POLMAP + 4, "<I", 0)),
    ("zero coefficient", lambda g: corrupt(g, OFF_PDATA + 2, "<B", 0)),
    ("coefficient divisible by p", lambda g: corrupt(g, OFF_PDATA + 5, "<B", 251)),
    ("p too large", lambda g: corrupt(g, 12, "<Q", 1 << 17)),
])
def test_malformed_format2_rejected(name, make):
    good = hand_format2(1, 251, "B", [5, 6, 7, 9, 3, 250])
    F.decode_format2(good)
    with pytest.raises(F.FormatError):
        F.decode_format2(make(good))


MUTATIONS = [
    ("if x & MASK31:", "if x & 0:"),                                   # lone-column mask never seen
    ("j = int(polmap[i])", "j = i"),                                   # coefficients by row, not polmap
    ("return _TYPES[(u, v)]", "return _TYPES[(1 - u, v)]"),            # type bit read the other way round
    ("out.extend(range(x, x + s))", "out.extend(range(x, x + s - 1))"),  # runs one column short
]


@pytest.mark.parametrize("old,new", MUTATIONS)
def test_planted_mistakes_in_the_reader_fail_the_pins(old, new):
    """Each plausible mistake, planted in a copy of the reader, fails the
    hand-worked files."""
    import types
    src = open(F.__file__).read()
    assert src.count(old) == 1
    mod = types.ModuleType("formats_mutant")
    exec(compile(src.replace(old, new), "formats_mutant", "exec"), mod.__dict__)
    failed = 0
    for b, p, fmt, data, want in [(1, 251, "B", [5, 6, 7, 9, 3, 250], [5, 6, 7, 9, 3, 250, 5, 6, 7, 9]),
                                  (2, 7, "h", [1, -1, 2, 3, -3, 5], [1, 6, 2, 3, 4, 5, 1, 6, 2, 3])]:
        try:
            _, _, _, rp, c, v = mod.decode_format2(hand_format2(b, p, fmt, data))
            ok = (rp.tolist() == [0, 4, 6, 10] and c.tolist() == [1, 2, 3, 7, 4, 9, 2, 3, 4, 5]
                  and v.tolist() == want)
        except mod.FormatError:
            ok = False
        failed += not ok
    assert failed > 0
