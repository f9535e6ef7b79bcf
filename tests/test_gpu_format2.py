"""The device decoder of Format 2 files (Sec. 3.2) against the oracle reader,
and the decoded matrix through the reduction.

The decoder's parallel algorithm is also checked on the CPU
(test_format2_parallel_model.py).
"""
import numpy as np
import pytest

import oracle
from oracle import formats as F
from paper_1602_06097_gb300 import gbla, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def decoded(buf):
    d = gbla.decode_format2(buf)
    try:
        m, rp, c, v = d.to_host()
        return (m, d.n, d.p, rp, c, v)
    finally:
        d.free()


def same(a, b):
    assert a[:3] == b[:3]
    for x, y in zip(a[3:], b[3:]):
        assert np.array_equal(np.asarray(x, np.int64), np.asarray(y, np.int64))


@pytest.mark.parametrize("vtype,p", [(None, 65521), ("u1", 251), ("i1", 251), ("i2", 65521), ("u4", 65521),
                                     ("i4", 32003), ("u8", 65521), ("i8", 65521)])
def test_decoder_equals_oracle_reader(vtype, p):
    spec = synth.workload("fl_2000x3000", p=p)
    rp, c, v = synth.fl_matrix(spec)
    buf = synth.encode_format2(spec.m, spec.n, spec.p, rp, c, v, vtype)
    same(decoded(buf), F.decode_format2(buf))


def test_decoder_on_random_and_edge_files():
    rng = np.random.default_rng(3)
    for _ in range(20):
        m, n = int(rng.integers(1, 300)), int(rng.integers(1, 500))
        p = int(rng.choice([13, 251, 32003, 65521]))
        rp, c, v = synth.random_csr(rng, m, n, p, float(rng.uniform(0.0, 0.5)))
        buf = synth.encode_format2(m, n, p, rp, c, v)
        same(decoded(buf), F.decode_format2(buf))


def test_decoder_rejects_malformed_files():
    from test_formats import hand_format2, corrupt, OFF_COLID, OFF_POLMAP, OFF_PDATA
    good = hand_format2(1, 251, "B", [5, 6, 7, 9, 3, 250])
    same(decoded(good), F.decode_format2(good))
    for buf in [good[:-1], good + b"\0", corrupt(good, OFF_COLID + 8, "<Q", 5),
                corrupt(good, OFF_COLID + 16, "<Q", 10 | (1 << 31)), corrupt(good, OFF_POLMAP + 4, "<I", 0),
                corrupt(good, OFF_PDATA + 2, "<B", 0), corrupt(good, OFF_COLID + 48, "<Q", 4 | (1 << 31))]:
        with pytest.raises(gbla.GblaError):
            gbla.decode_format2(buf)


@pytest.mark.parametrize("vtype", [None, "i8"])
def test_decoded_matrix_reduces_like_the_file(vtype):
    spec = synth.workload("fl_2000x3000")
    rp, c, v = synth.fl_matrix(spec)
    d = gbla.decode_format2(synth.encode_format2(spec.m, spec.n, spec.p, rp, c, v, vtype))
    try:
        trp, tc, tv = d.tensors()
        res = gbla.reduce_device(trp, tc, tv, (d.m, d.n), d.p, want_reduced=True)
        try:
            got = res.to_host()
        finally:
            res.free()
    finally:
        d.free()
    want = oracle.rref(spec.m, spec.n, spec.p, rp, c, v)
    same((0, 0, 0) + tuple(got), (0, 0, 0) + tuple(want[:4]))


def test_timed_decode_from_a_page_locked_buffer():
    """The timed entry point from a numpy (page-locked) buffer decodes the
    same matrix and reports a positive device time."""
    spec = synth.scaled("fl_40000x60000", 0.3)
    rp, c, v = synth.fl_matrix(spec)
    buf = synth.encode_format2(spec.m, spec.n, spec.p, rp, c, v)
    pinned = torch.frombuffer(bytearray(buf), dtype=torch.uint8).pin_memory().numpy()
    d = gbla.decode_format2(pinned, timed=True)
    try:
        assert d.decode_ms is not None and d.decode_ms > 0
        m, drp, dc, dv = d.to_host()
    finally:
        d.free()
    same((m, 0, 0, drp, dc, dv), (spec.m, 0, 0, rp, c, v))
