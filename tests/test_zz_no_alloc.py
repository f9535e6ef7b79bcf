"""The allocation-free pivot analysis, called through the C ABI.

It exists for callers that must not allocate device memory during a call
(an application whose device memory is all reserved by its own pool, or a
latency-sensitive loop where an allocation could synchronise the device).
Its result must equal the allocating entry point's and the oracle's pivot
choice, on two calls in a row; malformed inputs must be rejected without
writing the caller's array.  This file is collected last so that, in a run
that stops at the first failure, every other test has already run.
"""
import numpy as np
import pytest

import oracle
from paper_1602_06097_gb300 import gbla, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def _dev(rp, c, v):
    return (torch.from_numpy(np.asarray(rp, np.int64)).cuda(),
            torch.from_numpy(np.asarray(c, np.int32)).cuda(),
            torch.from_numpy(np.asarray(v, np.uint16).view(np.int16)).cuda())


SPECS = [synth.FLSpec(m=900, n=1300, npiv=500, density=0.03, seed=4101),
         synth.FLSpec(m=2000, n=3000, npiv=1200, density=0.04, seed=4102, p=32003)]


@pytest.mark.parametrize("spec", SPECS, ids=["900x1300", "2000x3000"])
def test_noalloc_pivots_equal_allocating_entry_point_and_oracle_twice(spec):
    rp, c, v = synth.fl_matrix(spec)
    expect = oracle.pivots(spec.m, spec.n, rp, c)
    d = _dev(rp, c, v)
    ref, ref_npiv = gbla.pivots(*d, (spec.m, spec.n), spec.p)
    assert ref_npiv == int((expect >= 0).sum())
    for _ in range(2):
        out = torch.full((spec.n,), -7, dtype=torch.int64, device="cuda")
        npiv = gbla.pivots_noalloc(*d, (spec.m, spec.n), spec.p, out)
        assert npiv == ref_npiv
        assert torch.equal(out, ref)
        assert (out.cpu().numpy() == expect).all()


def test_noalloc_pivots_on_a_side_stream_and_degenerate_shapes():
    spec = SPECS[0]
    rp, c, v = synth.fl_matrix(spec)
    d = _dev(rp, c, v)
    s = torch.cuda.Stream()
    out = torch.full((spec.n,), -7, dtype=torch.int64, device="cuda")
    with torch.cuda.stream(s):
        npiv = gbla.pivots_noalloc(*d, (spec.m, spec.n), spec.p, out, stream=s)
    assert (out.cpu().numpy() == oracle.pivots(spec.m, spec.n, rp, c)).all()
    assert npiv == int((out >= 0).sum())
    # empty rows between nonempty ones, a matrix without rows, one without columns
    dense = np.array([[0, 0, 0, 0], [0, 3, 0, 1], [0, 0, 0, 0], [0, 2, 5, 0], [4, 0, 0, 0]])
    rp2, c2, v2 = synth.dense_to_csr(dense)
    out2 = torch.full((4,), -7, dtype=torch.int64, device="cuda")
    assert gbla.pivots_noalloc(*_dev(rp2, c2, v2), (5, 4), 7, out2) == 2
    assert list(out2.cpu().numpy()) == list(oracle.pivots(5, 4, rp2, c2))
    out3 = torch.full((6,), -7, dtype=torch.int64, device="cuda")
    assert gbla.pivots_noalloc(*_dev(np.zeros(1, np.int64), [], []), (0, 6), 7, out3) == 0
    assert (out3.cpu().numpy() == -1).all()
    out4 = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    assert gbla.pivots_noalloc(*_dev(np.zeros(3, np.int64), [], []), (2, 0), 7, out4) == 0
    assert int(out4[0]) == -7


# (row_ptr, col, val, shape, p) of malformed matrices, one per rule
MALFORMED = {
    "unsorted row": ([0, 3], [2, 1, 3], [1, 1, 1], (1, 4), 7),
    "duplicate column": ([0, 2], [1, 1], [1, 2], (1, 4), 7),
    "explicit zero": ([0, 2], [0, 2], [1, 0], (1, 4), 7),
    "value >= p": ([0, 2], [0, 2], [1, 7], (1, 4), 7),
    "column out of range": ([0, 1, 2], [0, 4], [1, 1], (2, 4), 7),
    "row_ptr decreasing": ([0, 2, 1, 3], [0, 1, 2], [1, 1, 1], (3, 4), 7),
    "row_ptr end != nnz": ([0, 1, 2], [0, 1, 2], [1, 1, 1], (2, 4), 7),
}


@pytest.mark.parametrize("case", sorted(MALFORMED))
def test_noalloc_pivots_rejects_malformed_csr_without_writing(case):
    rp, c, v, shape, p = MALFORMED[case]
    out = torch.full((shape[1],), -7, dtype=torch.int64, device="cuda")
    with pytest.raises(gbla.GblaError) as e:
        gbla.pivots_noalloc(*_dev(rp, c, v), shape, p, out)
    assert e.value.code == 1
    assert (out.cpu().numpy() == -7).all()
    # the scratch array still serves a valid call afterwards
    spec = SPECS[0]
    rp2, c2, v2 = synth.fl_matrix(spec)
    out2 = torch.empty(spec.n, dtype=torch.int64, device="cuda")
    gbla.pivots_noalloc(*_dev(rp2, c2, v2), (spec.m, spec.n), spec.p, out2)
    assert (out2.cpu().numpy() == oracle.pivots(spec.m, spec.n, rp2, c2)).all()


def test_noalloc_pivots_rejects_too_many_columns():
    n = (1 << 20) + 1
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    with pytest.raises(gbla.GblaError) as e:
        gbla.pivots_noalloc(*_dev(np.zeros(1, np.int64), [], []), (0, n), 65521, out)
    assert e.value.code == 1
