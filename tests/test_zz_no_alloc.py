"""The allocation-free pivot analysis, called through the C ABI, gives the
same result as gbla_pivots on two calls in a row.

It exists for callers that must not allocate device memory during a call
(an application whose device memory is all reserved by its own pool, or a
latency-sensitive loop where an allocation could synchronise the device).
This file is collected last so that, in a run that stops at the first
failure, every other test has already run.
"""
import numpy as np
import pytest

from paper_1602_06097_gb300 import gbla, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def _dev(spec):
    rp, c, v = synth.fl_matrix(spec)
    return (torch.from_numpy(rp).cuda(), torch.from_numpy(c).cuda(),
            torch.from_numpy(v.view(np.int16)).cuda())


def test_noalloc_pivots_equal_allocating_entry_point_twice():
    specs = [synth.FLSpec(m=900, n=1300, npiv=500, density=0.03, seed=4101),
             synth.FLSpec(m=2000, n=3000, npiv=1200, density=0.04, seed=4102, p=32003)]
    for spec in specs:
        rp, c, v = _dev(spec)
        ref, ref_npiv = gbla.pivots(rp, c, v, (spec.m, spec.n), spec.p)
        for _ in range(2):
            out = torch.full((spec.n,), -7, dtype=torch.int64, device="cuda")
            npiv = gbla.pivots_noalloc(rp, c, v, (spec.m, spec.n), spec.p, out)
            assert npiv == ref_npiv
            assert torch.equal(out, ref)


def test_noalloc_pivots_rejects_too_many_columns():
    z64 = torch.zeros(2, dtype=torch.int64, device="cuda")
    z32 = torch.zeros(1, dtype=torch.int32, device="cuda")
    z16 = torch.ones(1, dtype=torch.int16, device="cuda")
    out = torch.empty(1, dtype=torch.int64, device="cuda")
    with pytest.raises(gbla.GblaError) as e:
        gbla.pivots_noalloc(z64[:1], z32[:0], z16[:0], (0, (1 << 20) + 1), 65521, out)
    assert e.value.code == 1
