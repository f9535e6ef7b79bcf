"""The original order of the FL steps (Sec. 4.1 steps 2-3: B <- A^-1 B
first, then D <- D - C B) against the oracle, in both output forms, and
against the new order (Sec. 4.3), bit for bit."""
import numpy as np
import pytest

import oracle
from paper_1602_06097_gb300 import gbla, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def same(a, b):
    assert a[0] == b[0], f"rank {a[0]} != {b[0]}"
    for x, y, what in zip(a[1:4], b[1:4], ("row_ptr", "col", "val")):
        assert np.array_equal(np.asarray(x, np.int64), np.asarray(y, np.int64)), f"{what} differs"


SPECS = [
    synth.FLSpec(m=600, n=900, npiv=360, density=0.04, run_len=(4, 24), seed=1101),
    synth.FLSpec(m=1500, n=2100, npiv=1000, density=0.03, run_len=(8, 40), seed=1102, p=32003),
    synth.FLSpec(m=2600, n=3700, npiv=1900, density=0.02, run_len=(16, 64), group=(2, 8), seed=1103),
    synth.FLSpec(m=400, n=500, npiv=300, density=0.05, run_len=(2, 8), seed=1104, p=7),
    synth.FLSpec(m=300, n=300, npiv=300, density=0.05, run_len=(2, 8), seed=1105),   # no B block
]


@pytest.mark.parametrize("spec", SPECS, ids=[f"{s.m}x{s.n}p{s.p}" for s in SPECS])
@pytest.mark.parametrize("reduced", [True, False])
def test_trsm_first_equals_oracle(spec, reduced):
    rp, c, v = synth.fl_matrix(spec)
    res = gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, want_reduced=reduced, order=gbla.ORDER_TRSM_FIRST,
                      stats=True)
    assert res[4]["path"] == gbla.PATH_DENSE
    ref = (oracle.rref if reduced else oracle.echelon)(spec.m, spec.n, spec.p, rp, c, v)
    same(res, ref)


def test_trsm_first_equals_new_order_on_a_scaled_bench_workload():
    spec = synth.scaled("fl_40000x60000", 0.2)
    rp, c, v = synth.fl_matrix(spec)
    a = gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, want_reduced=True, order=gbla.ORDER_TRSM_FIRST)
    b = gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, want_reduced=True)
    same(a, b)


def test_trsm_first_refusals():
    spec = SPECS[0]
    rp, c, v = synth.fl_matrix(spec)
    with pytest.raises(gbla.GblaError) as e:
        gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, order=gbla.ORDER_TRSM_FIRST, path=gbla.PATH_SPARSE)
    assert e.value.code == 6
    with pytest.raises(gbla.GblaError) as e:
        gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, order=2)
    assert e.value.code == 1
