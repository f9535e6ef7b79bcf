"""The sparse forward pass of the echelon step (GBLA_ECHELON_SGE: the
paper's structured Gaussian elimination with sparse pivot rows, Alg. 3 and its
parallel form of Sec. 5.1) against the oracle, bit for bit, in both output
forms, on Schur complements that stay sparse (the pass completes) and on dense
ones (its pivot pool may fill up and the panels finish the pass)."""
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


SPARSE_D = [   # few pivots, short rows: the Schur complement stays sparse
    synth.FLSpec(m=3000, n=9000, npiv=1500, density=0.002, run_len=(1, 4), seed=1501),
    synth.FLSpec(m=6000, n=20000, npiv=2000, density=0.0008, run_len=(1, 3), seed=1502, p=32003),
    synth.FLSpec(m=5000, n=12000, npiv=1000, density=0.001, run_len=(1, 2), seed=1503, p=7),
]
DENSE_D = [
    synth.FLSpec(m=600, n=900, npiv=360, density=0.04, run_len=(4, 24), seed=1511),
    synth.FLSpec(m=2600, n=3700, npiv=1900, density=0.02, run_len=(16, 64), group=(2, 8), seed=1512),
]


@pytest.mark.parametrize("spec", SPARSE_D + DENSE_D, ids=[f"{s.m}x{s.n}p{s.p}" for s in SPARSE_D + DENSE_D])
@pytest.mark.parametrize("reduced", [False, True])
def test_sge_equals_oracle(spec, reduced):
    rp, c, v = synth.fl_matrix(spec)
    res = gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, want_reduced=reduced, echelon=gbla.ECHELON_SGE,
                      stats=True)
    same(res, (oracle.rref if reduced else oracle.echelon)(spec.m, spec.n, spec.p, rp, c, v))
    st = res[4]
    assert st["echelon_method"] in (gbla.ECHELON_SGE, gbla.ECHELON_PANELS)
    assert 0.0 <= st["d_density"] <= 1.0 or st["m_cd"] == 0


@pytest.mark.parametrize("spec", SPARSE_D[:2], ids=["a", "b"])
def test_sge_completes_on_a_sparse_schur_complement(spec):
    rp, c, v = synth.fl_matrix(spec)
    res = gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, echelon=gbla.ECHELON_SGE, stats=True)
    assert res[4]["echelon_method"] == gbla.ECHELON_SGE
    same(res, gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, echelon=gbla.ECHELON_PANELS))


def test_sge_with_dependent_rows():
    """Duplicated and combined non-pivot rows: their reductions end in zero."""
    rng = np.random.default_rng(1520)
    spec = SPARSE_D[0]
    rp, c, v = synth.fl_matrix(spec)
    dense = np.zeros((spec.m, spec.n), np.int64)
    for i in range(spec.m):
        dense[i, c[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
    extra = np.concatenate([dense[rng.choice(spec.m, 200)], (dense[:100] * 3 + dense[100:200] * 5) % spec.p])
    M = np.concatenate([dense, extra[np.any(extra != 0, axis=1)]])
    rp2, c2, v2 = synth.dense_to_csr(M)
    res = gbla.reduce(rp2, c2, v2, M.shape, spec.p, echelon=gbla.ECHELON_SGE, want_reduced=True)
    same(res, oracle.rref(M.shape[0], M.shape[1], spec.p, rp2, c2, v2))


def test_sge_option_is_validated():
    spec = DENSE_D[0]
    rp, c, v = synth.fl_matrix(spec)
    with pytest.raises(gbla.GblaError) as e:
        gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, echelon=3)
    assert e.value.code == 1
