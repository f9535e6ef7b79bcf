"""GPU parity of the sparse path: the K-compacted tensor-core product on its
own (gbla_spmm, against exact int64 numpy) and whole reductions on the sparse
path against the oracle and against the dense path, bit for bit.

The sparse path keeps the pivot rows sparse (Table 4: A and B are sparse):
C*A^-1 and the Schur update run as tensor-core products whose K is, per
128-column tile, the list of rows that meet the tile.
"""
import numpy as np
import pytest

import oracle
from paper_1602_06097_gb300 import gbla, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def t16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint16).view(np.int16)).cuda()


def from_t16(t):
    return t.cpu().numpy().view(np.uint16).astype(np.int64)


def same(a, b):
    assert a[0] == b[0], f"rank {a[0]} != {b[0]}"
    for x, y, what in zip(a[1:4], b[1:4], ("row_ptr", "col", "val")):
        assert np.array_equal(np.asarray(x, np.int64), np.asarray(y, np.int64)), f"{what} differs"


def run_spmm(X, S, C, p, sign, lead=None):
    rp, c, v = synth.dense_to_csr(S)
    tc = t16(C)
    gbla.spmm(t16(X), torch.from_numpy(rp).cuda(), torch.from_numpy(c).cuda(), t16(v), S.shape[1], tc, p,
              sign=sign, x_lead=None if lead is None else torch.from_numpy(np.asarray(lead, np.int32)).cuda())
    return from_t16(tc)


def ref(X, S, C, p, sign):
    return (C + sign * (X.astype(np.int64) @ S.astype(np.int64))) % p


def runs_matrix(rng, K, N, p, density, run=(4, 40)):
    """Sparse K x N matrix with horizontal runs (the F4 pattern of Sec. 4.2)."""
    S = np.zeros((K, N), np.int64)
    for i in range(K):
        left = int(density * N)
        while left > 0:
            L = int(rng.integers(run[0], run[1] + 1))
            c0 = int(rng.integers(0, N))
            S[i, c0:c0 + L] = rng.integers(1, p, size=len(range(c0, min(N, c0 + L))))
            left -= L
    return S


def staircase(rng, M, K, p, density=1.0):
    lead = np.sort(rng.integers(0, K, size=M))
    X = np.where(rng.random((M, K)) < density, rng.integers(0, p, size=(M, K)), 0)
    X[np.arange(K)[None, :] < lead[:, None]] = 0
    return X, lead.astype(np.int32)


@pytest.mark.parametrize("shape", [(1, 1, 1), (130, 70, 200), (257, 385, 1000), (300, 129, 1536), (640, 520, 2300)])
@pytest.mark.parametrize("p", [65521, 32003, 8191, 11])
@pytest.mark.parametrize("sign", [-1, 1])
def test_spmm_random_runs(shape, p, sign):
    M, N, K = shape
    rng = np.random.default_rng(M + 3 * N + 7 * K + p + sign)
    X = rng.integers(0, p, size=(M, K))
    S = runs_matrix(rng, K, N, p, 0.03)
    C = rng.integers(0, p, size=(M, N))
    assert np.array_equal(run_spmm(X, S, C, p, sign), ref(X, S, C, p, sign))


@pytest.mark.parametrize("seed", range(3))
def test_spmm_staircase_leads(seed):
    """X zero left of ascending row leads: tiles skip the list entries left of
    their raster group's first lead."""
    rng = np.random.default_rng(40 + seed)
    p = 65521
    M, N, K = 900, 700, 3000
    X, lead = staircase(rng, M, K, p)
    S = runs_matrix(rng, K, N, p, 0.02)
    C = rng.integers(0, p, size=(M, N))
    assert np.array_equal(run_spmm(X, S, C, p, -1, lead), ref(X, S, C, p, -1))


@pytest.mark.parametrize("K", [511, 512, 513, 1023, 1024, 1025, 2048 + 64, 3072 + 5])
@pytest.mark.parametrize("fill", ["pm1", "half", "halfp1", "mixed"])
def test_spmm_at_the_k_block_bound(K, fill):
    """A dense S makes every tile's list K long: all-extreme digits at and
    around the 1,024-deep exact fp32 block of the gathered product (each of
    its four digit-product sums reaches 2^24 with the "half" fill)."""
    p = 65521
    M, N = 256, 200
    h = (p - 1) // 2
    vals = {"pm1": p - 1, "half": h, "halfp1": h + 1}
    if fill == "mixed":
        rng = np.random.default_rng(K)
        choices = np.array([p - 1, h, h + 1, 1, 32640, p - 32640, 128, p - 128])
        X = rng.choice(np.append(choices, 0), size=(M, K))
        S = rng.choice(choices, size=(K, N))
    else:
        X = np.full((M, K), vals[fill])
        S = np.full((K, N), vals[fill])
    C = np.zeros((M, N), np.int64)
    assert np.array_equal(run_spmm(X, S, C, p, 1), ref(X, S, C, p, 1))


def test_spmm_empty_tiles_rows_and_columns():
    rng = np.random.default_rng(3)
    p = 32003
    M, N, K = 300, 600, 900
    X = rng.integers(0, p, size=(M, K))
    S = runs_matrix(rng, K, N, p, 0.02)
    S[:, 128:384] = 0          # two column tiles without any row
    S[200:500] = 0             # empty rows of S
    S[:, -1] = 0
    C = rng.integers(0, p, size=(M, N))
    assert np.array_equal(run_spmm(X, S, C, p, -1), ref(X, S, C, p, -1))
    # no nonzero at all: C unchanged
    Z = np.zeros((K, N), np.int64)
    assert np.array_equal(run_spmm(X, Z, C, p, -1), C)


@pytest.mark.parametrize("case", ["unsorted", "explicit zero", "value >= p", "column out of range"])
def test_spmm_rejects_malformed_sparse_operand(case):
    p = 11
    rp = np.array([0, 2, 3], np.int64)
    col = {"unsorted": [2, 1, 0], "explicit zero": [0, 1, 2], "value >= p": [0, 1, 2],
           "column out of range": [0, 1, 9]}[case]
    val = {"explicit zero": [1, 0, 1], "value >= p": [1, 11, 1]}.get(case, [1, 2, 3])
    X = torch.zeros((4, 2), dtype=torch.int16, device="cuda")
    C = torch.full((4, 5), 3, dtype=torch.int16, device="cuda")
    with pytest.raises(gbla.GblaError) as e:
        gbla.spmm(X, torch.from_numpy(rp).cuda(), torch.tensor(col, dtype=torch.int32, device="cuda"),
                  t16(np.array(val)), 5, C, p)
    assert e.value.code == 1
    assert bool((C == 3).all())


# ------------------------------------------------------- whole reductions
FL_SPECS = [
    synth.FLSpec(m=600, n=900, npiv=360, density=0.04, run_len=(4, 24), seed=701),
    synth.FLSpec(m=1500, n=2100, npiv=1000, density=0.03, run_len=(8, 40), seed=702, p=32003),
    synth.FLSpec(m=2600, n=3700, npiv=1900, density=0.02, run_len=(16, 64), group=(2, 8), seed=703),
    synth.FLSpec(m=3000, n=3300, npiv=2700, density=0.01, run_len=(4, 32), seed=704, p=8191),
]


@pytest.mark.parametrize("spec", FL_SPECS, ids=[f"{s.m}x{s.n}" for s in FL_SPECS])
@pytest.mark.parametrize("leaf", [0, 128, 1024])
def test_sparse_path_equals_oracle(spec, leaf):
    rp, c, v = synth.fl_matrix(spec)
    res = gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, path=gbla.PATH_SPARSE, leaf=leaf, stats=True)
    assert res[4]["path"] == gbla.PATH_SPARSE
    same(res, oracle.echelon(spec.m, spec.n, spec.p, rp, c, v))


@pytest.mark.parametrize("spec", FL_SPECS[:2], ids=[f"{s.m}x{s.n}" for s in FL_SPECS[:2]])
def test_sparse_path_reduced_form_equals_oracle(spec):
    rp, c, v = synth.fl_matrix(spec)
    res = gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, want_reduced=True, path=gbla.PATH_SPARSE)
    same(res, oracle.rref(spec.m, spec.n, spec.p, rp, c, v))


def test_sparse_and_dense_paths_agree_on_a_scaled_bench_workload():
    spec = synth.scaled("fl_40000x60000", 0.15)
    rp, c, v = synth.fl_matrix(spec)
    a = gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, path=gbla.PATH_SPARSE, stats=True)
    b = gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, path=gbla.PATH_DENSE, stats=True)
    assert a[4]["path"] == gbla.PATH_SPARSE and b[4]["path"] == gbla.PATH_DENSE
    same(a, b)
    same(a, oracle.echelon(spec.m, spec.n, spec.p, rp, c, v))


def test_sparse_path_is_refused_where_it_cannot_run():
    small = synth.FLSpec(m=60, n=90, npiv=30, density=0.1, run_len=(2, 6), seed=5, p=7)
    rp, c, v = synth.fl_matrix(small)
    with pytest.raises(gbla.GblaError) as e:
        gbla.reduce(rp, c, v, (small.m, small.n), small.p, path=gbla.PATH_SPARSE)
    assert e.value.code == 6
    # the automatic choice takes the dense path there
    res = gbla.reduce(rp, c, v, (small.m, small.n), small.p, stats=True)
    assert res[4]["path"] == gbla.PATH_DENSE
    same(res, oracle.echelon(small.m, small.n, small.p, rp, c, v))
    spec = FL_SPECS[0]
    rp, c, v = synth.fl_matrix(spec)
    with pytest.raises(gbla.GblaError) as e:
        gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, path=gbla.PATH_SPARSE, variant=gbla.GEMM_SIMT)
    assert e.value.code == 6
