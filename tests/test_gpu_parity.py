"""GPU parity: the CUDA path, called through the C ABI, against the CPU oracle.

Every comparison is bit-exact (integer arithmetic mod p): ranks, row
pointers, column indices and values must be identical.
"""
import numpy as np
import pytest

import oracle
from paper_1602_06097_gb300 import gbla, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def same(a, b):
    ra, pa, ca, va = a[:4]
    rb, pb, cb, vb = b[:4]
    assert ra == rb, f"rank {ra} != {rb}"
    assert np.array_equal(np.asarray(pa), np.asarray(pb)), "row_ptr differs"
    assert np.array_equal(np.asarray(ca, np.int64), np.asarray(cb, np.int64)), "col differs"
    assert np.array_equal(np.asarray(va, np.int64), np.asarray(vb, np.int64)), "val differs"


def t16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint16).view(np.int16)).cuda()


def from_t16(t):
    return t.cpu().numpy().view(np.uint16).astype(np.int64)


# ------------------------------------------------------------ modular GEMM
def ref_gemm(A, B, C, p, sign):
    # exact: entries < 2^16, K <= 2^15 terms of < 2^32 each fit int64
    return (C + sign * (A.astype(np.int64) @ B.astype(np.int64))) % p


@pytest.mark.parametrize("variant", [gbla.GEMM_SIMT, gbla.GEMM_TCGEN05])
@pytest.mark.parametrize("shape", [(1, 1, 1), (130, 70, 200), (257, 385, 1000), (128, 256, 640), (300, 129, 1536)])
@pytest.mark.parametrize("p", [65521, 32003, 8191, 11])
@pytest.mark.parametrize("sign", [-1, 1])
def test_modmatmul_random(variant, shape, p, sign):
    M, N, K = shape
    rng = np.random.default_rng(M * 7 + N * 13 + K + p + sign)
    A = rng.integers(0, p, size=(M, K))
    B = rng.integers(0, p, size=(K, N))
    C = rng.integers(0, p, size=(M, N))
    tc = t16(C)
    gbla.modmatmul(t16(A), t16(B), tc, p, sign=sign, variant=variant)
    assert np.array_equal(from_t16(tc), ref_gemm(A, B, C, p, sign))


@pytest.mark.parametrize("variant", [gbla.GEMM_SIMT, gbla.GEMM_TCGEN05])
@pytest.mark.parametrize("K", [511, 512, 513, 1024, 2048 + 64])
@pytest.mark.parametrize("fill", ["pm1", "half", "halfp1", "digit_extreme", "mixed"])
@pytest.mark.parametrize("M", [128, 384])
def test_modmatmul_at_the_k_block_bound(variant, K, fill, M):
    """All-extreme operands at and around the 512-deep exact fp32 block: every
    digit product has the largest magnitude the split allows.  M = 384 gives
    three row tiles, a ragged raster group (the CTA-pair form of the same
    product runs in tests/test_gpu_env_variants.py)."""
    p = 65521
    N = 128
    h = (p - 1) // 2
    vals = {"pm1": p - 1, "half": h, "halfp1": h + 1, "digit_extreme": (128 * 256 - 128) % p}
    if fill == "mixed":
        rng = np.random.default_rng(K)
        choices = np.array([p - 1, h, h + 1, 1, 0, 32640, p - 32640, 128, p - 128])
        A = rng.choice(choices, size=(M, K))
        B = rng.choice(choices, size=(K, N))
    else:
        A = np.full((M, K), vals[fill])
        B = np.full((K, N), vals[fill])
    C = np.zeros((M, N), np.int64)
    tc = t16(C)
    gbla.modmatmul(t16(A), t16(B), tc, p, sign=1, variant=variant)
    assert np.array_equal(from_t16(tc), ref_gemm(A, B, C, p, 1))


def test_modmatmul_tc_matches_simt_large():
    p = 65521
    rng = np.random.default_rng(5)
    M, N, K = 700, 900, 3000
    A = rng.integers(0, p, size=(M, K))
    B = rng.integers(0, p, size=(K, N))
    C = rng.integers(0, p, size=(M, N))
    c1, c2 = t16(C), t16(C)
    gbla.modmatmul(t16(A), t16(B), c1, p, -1, gbla.GEMM_TCGEN05)
    gbla.modmatmul(t16(A), t16(B), c2, p, -1, gbla.GEMM_SIMT)
    assert torch.equal(c1, c2)
    assert np.array_equal(from_t16(c1), ref_gemm(A, B, C, p, -1))


# ------------------------------------------------------------ FL step 1
@pytest.mark.parametrize("seed", range(4))
def test_pivots_match_oracle(seed):
    spec = synth.FLSpec(m=900, n=1300, npiv=500, density=0.03, seed=100 + seed)
    rp, c, v = synth.fl_matrix(spec)
    piv, npiv = gbla.pivots(torch.from_numpy(rp).cuda(), torch.from_numpy(c).cuda(), t16(v), (spec.m, spec.n), spec.p)
    ref = oracle.pivots(spec.m, spec.n, rp, c)
    assert npiv == int((ref >= 0).sum())
    assert np.array_equal(piv.cpu().numpy(), ref)


def test_multiline_example1():
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "multiline_example1.json")))
    dense = np.array([g["r1"], g["r2"]])
    rp, c, v = synth.dense_to_csr(dense)
    ptr, pos, val = gbla.multiline(rp, c, v, 2)
    assert list(ptr) == [0, len(g["ml_pos"])]
    assert list(pos) == g["ml_pos"]
    assert list(val) == g["ml_val"]


def test_multiline_random_pairs_match_oracle():
    rng = np.random.default_rng(9)
    dense = np.where(rng.random((9, 40)) < 0.3, rng.integers(1, 65521, size=(9, 40)), 0)
    rp, c, v = synth.dense_to_csr(dense)
    ptr, pos, val = gbla.multiline(rp, c, v, 9)
    for q in range(5):
        r1 = dense[2 * q]
        r2 = dense[2 * q + 1] if 2 * q + 1 < 9 else np.zeros(40, np.int64)
        p1, p2 = np.nonzero(r1)[0], np.nonzero(r2)[0]
        opos, oval = oracle.multiline(p1, r1[p1], p2, r2[p2])
        assert list(pos[ptr[q]:ptr[q + 1]]) == list(opos)
        assert list(val[2 * ptr[q]:2 * ptr[q + 1]]) == list(oval)


# ------------------------------------------------------ whole reduction
SMALL = [
    synth.FLSpec(m=300, n=450, npiv=180, density=0.05, run_len=(3, 12), seed=11),
    synth.FLSpec(m=700, n=1000, npiv=420, density=0.03, run_len=(4, 32), seed=12),
    synth.FLSpec(m=1100, n=1500, npiv=300, density=0.02, run_len=(4, 32), seed=13, p=32003),
    synth.FLSpec(m=520, n=700, npiv=500, density=0.04, run_len=(2, 8), seed=14),       # few C rows
    synth.FLSpec(m=900, n=600, npiv=200, density=0.08, run_len=(4, 16), seed=15),      # more rows than columns
    synth.FLSpec(m=640, n=900, npiv=400, density=0.02, seed=16, group=(2, 16), share=0.8, run_len=(20, 60)),
    # small primes through the tensor-core path (p >= 8), ragged widths
    synth.FLSpec(m=700, n=1003, npiv=300, density=0.03, run_len=(4, 16), seed=17, p=11),
    synth.FLSpec(m=800, n=1201, npiv=350, density=0.03, run_len=(4, 16), seed=18, p=257),
]


@pytest.mark.parametrize("idx", range(len(SMALL)))
@pytest.mark.parametrize("want_reduced", [False, True])
def test_reduce_matches_oracle(idx, want_reduced):
    spec = SMALL[idx]
    rp, c, v = synth.fl_matrix(spec)
    res = gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, want_reduced=want_reduced)
    ref = oracle.rref(spec.m, spec.n, spec.p, rp, c, v) if want_reduced else \
        oracle.echelon(spec.m, spec.n, spec.p, rp, c, v)[:4]
    same(res, ref)


@pytest.mark.parametrize("p", [11, 257, 32003, 65521])
@pytest.mark.parametrize("want_reduced", [False, True])
def test_panel_path_matches_oracle(p, want_reduced):
    """The column-panel forward pass (fused tensor-core application of each
    wave) at small and large primes, on a D' the automatic choice would give
    to the sparse SGE."""
    spec = synth.FLSpec(m=900, n=1301, npiv=300, density=0.04, run_len=(4, 16), seed=19 + p, p=p)
    rp, c, v = synth.fl_matrix(spec)
    res = gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, want_reduced=want_reduced, echelon=gbla.ECHELON_PANELS,
                      stats=True)
    assert res[4]["echelon_method"] == gbla.ECHELON_PANELS
    ref = oracle.rref(spec.m, spec.n, spec.p, rp, c, v) if want_reduced else \
        oracle.echelon(spec.m, spec.n, spec.p, rp, c, v)[:4]
    same(res, ref)


@pytest.mark.parametrize("want_reduced", [False, True])
def test_reduce_simt_variant_matches_oracle(want_reduced):
    spec = SMALL[1]
    rp, c, v = synth.fl_matrix(spec)
    res = gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, want_reduced=want_reduced, variant=gbla.GEMM_SIMT)
    ref = oracle.rref(spec.m, spec.n, spec.p, rp, c, v) if want_reduced else \
        oracle.echelon(spec.m, spec.n, spec.p, rp, c, v)[:4]
    same(res, ref)


def test_reduce_small_workload_rref():
    """The 2,000 x 3,000 workload (1,200 pivots, 4% density, runs of 4-32),
    reduced to RREF, equals the oracle's RREF bit for bit."""
    spec = synth.WORKLOADS["fl_2000x3000"]
    rp, c, v = synth.fl_matrix(spec)
    res = gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, want_reduced=True)
    same(res, oracle.rref(spec.m, spec.n, spec.p, rp, c, v))
    res0 = gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, want_reduced=False)
    same(res0, oracle.echelon(spec.m, spec.n, spec.p, rp, c, v)[:4])


def dense_case(dense, p):
    dense = np.asarray(dense, np.int64) % p
    return synth.dense_to_csr(dense), dense.shape[0], dense.shape[1], p


@pytest.mark.parametrize("want_reduced", [False, True])
@pytest.mark.parametrize("case", ["empty_rows", "identity", "perm_identity", "zero", "duplicates",
                                  "rank_one", "all_pivots", "no_b_block", "p2", "p3", "p7", "wide",
                                  "m0", "n1", "dependent_schur", "dense_square", "dense_tall"])
def test_edge_cases(case, want_reduced):
    rng = np.random.default_rng(hash(case) % 2**32)
    p = 65521
    if case == "empty_rows":
        d = np.where(rng.random((40, 50)) < 0.2, rng.integers(1, p, (40, 50)), 0)
        d[::3] = 0
    elif case == "identity":
        d = np.eye(64, dtype=np.int64)
    elif case == "perm_identity":
        d = np.eye(200, dtype=np.int64)[rng.permutation(200)] * 7
    elif case == "zero":
        d = np.zeros((10, 20), np.int64)
    elif case == "duplicates":
        base = np.where(rng.random((30, 60)) < 0.2, rng.integers(1, p, (30, 60)), 0)
        d = np.vstack([base, base, base[::2] * 3])
    elif case == "rank_one":
        u = rng.integers(1, p, 25)
        w = np.where(rng.random(70) < 0.4, rng.integers(1, p, 70), 0)
        w[3] = 5
        d = np.outer(u, w) % p
    elif case == "all_pivots":
        d = np.triu(rng.integers(1, p, (150, 150)))
    elif case == "no_b_block":
        d = np.triu(rng.integers(0, p, (80, 80))) + np.eye(80, dtype=np.int64)
        d = np.vstack([d, d[5:20] * 2])
    elif case in ("p2", "p3", "p7"):
        p = {"p2": 2, "p3": 3, "p7": 7}[case]
        d = np.where(rng.random((150, 190)) < 0.1, rng.integers(1, p, (150, 190)), 0)
    elif case == "wide":
        d = np.where(rng.random((20, 900)) < 0.05, rng.integers(1, p, (20, 900)), 0)
    elif case == "m0":
        d = np.zeros((0, 30), np.int64)
    elif case == "n1":
        d = rng.integers(0, 3, (12, 1))
    elif case == "dependent_schur":
        # Schur complement of rank < its row count: rows that cancel inside D
        g = rng.integers(0, p, (60, 40))
        basis = np.where(rng.random((40, 300)) < 0.1, rng.integers(1, p, (40, 300)), 0)
        d = (g @ basis) % p
    elif case in ("dense_square", "dense_tall"):
        # one pivot row (column 0), then a Schur complement of full column
        # rank: every column of D' is a pivot column of its echelon form
        d = rng.integers(1, p, (70 if case == "dense_square" else 130, 70))
    (rp, c, v), m, n, p = dense_case(d, p)
    res = gbla.reduce(rp, c, v, (m, n), p, want_reduced=want_reduced)
    ref = oracle.rref(m, n, p, rp, c, v) if want_reduced else oracle.echelon(m, n, p, rp, c, v)[:4]
    same(res, ref)


def test_invalid_inputs_rejected():
    p = 65521
    bad = [
        (np.array([0, 2]), np.array([3, 1]), np.array([1, 1]), (1, 5)),      # unsorted columns
        (np.array([0, 2]), np.array([1, 1]), np.array([1, 1]), (1, 5)),      # duplicate column
        (np.array([0, 1]), np.array([7]), np.array([1]), (1, 5)),            # column out of range
        (np.array([0, 1]), np.array([2]), np.array([0]), (1, 5)),            # explicit zero
        (np.array([0, 1]), np.array([2]), np.array([65521]), (1, 5)),        # value >= p
    ]
    for rp, c, v, shape in bad:
        with pytest.raises(gbla.GblaError) as e:
            gbla.reduce(rp, c, v, shape, p)
        assert e.value.code == 1
    # the context stays usable after a rejected input
    d = np.eye(5, dtype=np.int64)
    rp, c, v = synth.dense_to_csr(d)
    assert gbla.reduce(rp, c, v, (5, 5), p)[0] == 5


def test_device_pointer_path_matches_host_path():
    spec = SMALL[1]
    rp, c, v = synth.fl_matrix(spec)
    host = gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p)
    dev = gbla.reduce_device(torch.from_numpy(rp).cuda(), torch.from_numpy(c).cuda(), t16(v),
                             (spec.m, spec.n), spec.p)
    try:
        same(dev.to_host(), host)
    finally:
        dev.free()


def test_repeatable_bits():
    """The same input gives the same output bits on repeated runs (catches
    races in the level-blocked solve and the pipelines)."""
    spec = SMALL[5]
    rp, c, v = synth.fl_matrix(spec)
    first = gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p)
    for _ in range(5):
        same(gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p), first)


def test_scaled_grouped_workload_matches_oracle():
    """The 40,000 x 60,000 grouped workload scaled by 0.15 (several tiles of
    every kernel, ragged tails): bit-exact against the oracle."""
    spec = synth.scaled("fl_40000x60000", 0.15, seed=777)
    rp, c, v = synth.fl_matrix(spec)
    res = gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, want_reduced=False)
    same(res, oracle.echelon(spec.m, spec.n, spec.p, rp, c, v)[:4])


def test_bounded_wait_expires_cleanly_and_context_survives():
    """A product whose loads are withheld: the MMA issuer's bounded wait
    expires (about a second), the kernel reports a timeout instead of hanging,
    and later products on the same context are still exact."""
    import time
    t0 = time.time()
    assert gbla.selftest_wait_timeout() == 4          # GBLA_E_TIMEOUT
    assert time.time() - t0 < 30
    p = 65521
    rng = np.random.default_rng(3)
    A = rng.integers(0, p, size=(130, 200))
    B = rng.integers(0, p, size=(200, 70))
    C = rng.integers(0, p, size=(130, 70))
    tc = t16(C)
    gbla.modmatmul(t16(A), t16(B), tc, p, sign=-1, variant=gbla.GEMM_TCGEN05)
    assert np.array_equal(from_t16(tc), ref_gemm(A, B, C, p, -1))
