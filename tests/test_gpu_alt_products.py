"""GPU parity of the Schur update's measured alternatives (GBLA_GEMM_FP64 on
mma.sync f64, GBLA_GEMM_U8 on mma.sync u8), against exact int64 numpy and
closed forms at and beyond their exactness bounds, and of whole reductions
whose Schur update runs on them, against the oracle.

Bounds: FP64 accumulates balanced residues (|s| <= 32760), exact over k-blocks
of 2^23 (2^23 * 32760^2 < 2^53); U8 accumulates byte products in s32, the
middle accumulator taking two products of at most 255^2 per k, exact over
k-blocks of 2^14 (2 * 255^2 * 2^14 < 2^31).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1602_06097_gb300 import gbla, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

VARIANTS = [gbla.GEMM_FP64, gbla.GEMM_U8]
IDS = ["fp64", "u8"]


def t16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint16).view(np.int16)).cuda()


def from_t16(t):
    return t.cpu().numpy().view(np.uint16).astype(np.int64)


def ref_gemm(A, B, C, p, sign):
    return (C + sign * (A.astype(np.int64) @ B.astype(np.int64))) % p


def same(a, b):
    assert a[0] == b[0], f"rank {a[0]} != {b[0]}"
    for x, y, what in zip(a[1:4], b[1:4], ("row_ptr", "col", "val")):
        assert np.array_equal(np.asarray(x, np.int64), np.asarray(y, np.int64)), f"{what} differs"


@pytest.mark.parametrize("variant", VARIANTS, ids=IDS)
@pytest.mark.parametrize("shape", [(1, 1, 1), (65, 63, 33), (130, 70, 200), (257, 385, 1000), (300, 129, 1536)])
@pytest.mark.parametrize("p", [65521, 32003, 8191, 11, 3])
@pytest.mark.parametrize("sign", [-1, 1])
def test_alt_modmatmul_random(variant, shape, p, sign):
    M, N, K = shape
    rng = np.random.default_rng(M * 7 + N * 13 + K + p + sign + 5 * variant)
    A = rng.integers(0, p, size=(M, K))
    B = rng.integers(0, p, size=(K, N))
    C = rng.integers(0, p, size=(M, N))
    tc = t16(C)
    gbla.modmatmul(t16(A), t16(B), tc, p, sign=sign, variant=variant)
    assert np.array_equal(from_t16(tc), ref_gemm(A, B, C, p, sign))


@pytest.mark.parametrize("K", [16383, 16384, 16385, 20000, 32768 + 32, 40001])
@pytest.mark.parametrize("fill", ["max_mid", "pm1", "mixed"])
def test_u8_at_and_beyond_the_k_block_bound(K, fill):
    """Operands whose byte products are the largest the residues of 65521
    allow: a = 0xFEFF (bytes 254, 255) against b = 0xFFF0 (255, 240) gives a
    middle sum of 125,985 per k, which exceeds 2^31 after 17,046 terms, so any
    K >= 20,000 is exact only if the k-blocks are drained."""
    p = 65521
    M, N = 130, 72
    if fill == "max_mid":
        A = np.full((M, K), 0xFEFF)
        B = np.full((K, N), 0xFFF0)
    elif fill == "pm1":
        A = np.full((M, K), p - 1)
        B = np.full((K, N), p - 1)
    else:
        rng = np.random.default_rng(K)
        choices = np.array([0xFEFF, 0xFFF0, p - 1, 0xFF00, 0x00FF, 1, 0])
        A = rng.choice(choices, size=(M, K))
        B = rng.choice(choices, size=(K, N))
    C = np.zeros((M, N), np.int64)
    tc = t16(C)
    gbla.modmatmul(t16(A), t16(B), tc, p, sign=1, variant=gbla.GEMM_U8)
    assert np.array_equal(from_t16(tc), ref_gemm(A, B, C, p, 1))


@pytest.mark.parametrize("K", [100000, 3 * 16384 + 7])
@pytest.mark.parametrize("sign", [-1, 1])
def test_u8_constant_operands_closed_form(K, sign):
    """Constant operands: every output is (C + sign * K * a * b) mod p."""
    p = 65521
    a, b, c0 = 0xFEFF, 0xFFF0, 12345
    M, N = 64, 64
    A = torch.full((M, K), a - 65536, dtype=torch.int16, device="cuda")
    B = torch.full((K, N), b - 65536, dtype=torch.int16, device="cuda")
    C = torch.full((M, N), c0, dtype=torch.int16, device="cuda")
    gbla.modmatmul(A, B, C, p, sign=sign, variant=gbla.GEMM_U8)
    want = (c0 + sign * K * a * b) % p
    assert bool(((C.to(torch.int32) & 0xFFFF) == want).all())


def test_fp64_beyond_the_k_block_bound():
    """Balanced operands 32759 and -32759 (odd products of 32759^2): the
    running sum passes 2^53 after 8,393,000 terms, where fp64 can no longer
    hold an odd integer, so K = 2^23 + 2^16 + 32 is exact only if the k-block
    of 2^23 is drained.  The result follows in closed form."""
    p = 65521
    K = (1 << 23) + (1 << 16) + 32
    a, b = 32759, p - 32759
    assert 32759 ** 2 * K > 2 ** 53
    M, N = 64, 64
    A = torch.full((M, K), a, dtype=torch.int16, device="cuda")
    B = torch.full((K, N), b, dtype=torch.int16, device="cuda")
    C = torch.zeros((M, N), dtype=torch.int16, device="cuda")
    gbla.modmatmul(A, B, C, p, sign=1, variant=gbla.GEMM_FP64)
    want = (K * a * b) % p
    got = C.to(torch.int32) & 0xFFFF
    del A, B
    torch.cuda.empty_cache()
    assert bool((got == want).all())


@pytest.mark.parametrize("variant", VARIANTS, ids=IDS)
@pytest.mark.parametrize("fill", ["pm1", "half", "halfp1"])
def test_alt_extreme_operands(variant, fill):
    p = 65521
    h = (p - 1) // 2
    v = {"pm1": p - 1, "half": h, "halfp1": h + 1}[fill]
    M, N, K = 200, 130, 5000
    A = np.full((M, K), v)
    B = np.full((K, N), v)
    C = np.full((M, N), p - 1)
    tc = t16(C)
    gbla.modmatmul(t16(A), t16(B), tc, p, sign=-1, variant=variant)
    assert np.array_equal(from_t16(tc), ref_gemm(A, B, C, p, -1))


FL_SPECS = [
    synth.FLSpec(m=600, n=900, npiv=360, density=0.04, run_len=(4, 24), seed=801),
    synth.FLSpec(m=1500, n=2100, npiv=1000, density=0.03, run_len=(8, 40), seed=802, p=32003),
    synth.FLSpec(m=2600, n=3700, npiv=1900, density=0.02, run_len=(16, 64), group=(2, 8), seed=803),
]


@pytest.mark.parametrize("variant", VARIANTS, ids=IDS)
@pytest.mark.parametrize("spec", FL_SPECS, ids=[f"{s.m}x{s.n}" for s in FL_SPECS])
def test_reduction_with_alt_schur_equals_oracle(variant, spec):
    rp, c, v = synth.fl_matrix(spec)
    res = gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, variant=variant, stats=True)
    assert res[4]["path"] == gbla.PATH_DENSE
    same(res, oracle.echelon(spec.m, spec.n, spec.p, rp, c, v))


@pytest.mark.parametrize("variant", VARIANTS, ids=IDS)
def test_reduced_form_with_alt_schur_equals_oracle(variant):
    spec = FL_SPECS[0]
    rp, c, v = synth.fl_matrix(spec)
    res = gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, want_reduced=True, variant=variant)
    same(res, oracle.rref(spec.m, spec.n, spec.p, rp, c, v))


@pytest.mark.parametrize("variant", VARIANTS, ids=IDS)
def test_alt_schur_refusals(variant):
    spec = FL_SPECS[0]
    rp, c, v = synth.fl_matrix(spec)
    with pytest.raises(gbla.GblaError) as e:
        gbla.reduce(rp, c, v, (spec.m, spec.n), spec.p, variant=variant, path=gbla.PATH_SPARSE)
    assert e.value.code == 6
    small = synth.FLSpec(m=60, n=90, npiv=30, density=0.1, run_len=(2, 6), seed=5, p=7)
    rp, c, v = synth.fl_matrix(small)
    with pytest.raises(gbla.GblaError) as e:
        gbla.reduce(rp, c, v, (small.m, small.n), small.p, variant=variant)
    assert e.value.code == 6


@pytest.mark.parametrize("variant", VARIANTS, ids=IDS)
def test_pipe_peak_is_measured(variant):
    tops = gbla.pipe_peak(variant)
    assert math.isfinite(tops) and tops > 0.0


def test_pipe_peak_rejects_other_variants():
    for v in (gbla.GEMM_AUTO, gbla.GEMM_TCGEN05, gbla.GEMM_SIMT, 7):
        with pytest.raises(gbla.GblaError) as e:
            gbla.pipe_peak(v)
        assert e.value.code == 1
