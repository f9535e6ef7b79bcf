"""The exact modular product for 32-bit coefficients (gbla_modmatmul32: four
balanced 8-bit digits per residue in bf16, seven fp32 tensor-memory
accumulators, exact over k-blocks of 256) against exact int64 numpy, at and
beyond its k-block bound with all-extreme operands, and against the 16-bit
product for primes below 2^16."""
import numpy as np
import pytest

from paper_1602_06097_gb300 import gbla

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

PRIMES = [2147483647, 1000000007, 2013265921, 65521, 40009, 3]


def t32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def from_t32(t):
    return t.cpu().numpy().view(np.uint32).astype(np.int64)


def ref32(A, B, C, p, sign):
    """Exact in int64: B split into 16-bit halves keeps every sum below 2^62."""
    A, B = A.astype(np.int64), B.astype(np.int64)
    lo = (A @ (B & 0xFFFF)) % p
    hi = (A @ (B >> 16)) % p
    X = (lo + hi * (65536 % p)) % p
    return (C + sign * X) % p


@pytest.mark.parametrize("shape", [(1, 1, 1), (130, 70, 200), (257, 65, 1000), (300, 129, 1536), (128, 64, 256)])
@pytest.mark.parametrize("p", PRIMES)
@pytest.mark.parametrize("sign", [-1, 1])
def test_modmatmul32_random(shape, p, sign):
    M, N, K = shape
    rng = np.random.default_rng(M + 3 * N + 7 * K + p % 1000 + sign)
    A = rng.integers(0, p, size=(M, K))
    B = rng.integers(0, p, size=(K, N))
    C = rng.integers(0, p, size=(M, N))
    tc = t32(C)
    gbla.modmatmul32(t32(A), t32(B), tc, p, sign=sign)
    assert np.array_equal(from_t32(tc), ref32(A, B, C, p, sign))


@pytest.mark.parametrize("K", [255, 256, 257, 1024, 4096 + 64])
@pytest.mark.parametrize("fill", ["pm1", "half", "halfp1", "mixed"])
@pytest.mark.parametrize("p", [2147483647, 2013265921])
def test_modmatmul32_at_the_k_block_bound(K, fill, p):
    """All-extreme operands: the balanced digits of (p-1)/2 and (p+1)/2 are
    the largest the split gives; every accumulator takes up to four maximal
    products per k."""
    M, N = 192, 96
    h = (p - 1) // 2
    vals = {"pm1": p - 1, "half": h, "halfp1": h + 1}
    if fill == "mixed":
        rng = np.random.default_rng(K)
        choices = np.array([p - 1, h, h + 1, 1, 0, 0x7F7F7F7F % p, p - 0x7F7F7F7F % p, 128, p - 128])
        A = rng.choice(choices, size=(M, K))
        B = rng.choice(choices, size=(K, N))
    else:
        A = np.full((M, K), vals[fill])
        B = np.full((K, N), vals[fill])
    C = np.zeros((M, N), np.int64)
    tc = t32(C)
    gbla.modmatmul32(t32(A), t32(B), tc, p, sign=1)
    assert np.array_equal(from_t32(tc), ref32(A, B, C, p, 1))


def test_modmatmul32_equals_the_16_bit_product():
    p = 65521
    rng = np.random.default_rng(7)
    M, N, K = 300, 200, 2000
    A = rng.integers(0, p, size=(M, K))
    B = rng.integers(0, p, size=(K, N))
    C = rng.integers(0, p, size=(M, N))
    c32 = t32(C)
    gbla.modmatmul32(t32(A), t32(B), c32, p)
    c16 = torch.from_numpy(C.astype(np.uint16).view(np.int16)).cuda()
    gbla.modmatmul(torch.from_numpy(A.astype(np.uint16).view(np.int16)).cuda(),
                   torch.from_numpy(B.astype(np.uint16).view(np.int16)).cuda(), c16, p, sign=-1)
    assert np.array_equal(from_t32(c32), c16.cpu().numpy().view(np.uint16).astype(np.int64))


@pytest.mark.parametrize("p", [2, 4, 2147483648, 4294967291, 1000000008])
def test_modmatmul32_rejects_bad_primes(p):
    A = torch.zeros((4, 4), dtype=torch.int32, device="cuda")
    with pytest.raises(gbla.GblaError) as e:
        gbla.modmatmul32(A, A, A.clone(), p)
    assert e.value.code == 1
