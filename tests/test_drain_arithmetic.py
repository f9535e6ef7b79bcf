"""Host checks of the integer arithmetic the tensor-core product relies on.

The product accumulates balanced 8-bit digit products exactly in fp32 over a
k-block of 512 (every accumulator |x| <= 2^24) and drains, per element, the
pair (P, Q) into a running residue as (run + 256 P + Q) mod p.  The drain
converts P and Q exactly to integers, estimates q = round(P / p) with one
fused multiply-add of P * fl(1/p) into the 2^23 rounding window, forms
t = run + 256 (P - q p) + Q + bias with bias = 256 p + ceil(2^24 / p) p and
finishes with one Barrett step (multiplier floor(2^32 / p)) and one
conditional subtraction.  The digit planes hold each digit |v| <= 256 as the
high half of the fp32 pattern of v, built by adding v to the pattern of
1.5 * 2^23 and subtracting 1.5 * 2^23.

Here those steps are replayed with IEEE fp32 arithmetic (numpy float32; a
fused multiply-add is formed exactly in float64, where these products and
sums are exact, and rounded once) and compared with exact integer arithmetic
over the whole accumulator range, its ends included, for small and large
primes.  The gathered product's drain of four digit-product sums
(H, M1, M2, L: run + 65536 H + 256 (M1 + M2) + L, k-blocks of 1,024) is
replayed the same way.  A mistake in a bound (the 5p/8 remainder, the bias, the Barrett
range) shows up as a mismatch or a failed range assertion.
"""
import numpy as np
import pytest

MAGIC = np.float32(12582912.0)          # 1.5 * 2^23
MAGIC_BITS = 0x4B400000
PRIMES = [11, 13, 251, 257, 8191, 32003, 40009, 65519, 65521]


def fmaf(a, b, c):
    """fp32 fused multiply-add: exact in float64 for these operands, one rounding."""
    return (a.astype(np.float64) * np.float64(b) + np.float64(c)).astype(np.float32)


def accumulators(rng, n):
    """Exact fp32 accumulators |x| <= 2^24, a quarter of them at or next to the ends."""
    x = rng.integers(-(1 << 24), (1 << 24) + 1, n)
    k = n // 4
    x[:k] = rng.choice([-(1 << 24), -(1 << 24) + 1, -1, 0, 1, (1 << 24) - 1, 1 << 24], k)
    return x


def drain_step(run, pa, qa, p):
    """The drain of one k-block, step by step as the kernel does it."""
    pinv = np.float32(1.0 / p)
    bias = 256 * p + ((1 << 24) + p - 1) // p * p
    bm = 0xFFFFFFFF // p
    paf, qaf = pa.astype(np.float32), qa.astype(np.float32)
    ip = np.rint(paf).astype(np.int64)      # exact conversions
    iq = np.rint(qaf).astype(np.int64)
    qp = fmaf(paf, pinv, MAGIC).view(np.int32).astype(np.int64) - MAGIC_BITS
    rp = ip - qp * p
    assert np.abs(rp).max() <= 5 * p / 8
    t = run + bias + iq + 256 * rp
    assert t.min() >= 96 * p and t.max() < (1 << 25) + 418 * p < (1 << 32)
    q = (t.astype(np.uint64) * np.uint64(bm)) >> np.uint64(32)
    s = t - q.astype(np.int64) * p
    assert s.min() >= 0 and s.max() < 2 * p
    return np.where(s >= p, s - p, s)


@pytest.mark.parametrize("p", PRIMES)
def test_drain_step_is_exact(p):
    rng = np.random.default_rng(p)
    n = 60000
    pa, qa = accumulators(rng, n), accumulators(rng, n)
    run = rng.integers(0, p, n)
    assert np.array_equal(pa.astype(np.float32).astype(np.int64), pa)   # exact in fp32
    assert np.array_equal(drain_step(run, pa, qa, p), (run + 256 * pa + qa) % p)


@pytest.mark.parametrize("p", PRIMES)
def test_drain_over_k_blocks_equals_the_modular_dot_product(p):
    """Digits, their fp32 block sums and the drain chained over several
    k-blocks give the modular dot product of the residues."""
    rng = np.random.default_rng(1000 + p)
    rows, K, KB = 64, 3 * 512 + 77, 512
    a = rng.integers(0, p, (rows, K))
    b = rng.integers(0, p, K)
    a[0], b[:5] = p - 1, p - 1                     # extreme residues

    def split(x):                                  # balanced digits
        s = np.where(x > p // 2, x - p, x)
        hi = (s + 128) >> 8
        return hi, s - 256 * hi

    ah, al = split(a)
    bh, bl = split(b)
    bh2, bl2 = split(256 * b % p)
    run = np.zeros(rows, np.int64)
    for k0 in range(0, K, KB):
        sl = slice(k0, min(K, k0 + KB))
        P = (ah[:, sl] * bh2[sl] + al[:, sl] * bh[sl]).sum(axis=1)
        Q = (ah[:, sl] * bl2[sl] + al[:, sl] * bl[sl]).sum(axis=1)
        assert np.abs(P).max() <= 1 << 24 and np.abs(Q).max() <= 1 << 24
        run = drain_step(run, P, Q, p)
    assert np.array_equal(run, (a * b).sum(axis=1) % p)


def drain_step4(run, ha, m1a, m2a, la, p):
    """The gathered product's drain of its four digit-product sums
    (65536 H + 256 (M1 + M2) + L), step by step as the kernel does it:
    float-only rounded quotients and exact remainders read back through the
    1.5 * 2^23 bit pattern, their offsets folded into the bias mod 2^32."""
    pinv, pf = np.float32(1.0 / p), np.float32(p)
    bm = 0xFFFFFFFF // p
    c16 = 65536 % p
    if c16 > p // 2:
        c16 -= p
    bias = ((1 << 30) + (1 << 26) + p - 1) // p * p
    biasx = (bias - MAGIC_BITS * (513 + c16)) % (1 << 32)
    words = []
    for x in (ha, m1a, m2a, la):
        xf = x.astype(np.float32)
        q = fmaf(xf, pinv, MAGIC) - MAGIC
        r = fmaf(-q, pf, xf)
        assert np.array_equal(r.astype(np.int64), x - q.astype(np.int64) * p)   # exact remainder
        assert np.abs(r).max() <= p // 2 + 1
        words.append((r + MAGIC).view(np.uint32).astype(np.int64))
    rh, rm1, rm2, rl = words
    true = (run + bias + (rl - MAGIC_BITS) + 256 * (rm1 + rm2 - 2 * MAGIC_BITS)
            + c16 * (rh - MAGIC_BITS))
    assert true.min() >= 0 and true.max() < (1 << 31) + (1 << 27)
    t = (run + biasx + rl + 256 * (rm1 + rm2) + (c16 % (1 << 32)) * rh) % (1 << 32)
    assert np.array_equal(t, true)                                # the 32-bit word is the true sum
    q = (t.astype(np.uint64) * np.uint64(bm)) >> np.uint64(32)
    s = t - q.astype(np.int64) * p
    assert s.min() >= 0 and s.max() < 2 * p
    return np.minimum(s, np.where(s >= p, s - p, 1 << 40))


def sums(rng, n, lim):
    x = rng.integers(-lim, lim + 1, n)
    k = n // 4
    x[:k] = rng.choice([-lim, -lim + 1, -1, 0, 1, lim - 1, lim], k)
    return x


@pytest.mark.parametrize("p", PRIMES)
def test_drain_step4_is_exact(p):
    rng = np.random.default_rng(7 * p)
    n = 60000
    ha, m1a, m2a, la = (sums(rng, n, 1 << 24) for _ in range(4))
    run = rng.integers(0, p, n)
    assert np.array_equal(drain_step4(run, ha, m1a, m2a, la, p),
                          (run + 65536 * ha + 256 * (m1a + m2a) + la) % p)


@pytest.mark.parametrize("p", PRIMES)
def test_drain4_over_k_blocks_equals_the_modular_dot_product(p):
    """Balanced digits of both operands, the four fp32 block sums of digit
    products (H = ah bh, M1 = ah bl, M2 = al bh, L = al bl) and the drain
    chained over k-blocks of 1,024 give the modular dot product."""
    rng = np.random.default_rng(2000 + p)
    rows, K, KB = 64, 2 * 1024 + 77, 1024
    a = rng.integers(0, p, (rows, K))
    b = rng.integers(0, p, K)
    a[0], b[:5] = p - 1, p - 1
    a[1], b[5:1100] = (p + 1) // 2, (p + 1) // 2    # most negative balanced residue

    def split(x):
        s = np.where(x > p // 2, x - p, x)
        hi = (s + 128) >> 8
        return hi, s - 256 * hi

    ah, al = split(a)
    bh, bl = split(b)
    assert max(np.abs(ah).max(), np.abs(al).max(), np.abs(bh).max(), np.abs(bl).max()) <= 128
    run = np.zeros(rows, np.int64)
    for k0 in range(0, K, KB):
        sl = slice(k0, min(K, k0 + KB))
        H = (ah[:, sl] * bh[sl]).sum(axis=1)
        M1 = (ah[:, sl] * bl[sl]).sum(axis=1)
        M2 = (al[:, sl] * bh[sl]).sum(axis=1)
        L = (al[:, sl] * bl[sl]).sum(axis=1)
        assert max(np.abs(H).max(), np.abs(M1).max(), np.abs(M2).max(), np.abs(L).max()) <= 1 << 24
        run = drain_step4(run, H, M1, M2, L, p)
    assert np.array_equal(run, (a * b).sum(axis=1) % p)


def drain_step4_k128(ha, m1a, m2a, la, p):
    """The fused panel product's drain (K <= 128: every sum within 2^21):
    H and M1 + M2 by a rounded quotient, L straight through the 1.5 * 2^23
    window, offsets folded into the bias mod 2^32."""
    pinv, pf = np.float32(1.0 / p), np.float32(p)
    bm = 0xFFFFFFFF // p
    c16 = 65536 % p
    if c16 > p // 2:
        c16 -= p
    bias = ((1 << 30) + (1 << 24) + p - 1) // p * p
    biasy = (bias - MAGIC_BITS * (257 + c16)) % (1 << 32)
    words = []
    for x in (ha, m1a + m2a):
        xf = x.astype(np.float32)
        assert np.array_equal(xf.astype(np.int64), x)              # M1 + M2 exact in fp32
        q = fmaf(xf, pinv, MAGIC) - MAGIC
        r = fmaf(-q, pf, xf)
        assert np.abs(r).max() <= p // 2 + 1
        words.append((r + MAGIC).view(np.uint32).astype(np.int64))
    rh, rm = words
    lw = (la.astype(np.float32) + MAGIC).view(np.uint32).astype(np.int64)
    assert np.array_equal(lw - MAGIC_BITS, la)                     # L read exactly
    true = bias + (lw - MAGIC_BITS) + 256 * (rm - MAGIC_BITS) + c16 * (rh - MAGIC_BITS)
    assert true.min() >= 0 and true.max() < (1 << 31) + (1 << 25)
    t = (biasy + lw + 256 * rm + (c16 % (1 << 32)) * rh) % (1 << 32)
    assert np.array_equal(t, true)
    q = (t.astype(np.uint64) * np.uint64(bm)) >> np.uint64(32)
    s = t - q.astype(np.int64) * p
    assert s.min() >= 0 and s.max() < 2 * p
    return np.minimum(s, np.where(s >= p, s - p, 1 << 40))


@pytest.mark.parametrize("p", PRIMES)
def test_drain_step4_k128_is_exact(p):
    rng = np.random.default_rng(11 * p)
    n = 60000
    ha, m1a, m2a, la = (sums(rng, n, 1 << 21) for _ in range(4))
    assert np.array_equal(drain_step4_k128(ha, m1a, m2a, la, p), (65536 * ha + 256 * (m1a + m2a) + la) % p)


def test_digit_bf16_patterns():
    """High half of the fp32 pattern built from 1.5 * 2^23 equals the bf16
    round-to-nearest-even of every digit value, and the low half is zero."""
    v = np.arange(-256, 257, dtype=np.int64)
    f = (MAGIC_BITS + v).astype(np.uint32).view(np.float32) - MAGIC
    assert np.array_equal(f.astype(np.int64), v)
    bits = f.view(np.uint32).astype(np.uint64)
    assert np.all(bits & 0xFFFF == 0)
    ref = v.astype(np.float32).view(np.uint32).astype(np.uint64)
    rne = (ref + 0x7FFF + ((ref >> 16) & 1)) >> 16
    assert np.array_equal(bits >> 16, rne)
