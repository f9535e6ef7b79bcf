// common.cuh -- shared device helpers of the GB300 FL reduction library.
//
// Residues of GF(p), p < 2^16 prime, are uint16/uint32 values in [0, p).
// Products of two residues are < 2^32; sums of products are accumulated in
// uint64 and reduced with a Barrett step only when a value is read as a
// multiplier or stored (delayed reduction).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/gbla.h"

namespace gbla {

// ---------------------------------------------------------------- modulus
struct ModP {
    uint32_t p;
    uint32_t mu32;   // floor((2^32 - 1) / p)
    uint64_t mu64;   // floor((2^64 - 1) / p)
    float pf;        // (float)p
    float pinv;      // 1/p rounded to float
    uint32_t r256;   // 256 mod p
    uint32_t r32;    // 2^32 mod p
};

inline ModP make_modp(uint32_t p) {
    ModP m;
    m.p = p;
    m.mu32 = (uint32_t)(0xFFFFFFFFu / p);
    m.mu64 = (uint64_t)(~0ull / (uint64_t)p);
    m.pf = (float)p;
    m.pinv = 1.0f / (float)p;
    m.r256 = 256u % p;
    m.r32 = (uint32_t)((1ull << 32) % p);
    return m;
}

// x mod p for x < 2^32: quotient estimate from the high word of x*mu32 is
// low by at most 2.
__device__ __forceinline__ uint32_t mod32(uint32_t x, const ModP &m) {
    uint32_t q = __umulhi(x, m.mu32);
    uint32_t r = x - q * m.p;
    if (r >= m.p) r -= m.p;
    if (r >= m.p) r -= m.p;
    return r;
}

// x mod p for any 64-bit x.
__device__ __forceinline__ uint32_t mod64(uint64_t x, const ModP &m) {
    uint64_t q = __umul64hi(x, m.mu64);
    uint64_t r = x - q * (uint64_t)m.p;
    while (r >= m.p) r -= m.p;
    return (uint32_t)r;
}

// x mod p for x < 2^40 (sums of at most 256 products of residues): the high
// byte times 2^32 mod p stays below 2^24.
__device__ __forceinline__ uint32_t mod40(uint64_t x, const ModP &m) {
    const uint32_t hi = (uint32_t)(x >> 32);
    return mod32(mod32((uint32_t)x, m) + hi * m.r32, m);
}

__device__ __forceinline__ uint32_t mulmod(uint32_t a, uint32_t b, const ModP &m) {
    return mod32(a * b, m);
}

// a^(p-2) = a^-1 (Fermat), a != 0 mod p.
__device__ __forceinline__ uint32_t invmod(uint32_t a, const ModP &m) {
    uint32_t e = m.p - 2, r = 1, b = a % m.p;
    while (e) {
        if (e & 1) r = mulmod(r, b, m);
        b = mulmod(b, b, m);
        e >>= 1;
    }
    return r;
}

// ------------------------------------------------------- digit planes
// A residue a in [0,p) is written in balanced form s = a or a - p with
// |s| <= (p-1)/2 <= 32760, then split s = 256*hi + lo with lo in [-128,127]
// and hi in [-128,128].  Both digits are integers of at most 8 significant
// bits, hence exact in bf16; a product of two digits is at most 2^14 in
// magnitude, so up to 1024 of them (512 pairs) sum exactly in fp32.
__device__ __forceinline__ void digits(uint32_t a, uint32_t p, int &hi, int &lo) {
    int s = (a > (p >> 1)) ? (int)a - (int)p : (int)a;
    hi = (s + 128) >> 8;   // arithmetic shift = floor
    lo = s - (hi << 8);
}

// fp32 pattern of a digit |v| <= 256: v added to the pattern of 1.5 * 2^23
// (one unit in the last place each), then one fp32 subtraction; no
// integer-to-float conversion.  A digit has at most 8 significant bits, so the
// low half of the pattern is zero and the high half is the exact bf16.
__device__ __forceinline__ uint32_t digit_f32_bits(int v) {
    return __float_as_uint(__int_as_float(0x4B400000 + v) - 12582912.0f);
}

__device__ __forceinline__ __nv_bfloat16 i2bf(int v) {
    return __ushort_as_bfloat16((unsigned short)(digit_f32_bits(v) >> 16));
}

// Plane-set geometry.  An "A-operand" set holds 2 planes (hi, lo) of an
// M x K matrix, a "B-operand" set holds 4 planes (hi, lo of b, hi, lo of
// b' = 256*b mod p) of an N x K matrix (i.e. B transposed).  rows and kp (the
// padded K) are multiples of 128; padding is 0.  The planes are interleaved
// by 32-wide K chunks: a row is kp / 32 chunks, each holding 32 bf16 of every
// plane in turn, so that one 128-byte row segment carries the (hi, lo) pair of
// a chunk and the product loads operand tiles as 128-byte rows.
struct Planes {
    __nv_bfloat16 *ptr;
    int64_t rows;   // padded rows
    int64_t kp;     // padded K
    int nplanes;    // 2 or 4
    __host__ __device__ size_t plane_elems() const { return (size_t)rows * (size_t)kp; }
    __host__ __device__ int64_t row_elems() const { return kp * nplanes; }
    // element (r, k) of plane h
    __host__ __device__ __nv_bfloat16 *at(int h, int64_t r, int64_t k) const {
        return ptr + (size_t)r * (size_t)row_elems() + (size_t)(k >> 5) * (size_t)(32 * nplanes) + (size_t)(h * 32) +
               (size_t)(k & 31);
    }
};

__host__ __device__ inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// ------------------------------------------------------- error reporting
// Device-side status word: kernels atomicOr one of these bits; the host maps
// them to GBLA_* codes.
enum : uint32_t {
    DEV_ERR_INVAL = 1u,
    DEV_ERR_TIMEOUT = 2u,
    DEV_ERR_INTERNAL = 4u,
};

__device__ __forceinline__ void dev_fail(uint32_t *err, uint32_t bit) {
    if (err) atomicOr(err, bit);
}

// ------------------------------------------- transposing plane conversion
// One 64 x 64 tile of a transposing conversion into digit planes, run by a
// block of 256 threads:
//   dst row (row0 + r), column (dcol0 + k)  <-  src[g(k) * lds + col0 + r]
// for r in [r0, r0 + 64), k in [k0, k0 + 64); zero where r >= R, k >= Kc or
// g(k) < 0, with g(k) = rgather ? rgather[k] : k.  Source rows are read 64
// entries at a time; each plane row receives 128 contiguous bytes written as
// 16-byte vectors.  The residues b' = 256 * b mod p of a 4-plane set use a
// Barrett reduction.
constexpr int TP_TILE = 64;
// Transpose tile: row r (of the destination), k chunk c (8 residues) at
// t[r][c ^ ((r >> 3) & 7)]: both the scattered writes and the 16-byte row
// reads of the transpose are free of bank conflicts.
struct TpSmem {
    uint4 t[TP_TILE][TP_TILE / 8];
};

// Two digits as a bf16 pair (lo_elem in the low half).
__device__ __forceinline__ uint32_t pack_bf2(int lo_elem, int hi_elem) {
    return __byte_perm(digit_f32_bits(lo_elem), digit_f32_bits(hi_elem), 0x7632);
}

// Digit planes of 8 consecutive residues a[0..7] at row r, columns k0 .. k0+7
// (k0 a multiple of 8) of every plane: 16-byte stores.
__device__ __forceinline__ void store_digits8(const Planes &dst, int64_t r, int64_t k0, const uint32_t (&a)[8],
                                              const ModP &mp) {
    uint32_t vh[4], vl[4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
        int h0, l0, h1, l1;
        digits(a[e], mp.p, h0, l0);
        digits(a[e + 1], mp.p, h1, l1);
        vh[e / 2] = pack_bf2(h0, h1);
        vl[e / 2] = pack_bf2(l0, l1);
    }
    *reinterpret_cast<uint4 *>(dst.at(0, r, k0)) = make_uint4(vh[0], vh[1], vh[2], vh[3]);
    *reinterpret_cast<uint4 *>(dst.at(1, r, k0)) = make_uint4(vl[0], vl[1], vl[2], vl[3]);
    if (dst.nplanes == 4) {
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            int h0, l0, h1, l1;
            digits(mod32(a[e] * mp.r256, mp), mp.p, h0, l0);
            digits(mod32(a[e + 1] * mp.r256, mp), mp.p, h1, l1);
            vh[e / 2] = pack_bf2(h0, h1);
            vl[e / 2] = pack_bf2(l0, l1);
        }
        *reinterpret_cast<uint4 *>(dst.at(2, r, k0)) = make_uint4(vh[0], vh[1], vh[2], vh[3]);
        *reinterpret_cast<uint4 *>(dst.at(3, r, k0)) = make_uint4(vl[0], vl[1], vl[2], vl[3]);
    }
}

// 8 consecutive residues src[base .. base + 7] (positions at or past n read
// as 0): one 16-byte load when all are in range and aligned.
__device__ __forceinline__ void load8_u16(const uint16_t *__restrict__ p, int64_t avail, uint16_t (&w)[8]) {
    if (avail >= 8 && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
        const uint4 x = __ldg(reinterpret_cast<const uint4 *>(p));
        const uint32_t u[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int e = 0; e < 8; ++e) w[e] = (uint16_t)(u[e >> 1] >> ((e & 1) * 16));
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) w[e] = e < avail ? p[e] : (uint16_t)0;
    }
}

__device__ __forceinline__ void tp_tile(const Planes &dst, int64_t row0, int64_t r0, int64_t k0, int64_t R, int64_t Kc,
                                        const uint16_t *__restrict__ src, int64_t lds, int64_t col0,
                                        const int32_t *__restrict__ rgather, const ModP &mp, TpSmem &sm,
                                        int64_t dcol0 = 0)
{
    static_assert(TP_TILE == 64, "256 threads: 8 column groups x 32 rows, twice");
    const int tid = threadIdx.x;
    const int cq = tid & 7, kr = tid >> 3;   // source columns r0 + 8 cq .., source row k0 + kr (+ 32)
    uint16_t w[2][8];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int64_t k = k0 + kr + 32 * i;
        int64_t sr = -1;
        if (k < Kc) sr = rgather ? (int64_t)rgather[k] : k;
        const int64_t r = r0 + cq * 8;
        if (sr >= 0 && r < R) {
            load8_u16(src + sr * lds + col0 + r, R - r, w[i]);
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) w[i][e] = 0;
        }
    }
    uint16_t *t16 = reinterpret_cast<uint16_t *>(&sm.t[0][0]);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int kl = kr + 32 * i;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int rl = cq * 8 + e;   // (rl >> 3) & 7 == cq
            t16[rl * TP_TILE + ((((kl >> 3) ^ cq) << 3) | (kl & 7))] = w[i][e];
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = tid; it < TP_TILE * 8; it += 256) {
        const int c = it & 7, rr = it >> 3;
        const uint4 x = sm.t[rr][c ^ ((rr >> 3) & 7)];
        const uint32_t u[4] = {x.x, x.y, x.z, x.w};
        uint32_t a[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) a[e] = (u[e >> 1] >> ((e & 1) * 16)) & 0xFFFFu;
        store_digits8(dst, row0 + r0 + rr, dcol0 + k0 + c * 8, a, mp);
    }
}

}  // namespace gbla

#define GBLA_CUDA_TRY(expr)                                      \
    do {                                                         \
        cudaError_t _e = (expr);                                 \
        if (_e != cudaSuccess) {                                 \
            ::gbla::set_last_cuda_error(_e, #expr, __FILE__, __LINE__); \
            return (_e == cudaErrorMemoryAllocation) ? GBLA_E_NOMEM : GBLA_E_CUDA; \
        }                                                        \
    } while (0)

#define GBLA_TRY(expr)                  \
    do {                                \
        int _rc = (expr);               \
        if (_rc != GBLA_OK) return _rc; \
    } while (0)

namespace gbla {
void set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line);
// Kernel launches made by this thread (reported in gbla_stats.launches).
extern thread_local long long g_launches;
// Dense-product launches on CTA pairs made by this thread.
extern thread_local long long g_pair_launches;
// Call right after a kernel launch: counts it and returns the launch status.
inline cudaError_t launch_check() {
    ++g_launches;
    return cudaGetLastError();
}
}
