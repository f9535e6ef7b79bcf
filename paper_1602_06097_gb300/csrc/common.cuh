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

__device__ __forceinline__ __nv_bfloat16 i2bf(int v) { return __float2bfloat16_rn((float)v); }

// Plane-set geometry.  An "A-operand" set holds 2 planes (hi, lo) of an
// M x K matrix, a "B-operand" set holds 4 planes (hi, lo of b, hi, lo of
// b' = 256*b mod p) of an N x K matrix (i.e. B transposed).  Each plane is
// rows x kp bf16 row-major with rows and kp multiples of 128; padding is 0.
struct Planes {
    __nv_bfloat16 *ptr;
    int64_t rows;   // padded rows per plane
    int64_t kp;     // padded K (row length)
    int nplanes;    // 2 or 4
    __host__ __device__ size_t plane_elems() const { return (size_t)rows * (size_t)kp; }
    __host__ __device__ __nv_bfloat16 *plane(int h) const { return ptr + (size_t)h * plane_elems(); }
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
// Call right after a kernel launch: counts it and returns the launch status.
inline cudaError_t launch_check() {
    ++g_launches;
    return cudaGetLastError();
}
}
