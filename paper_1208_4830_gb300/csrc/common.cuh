// common.cuh -- device building blocks shared by the kernels of the SBLM library:
// a small complex type for FP32 and FP64, and the Philox4x64-10 generator.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sblm {

// ------------------------------------------------------------------------------------------
// complex arithmetic in T = float or double
// ------------------------------------------------------------------------------------------
template <typename T>
struct cx {
    T re, im;
};

template <typename T>
__device__ __forceinline__ cx<T> mk(T a, T b) { return cx<T>{a, b}; }
template <typename T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a) { return {-a.re, -a.im}; }
template <typename T>
__device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T>
__device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return {s * a.re, s * a.im}; }
template <typename T>
__device__ __forceinline__ cx<T> conj(cx<T> a) { return {a.re, -a.im}; }
template <typename T>
__device__ __forceinline__ T norm2(cx<T> a) { return a.re * a.re + a.im * a.im; }

// reciprocal of a positive real. FP32: the hardware approximation (the root iteration corrects
// its own rounding).
__device__ __forceinline__ float rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// FP64: hardware reciprocal approximation (relative error ~1e-6 on sm_103a) and two Newton
// steps r <- r (2 - x r), which square the error each time; the IEEE division is an order of
// magnitude dearer on the FP64 pipe. Zero, infinite and NaN inputs keep the approximation's
// value (inf, 0, NaN).
__device__ __forceinline__ double rcp(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    if (isfinite(r) && r != 0.0) {
        r = r * fma(-x, r, 2.0);
        r = r * fma(-x, r, 2.0);
    }
    return r;
}

__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
__device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }

template <typename T>
__device__ __forceinline__ cx<T> inv(cx<T> a) {
    T r = rcp(norm2(a));
    return {a.re * r, -a.im * r};
}
template <typename T>
__device__ __forceinline__ cx<T> div(cx<T> a, cx<T> b) { return a * inv(b); }

template <typename T>
__device__ __forceinline__ bool finite2(cx<T> a) { return isfinite(a.re) && isfinite(a.im); }

// ------------------------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds; each round multiplies
// words 0 and 2 by the round multipliers into 128-bit products, and the key advances by the
// Weyl constants between rounds.
// ------------------------------------------------------------------------------------------
struct u64x4 {
    uint64_t x[4];
};

__device__ __forceinline__ u64x4 philox4x64(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                            uint64_t k0, uint64_t k1) {
    constexpr uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    constexpr uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += W0;
            k1 += W1;
        }
        const uint64_t lo0 = M0 * c0, hi0 = __umul64hi(M0, c0);
        const uint64_t lo1 = M1 * c2, hi1 = __umul64hi(M1, c2);
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return u64x4{{c0, c1, c2, c3}};
}

// draw conventions: u01 in [0,1) from the top 53 bits, an integer in [0,n) from the top 32 bits,
// and the top bit
__device__ __forceinline__ double u01(uint64_t x) { return (double)(x >> 11) * 0x1.0p-53; }
__device__ __forceinline__ uint32_t uniform_int(uint64_t x, uint32_t n) {
    return (uint32_t)(((x >> 32) * (uint64_t)n) >> 32);
}
__device__ __forceinline__ uint32_t top_bit(uint64_t x) { return (uint32_t)(x >> 63); }

// operator identifiers (Philox counter word 1)
enum : uint64_t {
    OP_INIT_PERM = 1,
    OP_INIT_U = 2,
    OP_SELECT = 3,
    OP_MODE = 4,
    OP_F = 5,
    OP_MUT = 6,
};

}  // namespace sblm
