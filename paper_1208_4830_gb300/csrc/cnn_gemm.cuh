// cnn_gemm.cuh -- the proposal network's dense contractions on the tensor cores.
//
// One tile kernel computes C[M, N] = sum_k A(m, k) B(k, n) in BF16 with FP32 accumulation
// (mma.sync m16n8k16). Operands are produced by loader functors that return 8 consecutive BF16
// values along the operand's contiguous dimension, so the convolution's im2col and its adjoint
// col2im are never materialised: the loader gathers the rows straight from the activations.
// Each operand is staged in shared memory in one of two orientations:
//   K-major  (row = m or n, 8 consecutive k)   read with ldmatrix
//   MN-major (row = k, 8 consecutive m or n)   read with ldmatrix.trans
// Forward and input-gradient products are K-major on both sides; weight-gradient products
// (reductions over batch x position) are MN-major on both sides and split over K, each split
// writing its own FP32 partial so the reduction order is fixed.
// Epilogue functors receive two adjacent columns (m, n), (m, n + 1) per call.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace sblm {
namespace cnn {

constexpr int BM = 128, BN = 64, BK = 32;
constexpr int kGemmThreads = 128;  // 4 warps: 2 (m) x 2 (n), 64 x 32 outputs each
constexpr int kPad = 8;            // row padding (elements): conflict-free ldmatrix rows

__device__ __forceinline__ uint32_t pack_bf2(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ uint4 pack8(const float* v) {
    return make_uint4(pack_bf2(v[0], v[1]), pack_bf2(v[2], v[3]), pack_bf2(v[4], v[5]), pack_bf2(v[6], v[7]));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&r)[4]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t (&r)[4]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// shared-memory tile geometry of one operand: `rows_mn` is BM or BN
template <bool KMAJ, int ROWS_MN>
struct TileGeom {
    static constexpr int rows = KMAJ ? ROWS_MN : BK;         // stored rows
    static constexpr int cols = KMAJ ? BK : ROWS_MN;         // stored contiguous extent
    static constexpr int ld = cols + kPad;                   // elements per stored row
    static constexpr int elems = rows * ld;
    static constexpr int vecs = rows * cols / 8;             // 16-byte loads per tile
    static constexpr int vec_per_row = cols / 8;
};

// global -> registers for one tile: vector v covers stored row v / vec_per_row
template <bool KMAJ, int ROWS_MN, class L>
__device__ __forceinline__ void tile_fetch(const L& ld, int mn0, int k0, uint4* reg) {
    using G = TileGeom<KMAJ, ROWS_MN>;
    constexpr int per = G::vecs / kGemmThreads;
#pragma unroll
    for (int i = 0; i < per; ++i) {
        const int v = threadIdx.x + i * kGemmThreads;
        const int r = v / G::vec_per_row, c = (v % G::vec_per_row) * 8;
        reg[i] = KMAJ ? ld(mn0 + r, k0 + c) : ld(k0 + r, mn0 + c);
    }
}

template <bool KMAJ, int ROWS_MN>
__device__ __forceinline__ void tile_store(__nv_bfloat16* s, const uint4* reg) {
    using G = TileGeom<KMAJ, ROWS_MN>;
    constexpr int per = G::vecs / kGemmThreads;
#pragma unroll
    for (int i = 0; i < per; ++i) {
        const int v = threadIdx.x + i * kGemmThreads;
        const int r = v / G::vec_per_row, c = (v % G::vec_per_row) * 8;
        *reinterpret_cast<uint4*>(s + r * G::ld + c) = reg[i];
    }
}

// C[M, N] (+ epilogue) over the K-tiles [z * tps, (z + 1) * tps) of split z = blockIdx.z
template <bool AK, bool BKM, class LA, class LB, class EP>
__global__ void __launch_bounds__(kGemmThreads) gemm_kernel(LA la, LB lb, EP ep, int M, int N, int K, int tps) {
    using GA = TileGeom<AK, BM>;
    using GB = TileGeom<BKM, BN>;
    __shared__ __align__(16) __nv_bfloat16 sA[2][GA::elems];
    __shared__ __align__(16) __nv_bfloat16 sB[2][GB::elems];

    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int nt = (K + BK - 1) / BK;
    const int t_begin = blockIdx.z * tps, t_end = min(nt, t_begin + tps);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = (warp >> 1) * 64, wn = (warp & 1) * 32;

    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

    uint4 ra[GA::vecs / kGemmThreads], rb[GB::vecs / kGemmThreads];
    if (t_begin < t_end) {
        tile_fetch<AK, BM>(la, m0, t_begin * BK, ra);
        tile_fetch<BKM, BN>(lb, n0, t_begin * BK, rb);
        tile_store<AK, BM>(sA[0], ra);
        tile_store<BKM, BN>(sB[0], rb);
    }
    __syncthreads();
    int cur = 0;
    for (int t = t_begin; t < t_end; ++t) {
        const bool more = t + 1 < t_end;
        if (more) {
            tile_fetch<AK, BM>(la, m0, (t + 1) * BK, ra);
            tile_fetch<BKM, BN>(lb, n0, (t + 1) * BK, rb);
        }
        const __nv_bfloat16* A = sA[cur];
        const __nv_bfloat16* B = sB[cur];
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[4][4], bf[4][2];
#pragma unroll
            for (int mi = 0; mi < 4; ++mi) {
                const int mb = wm + mi * 16;
                if constexpr (AK) {
                    const int r = mb + (lane & 7) + ((lane >> 3) & 1) * 8, c = kk + (lane >> 4) * 8;
                    ldsm_x4(smem_u32(A + r * GA::ld + c), af[mi]);
                } else {
                    const int r = kk + (lane & 7) + (lane >> 4) * 8, c = mb + ((lane >> 3) & 1) * 8;
                    ldsm_x4_t(smem_u32(A + r * GA::ld + c), af[mi]);
                }
            }
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const int nb = wn + p * 16;
                uint32_t r4[4];
                if constexpr (BKM) {
                    const int r = nb + (lane & 7) + (lane >> 4) * 8, c = kk + ((lane >> 3) & 1) * 8;
                    ldsm_x4(smem_u32(B + r * GB::ld + c), r4);
                } else {
                    const int r = kk + (lane & 7) + ((lane >> 3) & 1) * 8, c = nb + (lane >> 4) * 8;
                    ldsm_x4_t(smem_u32(B + r * GB::ld + c), r4);
                }
                bf[2 * p][0] = r4[0];
                bf[2 * p][1] = r4[1];
                bf[2 * p + 1][0] = r4[2];
                bf[2 * p + 1][1] = r4[3];
            }
#pragma unroll
            for (int mi = 0; mi < 4; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], af[mi], bf[ni][0], bf[ni][1]);
        }
        if (more) {
            tile_store<AK, BM>(sA[cur ^ 1], ra);
            tile_store<BKM, BN>(sB[cur ^ 1], rb);
        }
        __syncthreads();
        cur ^= 1;
    }
    const int g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) {
            const int m = m0 + wm + mi * 16 + g, n = n0 + wn + ni * 8 + 2 * tq;
            ep(m, n, acc[mi][ni][0], acc[mi][ni][1], blockIdx.z);
            ep(m + 8, n, acc[mi][ni][2], acc[mi][ni][3], blockIdx.z);
        }
}

// ------------------------------------------------------------------------------------------
// loaders: operator()(row, col) returns the 8 values at stored (row, col .. col + 7), zero
// outside the operand
// ------------------------------------------------------------------------------------------

// dense BF16 matrix [rows][ld]; column `ones_col` (if >= cols) reads as 1 on valid rows
struct DenseBF {
    const __nv_bfloat16* p;
    int rows, cols, ld, ones_col;
    __device__ uint4 operator()(int r, int c) const {
        if (r >= rows) return make_uint4(0, 0, 0, 0);
        if (c + 8 <= cols && (ld & 7) == 0) return *reinterpret_cast<const uint4*>(p + (size_t)r * ld + c);
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int e = c + i;
            v[i] = e < cols ? __bfloat162float(p[(size_t)r * ld + e]) : (e == ones_col ? 1.f : 0.f);
        }
        return pack8(v);
    }
};

// dense FP32 matrix [rows][ld], rounded to BF16 on load
struct DenseF32 {
    const float* p;
    int rows, cols, ld;
    __device__ uint4 operator()(int r, int c) const {
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int e = c + i;
            v[i] = (r < rows && e < cols) ? p[(size_t)r * ld + e] : 0.f;
        }
        return pack8(v);
    }
};

// im2col of a [B][L][64] BF16 activation for a kernel-5, pad-2 convolution of stride s:
// row m = b * Lo + l, column k = kk * 64 + c -> h[b][l * s + kk - 2][c]   (K-major A)
struct Im2col {
    const __nv_bfloat16* h;
    int B, L, Lo, s;
    __device__ uint4 operator()(int m, int k) const {
        if (m >= B * Lo || k >= 5 * 64) return make_uint4(0, 0, 0, 0);
        const int b = m / Lo, l = m - b * Lo, kk = k >> 6, c = k & 63;
        const int i = l * s + kk - 2;
        if (i < 0 || i >= L) return make_uint4(0, 0, 0, 0);
        return *reinterpret_cast<const uint4*>(h + ((size_t)b * L + i) * 64 + c);
    }
};

// the same gather stored MN-major for the weight gradient: row = b * Lo + l, column m = kk * 64 + c,
// and column 320 reads as 1 (the bias row of the gradient)
struct Im2colT {
    const __nv_bfloat16* h;
    int B, L, Lo, s;
    __device__ uint4 operator()(int r, int m) const {
        if (r >= B * Lo || m > 5 * 64) return make_uint4(0, 0, 0, 0);
        if (m == 5 * 64) return make_uint4(pack_bf2(1.f, 0.f), 0, 0, 0);
        const int b = r / Lo, l = r - b * Lo, kk = m >> 6, c = m & 63;
        const int i = l * s + kk - 2;
        if (i < 0 || i >= L) return make_uint4(0, 0, 0, 0);
        return *reinterpret_cast<const uint4*>(h + ((size_t)b * L + i) * 64 + c);
    }
};

// im2col of the FP32 network input [B][256][2] for the first (stride-1) convolution:
// row m = b * 256 + l, column k = kk * 2 + c < 10   (K-major A)
struct InputIm2col {
    const float* x;
    int B;
    __device__ uint4 operator()(int m, int k) const {
        float v[8];
        const int b = m >> 8, l = m & 255;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int e = k + i, kk = e >> 1, c = e & 1, j = l + kk - 2;
            v[i] = (m < B * 256 && e < 10 && j >= 0 && j < 256) ? x[((size_t)b * 256 + j) * 2 + c] : 0.f;
        }
        return pack8(v);
    }
};

// MN-major twin for the first layer's weight gradient; column 10 reads as 1
struct InputIm2colT {
    const float* x;
    int B;
    __device__ uint4 operator()(int r, int m) const {
        float v[8];
        const int b = r >> 8, l = r & 255;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int e = m + i, kk = e >> 1, c = e & 1, j = l + kk - 2;
            float val = 0.f;
            if (r < B * 256) {
                if (e < 10) val = (j >= 0 && j < 256) ? x[((size_t)b * 256 + j) * 2 + c] : 0.f;
                else if (e == 10) val = 1.f;
            }
            v[i] = val;
        }
        return pack8(v);
    }
};

// col2im as a gather, for the input gradient of a convolution with output gradient dz [B][Lo][64]:
// row m = b * L + i (input position), column k = kk * 64 + o ->
// dz[b][(i + 2 - kk) / s][o] when s divides i + 2 - kk and the quotient is inside [0, Lo)
struct Col2im {
    const __nv_bfloat16* dz;
    int B, L, Lo, s;
    __device__ uint4 operator()(int m, int k) const {
        if (m >= B * L || k >= 5 * 64) return make_uint4(0, 0, 0, 0);
        const int b = m / L, i = m - b * L, kk = k >> 6, o = k & 63;
        const int num = i + 2 - kk;
        if (num < 0 || num % s) return make_uint4(0, 0, 0, 0);
        const int l = num / s;
        if (l >= Lo) return make_uint4(0, 0, 0, 0);
        return *reinterpret_cast<const uint4*>(dz + ((size_t)b * Lo + l) * 64 + o);
    }
};

// a convolution weight W [(kk * 64 + c)][o] read as the K-major B of the input gradient:
// stored row n = c, column k = kk * 64 + o
struct ConvWT {
    const __nv_bfloat16* w;
    __device__ uint4 operator()(int n, int k) const {
        if (n >= 64 || k >= 5 * 64) return make_uint4(0, 0, 0, 0);
        const int kk = k >> 6, o = k & 63;
        return *reinterpret_cast<const uint4*>(w + ((size_t)kk * 64 + n) * 64 + o);
    }
};

}  // namespace cnn
}  // namespace sblm
