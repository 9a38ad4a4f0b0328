// cnn_gemm.cuh -- the proposal network's dense contractions on the 5th-generation tensor cores.
//
// One tile kernel computes C[M, N] = sum_k A(m, k) B(k, n) with BF16 operands and FP32
// accumulators held in tensor memory: tcgen05.mma (kind::f16, M = 128, N = 64, K = 16 per
// instruction) issued by one thread, operands read by the tensor core from shared memory through
// matrix descriptors, results brought back with tcgen05.ld for the epilogue. Operands are
// produced by loader functors that return 8 consecutive BF16 values along the operand's
// contiguous dimension, so the convolution's im2col and its adjoint col2im are never
// materialised: the loader gathers the rows straight from the activations. Shared memory holds
// every tile in a no-swizzle core-matrix layout (8 rows x 16 bytes per core matrix): K-major
// operands (forward and input-gradient products) as 8-row groups of BK/8 core matrices along K;
// MN-major operands (weight-gradient products, reductions over batch x position, split over K
// with one FP32 partial per split so the reduction order is fixed) as 8-k groups of core
// matrices along M or N, read with the instruction descriptor's MN-major bit. In both layouts a
// core matrix's 16-byte rows are consecutive, so vector v of a tile lands at byte 16 v and each
// warp stores 512 contiguous bytes (the fetch assigns vectors to threads accordingly). The
// descriptors' leading-dimension offset is the step between core matrices along K, the
// stride-dimension offset the step between them along M or N. Two stages: the global loads of the next K-tile overlap the MMAs of the
// current one, each stage released by an mbarrier that tcgen05.commit arrives on. Every wait is
// bounded; a wait that gives up sets g_tc_timeout, which the host reads after the call. The
// give-up decision is made block-wide (__syncthreads_and) before any barrier or .sync.aligned
// instruction that depends on it: after it no further MMA is issued, the epilogue is skipped, and
// the block waits for the MMAs already issued (one more commit on a drain barrier) before it
// frees its tensor memory.
// The accumulators leave tensor memory through a shared-memory staging tile, so that each warp's
// epilogue covers one whole 64-column row (coalesced). Two tiles are fetched ahead in registers.
// Epilogue functors receive two adjacent columns (m, n), (m, n + 1) per call.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

namespace sblm {
namespace cnn {

constexpr int BM = 128, BN = 64, BK = 32;
constexpr int kGemmThreads = 256;  // 8 warps: warp w reads accumulator rows 32 (w % 4) .. + 31,
                                   // columns 32 (w / 4) .. + 31
constexpr int kStages = 2;
constexpr uint32_t kTileA = BM * BK * 2, kTileB = BN * BK * 2;
constexpr int kEpiLd = BN + 1;  // padded row of the accumulator staging tile (floats)
constexpr size_t kRing = kStages * (kTileA + kTileB);
constexpr size_t kEpiBytes = (size_t)BM * kEpiLd * 4;
constexpr size_t kGemmSmem = (kRing > kEpiBytes ? kRing : kEpiBytes) + 1024;  // + room to align to 1 KB
constexpr uint32_t kTmemCols = 64;                                 // FP32 accumulator columns (= BN)
constexpr int kWaitLimit = 1 << 24;

__device__ int g_tc_timeout;

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

// shared-memory matrix descriptor: start address, leading-dimension byte offset (between core
// matrices along K), stride-dimension byte offset (between 8-row groups), descriptor version 1,
// no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5), BF16 A and B (bits 7-9,
// 10-12), A and B MN-major flags (bits 15, 16), N / 8 at bits 17-22, M / 16 at bits 24-28
__host__ __device__ constexpr uint32_t idesc_f16(bool a_mn, bool b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
           ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, int limit = kWaitLimit) {
    for (int it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    atomicExch(&g_tc_timeout, 1);
    return false;
}

// global -> registers for one tile of ROWS (M or N) x BK. Vector v (8 BF16) is the 16-byte row
// of core matrix v / 8 at position v % 8: K-major, row group v / BK, k chunk (v % BK) / 8, row
// v % 8 of the group; MN-major, k group v / ROWS, m (or n) chunk (v % ROWS) / 8, k row v % 8.
template <bool KMAJ, int ROWS, class L>
__device__ __forceinline__ void tile_fetch(const L& ld, int mn0, int k0, uint4* reg) {
    constexpr int per = ROWS * BK / 8 / kGemmThreads;
#pragma unroll
    for (int i = 0; i < per; ++i) {
        const int v = threadIdx.x + i * kGemmThreads;
        if (KMAJ) {
            const int r = (v / BK) * 8 + (v & 7), c = ((v % BK) >> 3) * 8;
            reg[i] = ld(mn0 + r, k0 + c);
        } else {
            const int kr = (v / ROWS) * 8 + (v & 7), c = ((v % ROWS) >> 3) * 8;
            reg[i] = ld(k0 + kr, mn0 + c);
        }
    }
}

// registers -> the stage's tile: vector v at byte 16 v
template <int ROWS>
__device__ __forceinline__ void tile_store(unsigned char* s, const uint4* reg) {
    constexpr int per = ROWS * BK / 8 / kGemmThreads;
#pragma unroll
    for (int i = 0; i < per; ++i) reinterpret_cast<uint4*>(s)[threadIdx.x + i * kGemmThreads] = reg[i];
}

// matrix descriptor of the 16-k slice ks of a tile: K-major, core matrices along K 128 bytes
// apart and 8-row groups (BK/8) * 128 apart; MN-major, 8-k groups (ROWS/8) * 128 apart and
// core matrices along M or N 128 bytes apart
template <bool KMAJ, int ROWS>
__device__ __forceinline__ uint64_t tile_desc(uint32_t base, int ks) {
    if (KMAJ) return smem_desc(base + (uint32_t)ks * 256, 128, (BK / 8) * 128);
    return smem_desc(base + (uint32_t)ks * 2 * (ROWS / 8) * 128, (ROWS / 8) * 128, 128);
}

// C[M, N] (+ epilogue) over the K-tiles [z * tps, (z + 1) * tps) of split z = blockIdx.z
template <bool AK, bool BKM, class LA, class LB, class EP>
__global__ void __launch_bounds__(kGemmThreads) gemm_kernel(LA la, LB lb, EP ep, int M, int N, int K, int tps) {
    extern __shared__ unsigned char dsmem[];
    __shared__ __align__(8) uint64_t mbar[kStages];
    __shared__ __align__(8) uint64_t mbar_drain;  // completes once every MMA issued so far has (give-up path)
    __shared__ uint32_t s_tmem;
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)dsmem + 1023) & ~(uintptr_t)1023);
    unsigned char* sA[kStages] = {base, base + kTileA + kTileB};
    unsigned char* sB[kStages] = {base + kTileA, base + 2 * kTileA + kTileB};
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int nt = (K + BK - 1) / BK;
    const int t_begin = blockIdx.z * tps, t_end = min(nt, t_begin + tps);

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[s])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar_drain)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;

    constexpr int kPa = BM * BK / 8 / kGemmThreads, kPb = BN * BK / 8 / kGemmThreads;
    uint4 ra[2][kPa], rb[2][kPb];
    uint32_t parity[kStages] = {0u, 0u};
    bool pending[kStages] = {false, false};
    bool ok = true;
    // two tiles in flight in registers: tile t + 2 is fetched while the MMAs of tile t run
    if (t_begin < t_end) {
        tile_fetch<AK, BM>(la, m0, t_begin * BK, ra[0]);
        tile_fetch<BKM, BN>(lb, n0, t_begin * BK, rb[0]);
    }
    if (t_begin + 1 < t_end) {
        tile_fetch<AK, BM>(la, m0, (t_begin + 1) * BK, ra[1]);
        tile_fetch<BKM, BN>(lb, n0, (t_begin + 1) * BK, rb[1]);
    }
    // one K-tile through stage ST (a compile-time index, so the register tiles stay in registers)
    auto step = [&](auto stage, int t) {
        constexpr int st = decltype(stage)::value;
        if (pending[st]) {  // the MMAs that read this stage two tiles ago must be done
            ok = mbar_wait(smem_u32(&mbar[st]), parity[st]) && ok;
            parity[st] ^= 1u;
            pending[st] = false;
        }
        tile_store<BM>(sA[st], ra[st]);
        tile_store<BN>(sB[st], rb[st]);
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        ok = __syncthreads_and(ok) != 0;  // one decision for the block: no MMA is issued after a give-up
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0 && ok) {
            const uint32_t a0 = smem_u32(sA[st]), b0 = smem_u32(sB[st]);
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
                const uint64_t ad = tile_desc<AK, BM>(a0, ks);
                const uint64_t bd = tile_desc<BKM, BN>(b0, ks);
                const uint32_t acc = (t > t_begin || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc_f16(!AK, !BKM)), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar[st])));
        }
        pending[st] = ok;
        if (t + 2 < t_end) {
            tile_fetch<AK, BM>(la, m0, (t + 2) * BK, ra[st]);
            tile_fetch<BKM, BN>(lb, n0, (t + 2) * BK, rb[st]);
        }
    };
    for (int t = t_begin; t < t_end; t += 2) {
        step(std::integral_constant<int, 0>{}, t);
        if (t + 1 < t_end) step(std::integral_constant<int, 1>{}, t + 1);
    }
    for (int s = 0; s < kStages; ++s)
        if (pending[s]) {
            ok = mbar_wait(smem_u32(&mbar[s]), parity[s]) && ok;
            parity[s] ^= 1u;
        }
    asm volatile("tcgen05.fence::before_thread_sync;");
    ok = __syncthreads_and(ok) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!ok) {
        // a wait gave up: the MMAs issued so far may still be running. Track them all with one more
        // commit and wait for it (bounded again) before the tensor memory is freed
        if (tid == 0)
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar_drain)));
        mbar_wait(smem_u32(&mbar_drain), 0u);
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    if (ok && t_end > t_begin) {
        float* sE = reinterpret_cast<float*>(base);  // the tile ring is free: every MMA has completed
        const int q = warp & 3, half = warp >> 2;
#pragma unroll
        for (int h = 0; h < 32; h += 16) {
            uint32_t r[16];
            const int col = half * 32 + h;
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)col;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            float* row = sE + (q * 32 + lane) * kEpiLd + col;
#pragma unroll
            for (int j = 0; j < 16; ++j) row[j] = __uint_as_float(r[j]);
        }
        __syncthreads();
        // a warp covers one row's 32 column pairs
#pragma unroll 4
        for (int p = tid; p < BM * (BN / 2); p += kGemmThreads) {
            const int rr = p / (BN / 2), pc = p % (BN / 2);
            const float* e = sE + rr * kEpiLd + 2 * pc;
            ep(m0 + rr, n0 + 2 * pc, e[0], e[1], blockIdx.z);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
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
