// tcgen05 BF16 GEMM with chunked accumulation:
//     C = alpha * rowscale .* (sum_a A_a) B^T + beta * X1 + gamma * X2
// (A_a: M x K, a < NA, B: N x K, all K-major BF16; C, X1, X2 M x N FP32).
//
// Why chunks.  The tensor core adds each 16-deep MMA into its FP32
// accumulator with a rounding that drops up to an ulp of the running sum and
// always in one direction, so a long K loop shrinks every output by about
// (number of MMAs) x 2^-24 relative: 5e-5 for a 48374-deep sketch, which moves
// the STR spectrum by 1e-4.  Here the K loop is cut into chunks of CH k-steps
// (CH x 64 columns): each chunk accumulates in one of two tensor-memory
// buffers while the epilogue warps add the other buffer's finished partial
// into FP32 registers with round-to-nearest, so the one-sided error is that
// of one chunk (16 MMAs at CH = 4: about 5e-7 relative) and the sum of the
// chunk partials is unbiased.
//
// Roles (one CTA per 128 x BN tile, BN = 128 G):
//   warp 0, one thread : TMA producer -- NA A boxes (128 x 64) and one B box
//                        (BN x 64) per stage, S-stage mbarrier ring;
//   warp 1, one thread : MMA issuer -- chunk c into tensor-memory buffer
//                        c & 1 (BN columns each), tcgen05.commit after each
//                        stage (frees it) and after each chunk (hands the
//                        buffer to the epilogue);
//   warps 2 .. 2+4G-1  : epilogue -- warp w reads TMEM lanes 32 (w % 4) ..
//                        +31 (tile rows) and column group g = (w - 2) / 4
//                        (128 columns), keeping 128 FP32 running sums per
//                        thread; it frees the buffer for the chunk after next.
// Every mbarrier wait is bounded (2 s); a timeout records a code in the
// translation unit's g_gemm_err and the CTA winds down.
#pragma once

#include <cooperative_groups.h>

#include "gemm.cuh"

namespace mv {

constexpr int kChunkSteps = 4;          // k-steps of 64 per accumulation chunk

template <int BN, int NA>
struct GemmChunkCfg {
    static constexpr int G = BN / 128;                       // column groups of 128
    static constexpr int EPI_WARPS = 4 * G;
    static constexpr int THREADS = 64 + 32 * EPI_WARPS;
    static constexpr uint32_t A_BYTES = kBM * kBK * 2;
    static constexpr uint32_t B_BYTES = BN * kBK * 2;
    static constexpr uint32_t STAGE = NA * A_BYTES + B_BYTES;
    static constexpr int S = (int)((196608u / STAGE) < 8u ? (196608u / STAGE) : 8u);
    static constexpr int NBAR = 2 * S + 4;                   // full[S], empty[S], tfull[2], tempty[2]
    static constexpr size_t SMEM = 1024 + (size_t)S * STAGE + NBAR * 8 + 16;
    static constexpr uint32_t TMEM_COLS = 2 * BN;
};

// The epilogue of the chunked GEMM.
struct GemmEpi {
    float alpha = 1.0f;
    const float *X1 = nullptr;          // C += beta X1 (may alias C)
    int64_t ld1 = 0;
    float beta = 0.0f;
    const float *X2 = nullptr;          // C += gamma X2
    int64_t ld2 = 0;
    float gamma = 0.0f;
    const float *rscale = nullptr;      // row i of the product scaled by rscale[i]
};

// Epilogue store of one tile row: 128 columns from cb of the FP32 running
// sums acc, C[row][cb + j] = alpha rowscale[row] acc[j] + beta X1 + gamma X2.
__device__ __forceinline__ void chunk_store(const float (&acc)[128], int row, int cb, int N, float *__restrict__ C,
                                            int64_t ldc, const GemmEpi &e) {
    const float sc = e.rscale ? e.rscale[row] * e.alpha : e.alpha;
    float *crow = C + (int64_t)row * ldc;
    const float *x1 = e.X1 ? e.X1 + (int64_t)row * e.ld1 : nullptr;
    const float *x2 = e.X2 ? e.X2 + (int64_t)row * e.ld2 : nullptr;
    const bool vec = (ldc & 3) == 0 && (reinterpret_cast<uintptr_t>(C) & 15) == 0 &&
                     (!x1 || ((e.ld1 & 3) == 0 && (reinterpret_cast<uintptr_t>(e.X1) & 15) == 0)) &&
                     (!x2 || ((e.ld2 & 3) == 0 && (reinterpret_cast<uintptr_t>(e.X2) & 15) == 0));
#pragma unroll
    for (int qq = 0; qq < 32; ++qq) {
        const int col = cb + 4 * qq;
        if (vec && col + 4 <= N) {
            float4 v = make_float4(sc * acc[4 * qq], sc * acc[4 * qq + 1], sc * acc[4 * qq + 2],
                                   sc * acc[4 * qq + 3]);
            if (x1) {
                const float4 w = *reinterpret_cast<const float4 *>(x1 + col);
                v.x = fmaf(e.beta, w.x, v.x);
                v.y = fmaf(e.beta, w.y, v.y);
                v.z = fmaf(e.beta, w.z, v.z);
                v.w = fmaf(e.beta, w.w, v.w);
            }
            if (x2) {
                const float4 w = *reinterpret_cast<const float4 *>(x2 + col);
                v.x = fmaf(e.gamma, w.x, v.x);
                v.y = fmaf(e.gamma, w.y, v.y);
                v.z = fmaf(e.gamma, w.z, v.z);
                v.w = fmaf(e.gamma, w.w, v.w);
            }
            *reinterpret_cast<float4 *>(crow + col) = v;
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (col + u >= N) break;
                float v = sc * acc[4 * qq + u];
                if (x1) v = fmaf(e.beta, x1[col + u], v);
                if (x2) v = fmaf(e.gamma, x2[col + u], v);
                crow[col + u] = v;
            }
        }
    }
}

template <int BN, int NA>
__global__ void __launch_bounds__(GemmChunkCfg<BN, NA>::THREADS, 1)
gemm_chunk_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  const __grid_constant__ CUtensorMap tmA2, float *__restrict__ C, int M, int N, int K, int64_t ldc,
                  GemmEpi e, int raster) {
    using Cfg = GemmChunkCfg<BN, NA>;
    constexpr int S = Cfg::S;
    constexpr int CH = kChunkSteps;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;                        // stage s, operand a at sA + (s NA + a) A_BYTES
    uint8_t *sB = smem + S * NA * Cfg::A_BYTES;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + S * Cfg::STAGE);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + Cfg::NBAR);
    const uint32_t full0 = umma::smem_u32(bars), empty0 = umma::smem_u32(bars + S);
    const uint32_t tfull0 = umma::smem_u32(bars + 2 * S), tempty0 = umma::smem_u32(bars + 2 * S + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int rt = blockIdx.x, ct = blockIdx.y;
    if (raster && (int)gridDim.x > kRasterRows) {        // grouped raster (see gemm.cuh)
        const int nrt = (int)gridDim.x, nct = (int)gridDim.y;
        const int lin = (int)blockIdx.x + nrt * (int)blockIdx.y;
        const int per = kRasterRows * nct, g = lin / per, first = g * kRasterRows;
        const int gh = min(nrt - first, kRasterRows), rem = lin - g * per;
        rt = first + rem % gh;
        ct = rem / gh;
    }
    const int m0 = rt * kBM, n0 = ct * BN;
    const int nk = (K + kBK - 1) / kBK;
    const int nch = (nk + CH - 1) / CH;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            umma::mbar_init(full0 + 8 * s, 1);
            umma::mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            umma::mbar_init(tfull0 + 8 * b, 1);
            umma::mbar_init(tempty0 + 8 * b, Cfg::EPI_WARPS);
        }
        umma::mbar_fence_init();
    }
    if (warp == 1) {
        umma::tmem_alloc(umma::smem_u32(tmem_slot), Cfg::TMEM_COLS);
        umma::tmem_relinquish();
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            umma::prefetch_tensormap(&tmA);
            umma::prefetch_tensormap(&tmB);
            if (NA > 1) umma::prefetch_tensormap(&tmA2);
            for (int kt = 0; kt < nk; ++kt) {
                const int s = kt % S;
                const uint32_t ph = (uint32_t)(kt / S) & 1u;
                if (!umma::mbar_wait(empty0 + 8 * s, ph ^ 1u, kWaitNs)) {
                    atomicExch(&g_gemm_err, 11);
                    break;
                }
                umma::mbar_arrive_expect_tx(full0 + 8 * s, Cfg::STAGE);
                umma::tma_load_2d(umma::smem_u32(sA + s * NA * Cfg::A_BYTES), &tmA, kt * kBK, m0, full0 + 8 * s);
                if (NA > 1)
                    umma::tma_load_2d(umma::smem_u32(sA + (s * NA + 1) * Cfg::A_BYTES), &tmA2, kt * kBK, m0,
                                      full0 + 8 * s);
                umma::tma_load_2d(umma::smem_u32(sB + s * Cfg::B_BYTES), &tmB, kt * kBK, n0, full0 + 8 * s);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = umma::idesc_bf16_f32(kBM, BN);
            for (int kt = 0; kt < nk; ++kt) {
                const int c = kt / CH, j = kt - c * CH, b = c & 1;
                if (j == 0 && c >= 2) {            // buffer b must have been drained (chunk c - 2)
                    if (!umma::mbar_wait(tempty0 + 8 * b, (uint32_t)((c >> 1) - 1) & 1u, 2 * kWaitNs)) {
                        atomicExch(&g_gemm_err, 12);
                        break;
                    }
                    umma::fence_after_sync();
                }
                const int s = kt % S;
                const uint32_t ph = (uint32_t)(kt / S) & 1u;
                if (!umma::mbar_wait(full0 + 8 * s, ph, kWaitNs)) {
                    atomicExch(&g_gemm_err, 13);
                    break;
                }
                umma::fence_after_sync();
                const uint32_t dst = tmem + (uint32_t)(b * BN);
                const uint64_t db = umma::desc_kmajor_sw128(umma::smem_u32(sB + s * Cfg::B_BYTES));
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    const uint64_t da = umma::desc_kmajor_sw128(umma::smem_u32(sA + (s * NA + a) * Cfg::A_BYTES));
#pragma unroll
                    for (int k = 0; k < kBK / 16; ++k)
                        umma::mma_bf16(dst, da + 2 * k, db + 2 * k, idesc, (j | k | a) != 0 ? 1u : 0u);
                }
                umma::mma_commit(empty0 + 8 * s);
                if (j == CH - 1 || kt == nk - 1) umma::mma_commit(tfull0 + 8 * b);
            }
        }
        __syncwarp();
    } else {
        // Epilogue warp: rows 32 q .. 32 q + 31 of the tile, columns g 128 .. g 128 + 127.
        const int q = warp & 3, g = (warp - 2) >> 2;
        const int row = m0 + 32 * q + lane;
        float acc[128];
#pragma unroll
        for (int i = 0; i < 128; ++i) acc[i] = 0.0f;
        bool ok = true;
        for (int c = 0; c < nch; ++c) {
            const int b = c & 1;
            if (!umma::mbar_wait(tfull0 + 8 * b, (uint32_t)(c >> 1) & 1u, 4 * kWaitNs)) {
                ok = false;
                break;
            }
            umma::fence_after_sync();
            const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * BN + g * 128);
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                uint32_t r[32];
                umma::tmem_ld_32x32b_x32(ta + (uint32_t)(qq * 32), r);
                umma::tmem_ld_wait();
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) acc[qq * 32 + jj] += __uint_as_float(r[jj]);
            }
            umma::fence_before_sync();
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(tempty0 + 8 * b);
        }
        if (!ok) {
            if (lane == 0) atomicExch(&g_gemm_err, 14);
        } else if (row < M) {
            chunk_store(acc, row, n0 + g * 128, N, C, ldc, e);
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (warp == 1) umma::tmem_dealloc(tmem, Cfg::TMEM_COLS);
}

// ------------------------------------------------------------------ CTA-pair form
// The same product on 256 x 256 tiles, each run by a pair of CTAs (a cluster
// of 2) with cta_group::2 MMAs: CTA r of the pair loads rows 128 r .. of the
// A tile and rows 128 r .. of the B tile (half of it), rank 0 issues the
// 256 x 256 x 16 MMAs over both CTAs' shared memory, and each CTA's tensor
// memory accumulates its own 128 rows x 256 columns.  Per CTA and k-step
// that is 32 KB of operands for 128 x 256 x 64 multiply-adds, against 48 KB
// for the one-CTA 128 x 256 tile: a third fewer L2 -> SM bytes per MMA.
// Barriers: rank 0's full[s] counts both CTAs' bytes (the peer's TMA
// completes on it); a multicast commit frees stage s in both CTAs and hands
// buffer b to both epilogues; both CTAs' epilogue warps arrive on rank 0's
// tempty[b].  A cluster barrier opens and closes the kernel, so no CTA
// addresses a peer that has not started or has already left.
template <int NA>
struct GemmPairCfg {
    static constexpr int BN = 256;                           // columns of the pair's tile
    static constexpr int EPI_WARPS = 8;                      // 128 rows x 2 column groups
    static constexpr int THREADS = 64 + 32 * EPI_WARPS;
    static constexpr uint32_t A_BYTES = kBM * kBK * 2;       // this CTA's 128 rows
    static constexpr uint32_t B_BYTES = (BN / 2) * kBK * 2;  // this CTA's half of B
    static constexpr uint32_t STAGE = NA * A_BYTES + B_BYTES;
    static constexpr uint32_t BUDGET = 196608u;               // 192 KB of stages (7 measured the same)
    static constexpr int S = (int)((BUDGET / STAGE) < 8u ? (BUDGET / STAGE) : 8u);
    static constexpr int NBAR = 2 * S + 4;
    static constexpr size_t SMEM = 1024 + (size_t)S * STAGE + NBAR * 8 + 16;
    static constexpr uint32_t TMEM_COLS = 2 * BN;
};
static_assert(GemmPairCfg<1>::SMEM <= 232448 && GemmPairCfg<2>::SMEM <= 232448, "pair GEMM exceeds 227 KB");

template <int NA>
__global__ void __launch_bounds__(GemmPairCfg<NA>::THREADS, 1)
gemm_chunk_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                       const __grid_constant__ CUtensorMap tmA2, float *__restrict__ C, int M, int N, int K,
                       int64_t ldc, GemmEpi e, int raster) {
    using Cfg = GemmPairCfg<NA>;
    constexpr int S = Cfg::S;
    constexpr int CH = kChunkSteps;
    constexpr int BN = Cfg::BN;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;
    uint8_t *sB = smem + S * NA * Cfg::A_BYTES;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + S * Cfg::STAGE);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + Cfg::NBAR);
    const uint32_t full0 = umma::smem_u32(bars), empty0 = umma::smem_u32(bars + S);
    const uint32_t tfull0 = umma::smem_u32(bars + 2 * S), tempty0 = umma::smem_u32(bars + 2 * S + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = umma::cluster_ctarank();            // 0: issues the MMAs
    // the pair's tile (pr, ct); grouped raster over pairs as in gemm.cuh
    const int npr = (int)gridDim.x >> 1, nct = (int)gridDim.y;
    int pr = (int)blockIdx.x >> 1, ct = (int)blockIdx.y;
    if (raster && npr > kRasterRows / 2) {
        const int rows = kRasterRows / 2;
        const int lin = pr + npr * (int)blockIdx.y;
        const int per = rows * nct, g = lin / per, first = g * rows;
        const int gh = min(npr - first, rows), rem = lin - g * per;
        pr = first + rem % gh;
        ct = rem / gh;
    }
    const int m0 = (2 * pr + (int)rank) * kBM;                // this CTA's rows of A and of D
    const int n0 = ct * BN;                                    // the pair's columns
    const int nb0 = n0 + (int)rank * (BN / 2);                 // this CTA's half of B
    const int nk = (K + kBK - 1) / kBK;
    const int nch = (nk + CH - 1) / CH;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            umma::mbar_init(full0 + 8 * s, 1);
            umma::mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            umma::mbar_init(tfull0 + 8 * b, 1);
            umma::mbar_init(tempty0 + 8 * b, 2 * Cfg::EPI_WARPS);
        }
        umma::mbar_fence_init();
    }
    if (warp == 1) {
        umma::tmem_alloc_pair(umma::smem_u32(tmem_slot), Cfg::TMEM_COLS);
        umma::tmem_relinquish_pair();
    }
    umma::fence_before_sync();
    cooperative_groups::this_cluster().sync();                                 // both CTAs' barriers exist
    umma::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t full_r0 = umma::mapa_rank(full0, 0);         // rank 0's full[0], cluster address

    if (warp == 0) {
        if (lane == 0) {
            umma::prefetch_tensormap(&tmA);
            umma::prefetch_tensormap(&tmB);
            if (NA > 1) umma::prefetch_tensormap(&tmA2);
            for (int kt = 0; kt < nk; ++kt) {
                const int s = kt % S;
                const uint32_t ph = (uint32_t)(kt / S) & 1u;
                if (!umma::mbar_wait(empty0 + 8 * s, ph ^ 1u, kWaitNs)) {
                    atomicExch(&g_gemm_err, 21);
                    break;
                }
                const uint32_t fb = full_r0 + 8u * (uint32_t)s;
                if (rank == 0) umma::mbar_arrive_expect_tx(full0 + 8 * s, 2 * Cfg::STAGE);
                umma::tma_load_2d_pair(umma::smem_u32(sA + s * NA * Cfg::A_BYTES), &tmA, kt * kBK, m0, fb);
                if (NA > 1)
                    umma::tma_load_2d_pair(umma::smem_u32(sA + (s * NA + 1) * Cfg::A_BYTES), &tmA2, kt * kBK, m0,
                                           fb);
                umma::tma_load_2d_pair(umma::smem_u32(sB + s * Cfg::B_BYTES), &tmB, kt * kBK, nb0, fb);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {
            constexpr uint32_t idesc = umma::idesc_bf16_f32(2 * kBM, BN);
            for (int kt = 0; kt < nk; ++kt) {
                const int c = kt / CH, j = kt - c * CH, b = c & 1;
                if (j == 0 && c >= 2) {            // buffer b drained by both epilogues (chunk c - 2)
                    if (!umma::mbar_wait(tempty0 + 8 * b, (uint32_t)((c >> 1) - 1) & 1u, 2 * kWaitNs)) {
                        atomicExch(&g_gemm_err, 22);
                        break;
                    }
                    umma::fence_after_sync();
                }
                const int s = kt % S;
                const uint32_t ph = (uint32_t)(kt / S) & 1u;
                if (!umma::mbar_wait(full0 + 8 * s, ph, kWaitNs)) {
                    atomicExch(&g_gemm_err, 23);
                    break;
                }
                umma::fence_after_sync();
                const uint32_t dst = tmem + (uint32_t)(b * BN);
                const uint64_t db = umma::desc_kmajor_sw128(umma::smem_u32(sB + s * Cfg::B_BYTES));
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    const uint64_t da = umma::desc_kmajor_sw128(umma::smem_u32(sA + (s * NA + a) * Cfg::A_BYTES));
#pragma unroll
                    for (int k = 0; k < kBK / 16; ++k)
                        umma::mma_bf16_pair(dst, da + 2 * k, db + 2 * k, idesc, (j | k | a) != 0 ? 1u : 0u);
                }
                umma::mma_commit_pair(empty0 + 8 * s, (uint16_t)3);
                if (j == CH - 1 || kt == nk - 1) umma::mma_commit_pair(tfull0 + 8 * b, (uint16_t)3);
            }
        }
        __syncwarp();
    } else {
        const int q = warp & 3, g = (warp - 2) >> 2;
        const int row = m0 + 32 * q + lane;
        const uint32_t tempty_r0 = umma::mapa_rank(tempty0, 0);
        float acc[128];
#pragma unroll
        for (int i = 0; i < 128; ++i) acc[i] = 0.0f;
        bool ok = true;
        for (int c = 0; c < nch; ++c) {
            const int b = c & 1;
            if (!umma::mbar_wait(tfull0 + 8 * b, (uint32_t)(c >> 1) & 1u, 4 * kWaitNs)) {
                ok = false;
                break;
            }
            umma::fence_after_sync();
            const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * BN + g * 128);
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                uint32_t r[32];
                umma::tmem_ld_32x32b_x32(ta + (uint32_t)(qq * 32), r);
                umma::tmem_ld_wait();
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) acc[qq * 32 + jj] += __uint_as_float(r[jj]);
            }
            umma::fence_before_sync();
            __syncwarp();
            if (lane == 0) umma::mbar_arrive_cluster(tempty_r0 + 8u * (uint32_t)b);
        }
        if (!ok) {
            if (lane == 0) atomicExch(&g_gemm_err, 24);
        } else if (row < M) {
            chunk_store(acc, row, n0 + g * 128, N, C, ldc, e);
        }
    }
    umma::fence_before_sync();
    cooperative_groups::this_cluster().sync();                                 // the peer no longer reads or signals us
    umma::fence_after_sync();
    if (warp == 1) umma::tmem_dealloc_pair(tmem, Cfg::TMEM_COLS);
}

// Row-wise three-piece split (the non-transposed companion of split3_t_kernel
// in gemm.cuh): out[r][seg W + c] = piece(seg) of X[r][c] for c < cols, zero
// for cols <= c < W; out is R x 6W BF16 (row pitch ldo), X is R x cols FP32.
static __global__ void __launch_bounds__(256) split3_rows_kernel(const float *__restrict__ X, int R, int cols,
                                                                 int64_t ldx, int W, int side,
                                                                 __nv_bfloat16 *__restrict__ out, int64_t ldo) {
    const int64_t total = (int64_t)R * W;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / W), c = (int)(idx - (int64_t)r * W);
        const float x = c < cols ? X[(int64_t)r * ldx + c] : 0.0f;
        __nv_bfloat16 *o = out + (int64_t)r * ldo + c;
#pragma unroll
        for (int seg = 0; seg < kSplit3; ++seg) o[(int64_t)seg * W] = split3_get(x, split3_piece(side, seg));
    }
}

// ------------------------------------------------------------------ host
template <int BN, int NA>
static int gemmc_set_attrs() {
    static int st = -1;
    if (st < 0)
        st = cudaFuncSetAttribute(gemm_chunk_kernel<BN, NA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)GemmChunkCfg<BN, NA>::SMEM) == cudaSuccess
                 ? MV_OK
                 : record_message(MV_ERR_CUDA, "chunked GEMM: shared-memory attribute refused");
    return st;
}

// Enqueue C = epilogue(A B^T) with prebuilt tensor maps (capturable; K >= 1).
template <int BN, int NA>
static void gemmc_launch(const CUtensorMap &ta, const CUtensorMap &tb, const CUtensorMap *ta2, int64_t M, int64_t N,
                         int64_t K, float *C, int64_t ldc, const GemmEpi &e, cudaStream_t s, int raster = 1) {
    using Cfg = GemmChunkCfg<BN, NA>;
    dim3 grid((unsigned)((M + kBM - 1) / kBM), (unsigned)((N + BN - 1) / BN));
    gemm_chunk_kernel<BN, NA><<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(ta, tb, ta2 ? *ta2 : ta, C, (int)M, (int)N,
                                                                    (int)K, ldc, e, raster);
}

template <int NA>
static int gemmc_pair_set_attrs() {
    static int st = -1;
    if (st < 0)
        st = cudaFuncSetAttribute(gemm_chunk_pair_kernel<NA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)GemmPairCfg<NA>::SMEM) == cudaSuccess
                 ? MV_OK
                 : record_message(MV_ERR_CUDA, "chunked pair GEMM: shared-memory attribute refused");
    return st;
}

// gemmc<256> on CTA pairs (256 x 256 tiles; clusters of 2 along M).  Tensor
// maps: A boxes of 128 rows, B boxes of 128 rows (half a tile).
static int gemmc_pair(const void *A, const void *A2, int64_t M, int64_t lda, const void *B, int64_t N, int64_t ldb,
                      int64_t K, float *C, int64_t ldc, const GemmEpi &e, cudaStream_t s, int raster = 1) {
    if (K < 1) return record_message(MV_ERR_INVALID_ARG, "chunked GEMM: K must be >= 1");
    CUtensorMap ta, tb, ta2;
    MV_TRY(make_map_bf16(&ta, A, M, K, lda, kBM));
    MV_TRY(make_map_bf16(&tb, B, N, K, ldb, 128));
    if (A2) MV_TRY(make_map_bf16(&ta2, A2, M, K, lda, kBM));
    const unsigned pairs = (unsigned)((M + 2 * kBM - 1) / (2 * kBM));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * pairs, (unsigned)((N + 255) / 256));
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t err;
    if (A2) {
        MV_TRY(gemmc_pair_set_attrs<2>());
        cfg.blockDim = dim3(GemmPairCfg<2>::THREADS);
        cfg.dynamicSmemBytes = GemmPairCfg<2>::SMEM;
        err = cudaLaunchKernelEx(&cfg, gemm_chunk_pair_kernel<2>, ta, tb, ta2, C, (int)M, (int)N, (int)K, ldc, e,
                                 raster);
    } else {
        MV_TRY(gemmc_pair_set_attrs<1>());
        cfg.blockDim = dim3(GemmPairCfg<1>::THREADS);
        cfg.dynamicSmemBytes = GemmPairCfg<1>::SMEM;
        err = cudaLaunchKernelEx(&cfg, gemm_chunk_pair_kernel<1>, ta, tb, ta, C, (int)M, (int)N, (int)K, ldc, e,
                                 raster);
    }
    if (err != cudaSuccess) return record_cuda_error(err, "chunked pair GEMM launch", __FILE__, __LINE__);
    return MV_OK;
}

// 256-column tiles run on CTA pairs.
constexpr bool kChunkPairs = true;

// Tensor maps + launch, no synchronisation.  A2 non-NULL: (A + A2) B^T.
// BN = 256 takes the CTA-pair kernel (kChunkPairs).
template <int BN>
static int gemmc(const void *A, const void *A2, int64_t M, int64_t lda, const void *B, int64_t N, int64_t ldb,
                 int64_t K, float *C, int64_t ldc, const GemmEpi &e, cudaStream_t s, int raster = 1) {
    if (K < 1) return record_message(MV_ERR_INVALID_ARG, "chunked GEMM: K must be >= 1");
    if constexpr (BN == 256 && kChunkPairs) {
        return gemmc_pair(A, A2, M, lda, B, N, ldb, K, C, ldc, e, s, raster);
    } else {
        CUtensorMap ta, tb, ta2;
        MV_TRY(make_map_bf16(&ta, A, M, K, lda, kBM));
        MV_TRY(make_map_bf16(&tb, B, N, K, ldb, BN));
        if (A2) {
            MV_TRY(make_map_bf16(&ta2, A2, M, K, lda, kBM));
            MV_TRY((gemmc_set_attrs<BN, 2>()));
            gemmc_launch<BN, 2>(ta, tb, &ta2, M, N, K, C, ldc, e, s, raster);
        } else {
            MV_TRY((gemmc_set_attrs<BN, 1>()));
            gemmc_launch<BN, 1>(ta, tb, nullptr, M, N, K, C, ldc, e, s, raster);
        }
        MV_CUDA_TRY(cudaGetLastError());
        return MV_OK;
    }
}

// The translation unit's GEMM error word: clear before, read after (blocking).
static int gemm_err_clear(cudaStream_t s) {
    int zero = 0;
    MV_CUDA_TRY(cudaMemcpyToSymbolAsync(g_gemm_err, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    return MV_OK;
}
static int gemm_err_check(cudaStream_t s, const char *what) {
    int err = 0;
    MV_CUDA_TRY(cudaMemcpyFromSymbolAsync(&err, g_gemm_err, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    MV_CUDA_TRY(cudaStreamSynchronize(s));
    if (err != 0) {
        char msg[128];
        snprintf(msg, sizeof(msg), "%s: tcgen05 pipeline wait timed out (stage code %d)", what, err);
        return record_message(MV_ERR_TIMEOUT, msg);
    }
    return MV_OK;
}

}  // namespace mv
