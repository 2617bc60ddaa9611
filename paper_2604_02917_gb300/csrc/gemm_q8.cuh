// tcgen05 GEMM  C = A B^T  with A stored as FP8 e4m3 (K-major) and B as BF16
// (K-major); FP32 accumulation in tensor memory.  tcgen05.mma has no mixed
// FP8 x BF16 kind, so A is brought in by TMA as FP8 (half the bytes of BF16)
// and expanded in shared memory: e4m3 values are exact in BF16, so the
// product equals the BF16 GEMM on the dequantised A.  Used by the frontier
// solve on an FP8 factor (the row scales are folded into the B operand or
// applied by the consumer of C).
//
// One CTA computes a 128 x BN tile with a K loop in steps of 64:
//   warp 0, one thread : TMA producer -- 128x64 FP8 A box (no swizzle) and
//                        BNx64 BF16 B box (128-byte swizzle) per stage;
//   warps 6..9         : converters -- thread r expands row r of the FP8
//                        box into the 128-byte-swizzled BF16 layout the MMA
//                        descriptor expects, fences it for the async proxy
//                        and arrives on the stage's `conv` barrier;
//   warp 1, one thread : MMA issuer -- waits `conv`, four 128xBNx16 MMAs,
//                        tcgen05.commit frees the stage;
//   warps 2..5         : epilogue (as gemm.cuh).
// Every wait is bounded; a timeout records a code in g_gemm_err.
#pragma once

#include "gemm.cuh"

namespace mv {

constexpr int kQ8Threads = 320;

template <int BN>
struct Q8Cfg {
    static constexpr uint32_t A16_BYTES = kBM * kBK * 2;       // 16 KB, 1024-aligned
    static constexpr uint32_t B_BYTES = BN * kBK * 2;
    static constexpr uint32_t A8_BYTES = kBM * kBK;            // 8 KB
    static constexpr int S = (BN >= 256) ? 3 : (BN >= 128 ? 5 : 6);
    static constexpr size_t SMEM = 1024 + (size_t)S * (A16_BYTES + B_BYTES + A8_BYTES) + (3 * S + 1) * 8 + 16;
};

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_local(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

template <int BN, int EPI>
__global__ void __launch_bounds__(kQ8Threads, 1)
gemm_q8_tn_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, float *__restrict__ C,
                  int M, int N, int K, int64_t ldc, __nv_bfloat16 *__restrict__ Ct, int64_t ldct,
                  float *__restrict__ Cpart = nullptr, unsigned *__restrict__ tickets = nullptr) {
    using Cfg = Q8Cfg<BN>;
    constexpr int S = Cfg::S;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // aligned up to 1024 bytes by pointer arithmetic on the shared array (an
    // integer round trip would hide from the compiler that it is shared memory)
    uint8_t *smem = smem_raw + ((1024u - (uint32_t)(reinterpret_cast<uintptr_t>(smem_raw) & 1023u)) & 1023u);
    uint8_t *sA = smem;                                        // S x A16
    uint8_t *sB = sA + S * Cfg::A16_BYTES;                     // S x B
    uint8_t *sA8 = sB + S * Cfg::B_BYTES;                      // S x A8
    uint64_t *bars = reinterpret_cast<uint64_t *>(sA8 + S * Cfg::A8_BYTES);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 3 * S + 1);
    const uint32_t full0 = umma::smem_u32(bars), conv0 = umma::smem_u32(bars + S),
                   empty0 = umma::smem_u32(bars + 2 * S), accum = umma::smem_u32(bars + 3 * S);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    const int nk_all = (K + kBK - 1) / kBK, Z = gridDim.z;   // split-K as in gemm.cuh
    const int kb = (int)((int64_t)blockIdx.z * nk_all / Z), ke = (int)((int64_t)(blockIdx.z + 1) * nk_all / Z);
    const int nk = ke - kb;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            umma::mbar_init(full0 + 8 * s, 1);
            umma::mbar_init(conv0 + 8 * s, 128);
            umma::mbar_init(empty0 + 8 * s, 1);
        }
        umma::mbar_init(accum, 1);
        umma::mbar_fence_init();
    }
    if (warp == 1) {
        umma::tmem_alloc(umma::smem_u32(tmem_slot), BN);
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
            for (int kt = 0; kt < nk; ++kt) {
                const int s = kt % S;
                const uint32_t ph = (uint32_t)(kt / S) & 1u;
                if (!umma::mbar_wait(empty0 + 8 * s, ph ^ 1u, kWaitNs)) {
                    atomicExch(&g_gemm_err, 11);
                    break;
                }
                umma::mbar_arrive_expect_tx(full0 + 8 * s, Cfg::A8_BYTES + Cfg::B_BYTES);
                umma::tma_load_2d(umma::smem_u32(sA8 + s * Cfg::A8_BYTES), &tmA, (kb + kt) * kBK, m0, full0 + 8 * s);
                umma::tma_load_2d(umma::smem_u32(sB + s * Cfg::B_BYTES), &tmB, (kb + kt) * kBK, n0, full0 + 8 * s);
            }
        }
        __syncwarp();
    } else if (warp >= 6) {
        // Converters: thread r owns row r of the 128-row tile.
        const int r = threadIdx.x - 6 * 32;
        bool ok = true;
        for (int kt = 0; kt < nk && ok; ++kt) {
            const int s = kt % S;
            const uint32_t ph = (uint32_t)(kt / S) & 1u;
            if (!umma::mbar_wait(full0 + 8 * s, ph, kWaitNs)) {
                atomicExch(&g_gemm_err, 12);
                ok = false;
                break;
            }
            const uint8_t *src = sA8 + s * Cfg::A8_BYTES + r * kBK;
            uint8_t *dst = sA + s * Cfg::A16_BYTES + r * 128;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int qq = (q + r) & 3;                    // rotate to spread the banks
                const uint4 u = *reinterpret_cast<const uint4 *>(src + qq * 16);
                const uint32_t w[4] = {u.x, u.y, u.z, u.w};
                uint32_t o[8];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[h] & 0xffffu), __NV_E4M3);
                    __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[h] >> 16), __NV_E4M3);
                    const float2 a = __half22float2(*reinterpret_cast<__half2 *>(&lo));
                    const float2 b = __half22float2(*reinterpret_cast<__half2 *>(&hi));
                    const __nv_bfloat162 ba = __floats2bfloat162_rn(a.x, a.y);
                    const __nv_bfloat162 bb = __floats2bfloat162_rn(b.x, b.y);
                    o[2 * h] = *reinterpret_cast<const uint32_t *>(&ba);
                    o[2 * h + 1] = *reinterpret_cast<const uint32_t *>(&bb);
                }
                // elements 16qq .. 16qq+15 = BF16 chunks 2qq and 2qq+1 of the row
                const int c0 = 2 * qq, c1 = 2 * qq + 1;
                *reinterpret_cast<uint4 *>(dst + ((c0 ^ (r & 7)) << 4)) = make_uint4(o[0], o[1], o[2], o[3]);
                *reinterpret_cast<uint4 *>(dst + ((c1 ^ (r & 7)) << 4)) = make_uint4(o[4], o[5], o[6], o[7]);
            }
            fence_proxy_async_smem();
            mbar_arrive_local(conv0 + 8 * s);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = umma::idesc_bf16_f32(kBM, BN);
            bool ok = true;
            for (int kt = 0; kt < nk; ++kt) {
                const int s = kt % S;
                const uint32_t ph = (uint32_t)(kt / S) & 1u;
                if (!umma::mbar_wait(conv0 + 8 * s, ph, kWaitNs)) {
                    atomicExch(&g_gemm_err, 13);
                    ok = false;
                    break;
                }
                umma::fence_after_sync();
                const uint64_t da = umma::desc_kmajor_sw128(umma::smem_u32(sA + s * Cfg::A16_BYTES));
                const uint64_t db = umma::desc_kmajor_sw128(umma::smem_u32(sB + s * Cfg::B_BYTES));
#pragma unroll
                for (int k = 0; k < kBK / 16; ++k)
                    umma::mma_bf16(tmem, da + 2 * k, db + 2 * k, idesc, (kt | k) != 0 ? 1u : 0u);
                umma::mma_commit(empty0 + 8 * s);
            }
            if (ok) umma::mma_commit(accum);
        }
        __syncwarp();
    } else {
        // Epilogue: warps 2..5 own TMEM lanes 32*(w%4) .., i.e. tile rows.
        bool ok = umma::mbar_wait(accum, 0, 4 * kWaitNs);
        if (EPI == kEpiF32 && gridDim.z > 1) ok = epilogue_all(ok);
        __syncwarp();
        umma::fence_after_sync();
        if (ok) {
            const int lane_base = (warp & 3) * 32;
            const int row = m0 + lane_base + lane;
            const uint32_t tl = tmem + ((uint32_t)lane_base << 16);
            if constexpr (EPI == kEpiF32) {
                const bool split = Z > 1;
                const int64_t ld_out = split ? (int64_t)N : ldc;
                float *crow = (split ? Cpart + (int64_t)blockIdx.z * M * N : C) + (int64_t)row * ld_out;
#pragma unroll 1
                for (int c = 0; c < BN / 32; ++c) {
                    uint32_t rr[32];
                    umma::tmem_ld_32x32b_x32(tl + (uint32_t)(c * 32), rr);
                    umma::tmem_ld_wait();
                    const int col0 = n0 + c * 32;
                    if (row < M) {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (col0 + j < N) crow[col0 + j] = __uint_as_float(rr[j]);
                    }
                }
                if (split) {
                    const int tile = blockIdx.x * gridDim.y + blockIdx.y;
                    if (splitk_last(tickets, tile, Z, threadIdx.x - 64)) {
                        splitk_reduce_row<BN>(Cpart, (int64_t)M * N, Z, row, n0, M, N, C, ldc);
                        if (threadIdx.x == 64) tickets[tile] = 0u;
                    }
                }
            } else {
                constexpr int HB = BN / 2;
#pragma unroll 1
                for (int c = 0; c < HB / 32; ++c) {
                    uint32_t a[32], b[32];
                    umma::tmem_ld_32x32b_x32(tl + (uint32_t)(c * 32), a);
                    umma::tmem_ld_32x32b_x32(tl + (uint32_t)(HB + c * 32), b);
                    umma::tmem_ld_wait();
                    if (row < M) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int bcol = c * 32 + j;
                            const float zf = __uint_as_float(a[j]) + __uint_as_float(b[j]);
                            const __nv_bfloat16 hi = __float2bfloat16_rn(zf);
                            const __nv_bfloat16 lo = __float2bfloat16_rn(zf - __bfloat162float(hi));
                            Ct[(int64_t)bcol * ldct + row] = hi;
                            Ct[(int64_t)(HB + bcol) * ldct + row] = lo;
                        }
                    }
                }
            }
        } else if (lane == 0) {
            atomicExch(&g_gemm_err, 14);
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (warp == 1) umma::tmem_dealloc(tmem, BN);
}

// 2-D FP8 (byte) tensor map over a rows x cols row-major matrix, box = box_rows x 64, no swizzle.
static int make_map_u8(CUtensorMap *map, const void *base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
    auto enc = tensor_map_encoder();
    if (enc == nullptr) return record_message(MV_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld};
    cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        char msg[128];
        snprintf(msg, sizeof(msg), "cuTensorMapEncodeTiled (FP8) failed (%d)", (int)r);
        return record_message(MV_ERR_CUDA, msg);
    }
    return MV_OK;
}

template <int BN, int EPI>
static int gemm_q8_set_attrs() {
    static int st = -1;
    if (st < 0)
        st = cudaFuncSetAttribute(gemm_q8_tn_kernel<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)Q8Cfg<BN>::SMEM) == cudaSuccess
                 ? MV_OK
                 : MV_ERR_CUDA;
    return st;
}

template <int BN, int EPI>
static void gemm_q8_launch(const CUtensorMap &ta, const CUtensorMap &tb, int64_t M, int64_t N, int64_t K, float *C,
                           int64_t ldc, __nv_bfloat16 *Ct, int64_t ldct, cudaStream_t s, int splits = 1,
                           float *Cpart = nullptr, unsigned *tickets = nullptr) {
    dim3 grid((unsigned)((M + kBM - 1) / kBM), (unsigned)((N + BN - 1) / BN), (unsigned)splits);
    gemm_q8_tn_kernel<BN, EPI><<<grid, kQ8Threads, Q8Cfg<BN>::SMEM, s>>>(ta, tb, C, (int)M, (int)N, (int)K, ldc, Ct,
                                                                         ldct, Cpart, tickets);
}

}  // namespace mv
