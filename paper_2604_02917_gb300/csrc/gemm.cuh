// tcgen05 BF16 GEMM  C = A B^T  (A: M x K, B: N x K, both K-major BF16;
// FP32 accumulation in tensor memory).  Shared by the sketch (sketch.cu) and
// the batched frontier solve (the frontier section of solve.cu).
//
// One CTA computes a 128 x BN tile with a K loop in steps of 64:
//   warp 0, one thread : TMA producer -- 128x64 A box and BNx64 B box per
//                        stage (128-byte swizzle), S-stage ring of mbarriers;
//   warp 1, one thread : MMA issuer -- four 128xBNx16 tcgen05.mma per stage
//                        into a 128 x BN FP32 accumulator in TMEM, then
//                        tcgen05.commit frees the stage;
//   warps 2..5         : epilogue -- tcgen05.ld 32 lanes x 32 columns at a
//                        time (warp w reads TMEM lanes 32*(w%4) ..).
// Epilogues: kEpiF32 stores C row-major in FP32; kEpiAccF32 adds
// alpha times the tile to C in place (C += alpha A B^T, FP32); kEpiPairSplitT
// (BN = 2B) adds columns b and B+b of the tile (the hi and lo parts of a
// split operand), splits the FP32 sum into BF16 hi + lo and stores both
// transposed (rows b and B+b of a 2B x M BF16 matrix).
// Out-of-range rows/columns/K of the boxes are zero-filled by TMA.  Every
// mbarrier wait is bounded in time; on timeout an error code is recorded
// in the translation unit's g_gemm_err and the CTA winds down.
#pragma once

#include <stdio.h>

#include <algorithm>

#include <cudaTypedefs.h>

#include "umma.cuh"

namespace mv {

constexpr int kGemmThreads = 192;
constexpr int kBM = 128, kBK = 64;
constexpr int kRasterRows = 16;               // row tiles per raster group (plain F32 GEMMs)
constexpr uint64_t kWaitNs = 2000000000ull;   // 2 s per wait

static __device__ int g_gemm_err;

// NA = number of A operands that share each B box: 1 for C = A B^T; 2 for
// C = (A_1 + A_2) B^T, both products issued into one accumulator (an FP32
// operand carried as a BF16 hi + lo pair against a BF16 B).
template <int BN, int NA = 1>
struct GemmCfg {
    static constexpr uint32_t A_BYTES = kBM * kBK * 2;
    static constexpr uint32_t B_BYTES = BN * kBK * 2;
    static constexpr uint32_t STAGE = NA * A_BYTES + B_BYTES;
    static constexpr int S = (int)((196608u / STAGE) < 8u ? (196608u / STAGE) : 8u);   // stages in 192 KB
    static constexpr size_t SMEM = 1024 + (size_t)S * STAGE + (2 * S + 1) * 8 + 16;
};

constexpr int kEpiF32 = 0, kEpiPairSplitT = 1, kEpiAccF32 = 2;

// Split-K (gridDim.z > 1, F32 epilogue only): CTA z covers k-steps
// [z nk / Z, (z+1) nk / Z) and writes its partial tile to Cpart[z] (M x N,
// row pitch N); the last CTA of a tile (atomic ticket after a fence) adds the
// Z partials in order z = 0 .. Z-1 and writes C, so the result is
// deterministic.  Run by the four epilogue warps (threads 0..127 of them).
__device__ __forceinline__ bool splitk_last(unsigned *tickets, int tile, int Z, int et) {
    __shared__ int s_last;
    __threadfence();
    asm volatile("bar.sync 2, 128;" ::: "memory");
    if (et == 0) s_last = atomicAdd(&tickets[tile], 1u) == (unsigned)(Z - 1);
    asm volatile("bar.sync 2, 128;" ::: "memory");
    const bool last = s_last;
    if (last) __threadfence();
    return last;
}

// AND of `ok` over the four epilogue warps (named barrier 2).
__device__ __forceinline__ bool epilogue_all(bool ok) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 2, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)ok)
        : "memory");
    return r != 0;
}

template <int BN>
__device__ __forceinline__ void splitk_reduce_row(const float *__restrict__ Cpart, int64_t pstride, int Z, int row,
                                                  int n0, int M, int N, float *__restrict__ C, int64_t ldc) {
    if (row >= M) return;
    const float *src = Cpart + (int64_t)row * N + n0;
    float *dst = C + (int64_t)row * ldc + n0;
    if (n0 + BN <= N && (N & 3) == 0 && (ldc & 3) == 0) {
        // float4 columns, eight of them (x Z partials) in flight at a time
#pragma unroll 1
        for (int j = 0; j < BN; j += 32) {
            float4 acc[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int z = 0; z < Z; ++z) {
                float4 v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = __ldcg(reinterpret_cast<const float4 *>(src + z * pstride + j + 4 * u));
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    acc[u].x += v[u].x;
                    acc[u].y += v[u].y;
                    acc[u].z += v[u].z;
                    acc[u].w += v[u].w;
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) *reinterpret_cast<float4 *>(dst + j + 4 * u) = acc[u];
        }
        return;
    }
    for (int j = 0; j < BN && n0 + j < N; ++j) {
        float acc = 0.f;
        for (int z = 0; z < Z; ++z) acc += __ldcg(src + (int64_t)z * pstride + j);
        dst[j] = acc;
    }
}

template <int BN, int EPI, int NA = 1>
__global__ void __launch_bounds__(kGemmThreads, 1)
gemm_bf16_tn_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const __grid_constant__ CUtensorMap tmA2, float *__restrict__ C, int M, int N, int K,
                    int64_t ldc, __nv_bfloat16 *__restrict__ Ct, int64_t ldct, float *__restrict__ Cpart,
                    unsigned *__restrict__ tickets, float alpha, const float *__restrict__ rscale) {
    using Cfg = GemmCfg<BN, NA>;
    constexpr int S = Cfg::S;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;                        // stage s, operand a at sA + (s NA + a) A_BYTES
    uint8_t *sB = smem + S * NA * Cfg::A_BYTES;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + S * Cfg::STAGE);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * S + 1);
    const uint32_t full0 = umma::smem_u32(bars), empty0 = umma::smem_u32(bars + S), accum = umma::smem_u32(bars + 2 * S);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Tile of this CTA.  Plain F32 GEMMs (no split-K) take a grouped raster:
    // CTAs in launch order sweep kRasterRows row tiles before the next column
    // tile, so a wave of co-resident CTAs touches about 16 A and 10 B
    // operand panels instead of every A panel.
    int rt = blockIdx.x, ct = blockIdx.y;
    if (EPI == kEpiF32 && gridDim.z == 1 && (int)gridDim.x > kRasterRows) {
        const int nrt = (int)gridDim.x, nct = (int)gridDim.y;
        const int lin = (int)blockIdx.x + nrt * (int)blockIdx.y;
        const int per = kRasterRows * nct, g = lin / per, first = g * kRasterRows;
        const int gh = min(nrt - first, kRasterRows), rem = lin - g * per;
        rt = first + rem % gh;
        ct = rem / gh;
    }
    const int m0 = rt * kBM, n0 = ct * BN;
    const int nk_all = (K + kBK - 1) / kBK, Z = gridDim.z;
    const int kb = (int)((int64_t)blockIdx.z * nk_all / Z), ke = (int)((int64_t)(blockIdx.z + 1) * nk_all / Z);
    const int nk = ke - kb;                    // k-steps of this CTA (all of them without split-K)

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            umma::mbar_init(full0 + 8 * s, 1);
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
            if (NA > 1) umma::prefetch_tensormap(&tmA2);
            for (int kt = 0; kt < nk; ++kt) {
                const int s = kt % S;
                const uint32_t ph = (uint32_t)(kt / S) & 1u;
                if (!umma::mbar_wait(empty0 + 8 * s, ph ^ 1u, kWaitNs)) {
                    atomicExch(&g_gemm_err, 1);
                    break;
                }
                umma::mbar_arrive_expect_tx(full0 + 8 * s, Cfg::STAGE);
                umma::tma_load_2d(umma::smem_u32(sA + s * NA * Cfg::A_BYTES), &tmA, (kb + kt) * kBK, m0, full0 + 8 * s);
                if (NA > 1)
                    umma::tma_load_2d(umma::smem_u32(sA + (s * NA + 1) * Cfg::A_BYTES), &tmA2, (kb + kt) * kBK, m0,
                                      full0 + 8 * s);
                umma::tma_load_2d(umma::smem_u32(sB + s * Cfg::B_BYTES), &tmB, (kb + kt) * kBK, n0, full0 + 8 * s);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = umma::idesc_bf16_f32(kBM, BN);
            bool ok = true;
            for (int kt = 0; kt < nk; ++kt) {
                const int s = kt % S;
                const uint32_t ph = (uint32_t)(kt / S) & 1u;
                if (!umma::mbar_wait(full0 + 8 * s, ph, kWaitNs)) {
                    atomicExch(&g_gemm_err, 2);
                    ok = false;
                    break;
                }
                umma::fence_after_sync();
                const uint64_t db = umma::desc_kmajor_sw128(umma::smem_u32(sB + s * Cfg::B_BYTES));
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    const uint64_t da = umma::desc_kmajor_sw128(umma::smem_u32(sA + (s * NA + a) * Cfg::A_BYTES));
#pragma unroll
                    for (int k = 0; k < kBK / 16; ++k)   // +32 bytes along K per 16-element step
                        umma::mma_bf16(tmem, da + 2 * k, db + 2 * k, idesc, (kt | k | a) != 0 ? 1u : 0u);
                }
                umma::mma_commit(empty0 + 8 * s);
            }
            if (ok) umma::mma_commit(accum);
        }
        __syncwarp();
    } else {
        // Epilogue: warp w owns TMEM lanes 32*(w%4) .. +31, i.e. tile rows.
        bool ok = umma::mbar_wait(accum, 0, 4 * kWaitNs);
        if (EPI == kEpiF32 && gridDim.z > 1) ok = epilogue_all(ok);   // split-K barriers need one shared outcome
        __syncwarp();
        umma::fence_after_sync();
        if (ok) {
            const int lane_base = (warp & 3) * 32;
            const int row = m0 + lane_base + lane;
            const uint32_t tl = tmem + ((uint32_t)lane_base << 16);
            if constexpr (EPI == kEpiF32) {
                // Without split-K straight to C; with it to this CTA's partial tile.
                const bool split = Z > 1;
                const int64_t ld_out = split ? (int64_t)N : ldc;
                float *crow = (split ? Cpart + (int64_t)blockIdx.z * M * N : C) + (int64_t)row * ld_out;
#pragma unroll 1
                for (int c = 0; c < BN / 32; ++c) {
                    uint32_t r[32];
                    umma::tmem_ld_32x32b_x32(tl + (uint32_t)(c * 32), r);
                    umma::tmem_ld_wait();
                    const int col0 = n0 + c * 32;
                    if (row < M) {
                        if (rscale != nullptr) {     // row-scaled operand (FP8 storage): C = diag(s) A B^T
                            const float sc = rscale[row];
#pragma unroll
                            for (int j = 0; j < 32; ++j) r[j] = __float_as_uint(__uint_as_float(r[j]) * sc);
                        }
                        if (col0 + 32 <= N && (ld_out & 3) == 0) {
#pragma unroll
                            for (int j = 0; j < 32; j += 4)
                                *reinterpret_cast<float4 *>(crow + col0 + j) =
                                    make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                                __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
                        } else {
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                if (col0 + j < N) crow[col0 + j] = __uint_as_float(r[j]);
                        }
                    }
                }
                if (split) {
                    const int tile = blockIdx.x * gridDim.y + blockIdx.y;
                    if (splitk_last(tickets, tile, Z, threadIdx.x - 64)) {
                        splitk_reduce_row<BN>(Cpart, (int64_t)M * N, Z, row, n0, M, N, C, ldc);
                        if (threadIdx.x == 64) tickets[tile] = 0u;
                    }
                }
            } else if constexpr (EPI == kEpiAccF32) {
                float *crow = C + (int64_t)row * ldc;
#pragma unroll 1
                for (int c = 0; c < BN / 32; ++c) {
                    uint32_t r[32];
                    umma::tmem_ld_32x32b_x32(tl + (uint32_t)(c * 32), r);
                    umma::tmem_ld_wait();
                    const int col0 = n0 + c * 32;
                    if (row < M) {
                        if (col0 + 32 <= N && (ldc & 3) == 0 && (reinterpret_cast<uintptr_t>(C) & 15) == 0) {
#pragma unroll
                            for (int j = 0; j < 32; j += 4) {
                                float4 v = *reinterpret_cast<const float4 *>(crow + col0 + j);
                                v.x = fmaf(alpha, __uint_as_float(r[j]), v.x);
                                v.y = fmaf(alpha, __uint_as_float(r[j + 1]), v.y);
                                v.z = fmaf(alpha, __uint_as_float(r[j + 2]), v.z);
                                v.w = fmaf(alpha, __uint_as_float(r[j + 3]), v.w);
                                *reinterpret_cast<float4 *>(crow + col0 + j) = v;
                            }
                        } else {
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                if (col0 + j < N) crow[col0 + j] = fmaf(alpha, __uint_as_float(r[j]), crow[col0 + j]);
                        }
                    }
                }
            } else {
                constexpr int HB = BN / 2;          // columns b and HB + b hold the hi and lo parts
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
            atomicExch(&g_gemm_err, 3);
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (warp == 1) umma::tmem_dealloc(tmem, BN);
}

// ------------------------------------------------------------------ host
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D BF16 tensor map over a rows x cols row-major matrix (leading dim ld),
// box = box_rows x 64 columns, 128-byte swizzle, zero fill out of range.
static int make_map_bf16(CUtensorMap *map, const void *base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
    auto enc = tensor_map_encoder();
    if (enc == nullptr) return record_message(MV_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        char msg[128];
        snprintf(msg, sizeof(msg), "cuTensorMapEncodeTiled failed (%d)", (int)r);
        return record_message(MV_ERR_CUDA, msg);
    }
    return MV_OK;
}

template <int BN, int EPI, int NA = 1>
static int gemm_set_attrs() {
    static int st = -1;
    if (st < 0)
        st = cudaFuncSetAttribute(gemm_bf16_tn_kernel<BN, EPI, NA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)GemmCfg<BN, NA>::SMEM) == cudaSuccess
                 ? MV_OK
                 : MV_ERR_CUDA;
    return st;
}

// Enqueue C = A B^T with prebuilt tensor maps (no synchronisation; capturable).
template <int BN, int EPI, int NA = 1>
static void gemm_launch(const CUtensorMap &ta, const CUtensorMap &tb, int64_t M, int64_t N, int64_t K, float *C,
                        int64_t ldc, __nv_bfloat16 *Ct, int64_t ldct, cudaStream_t s, int splits = 1,
                        float *Cpart = nullptr, unsigned *tickets = nullptr, float alpha = 1.0f,
                        const CUtensorMap *ta2 = nullptr, const float *rscale = nullptr) {
    dim3 grid((unsigned)((M + kBM - 1) / kBM), (unsigned)((N + BN - 1) / BN), (unsigned)splits);
    gemm_bf16_tn_kernel<BN, EPI, NA><<<grid, kGemmThreads, GemmCfg<BN, NA>::SMEM, s>>>(
        ta, tb, ta2 ? *ta2 : ta, C, (int)M, (int)N, (int)K, ldc, Ct, ldct, Cpart, tickets, alpha, rscale);
}

// ------------------------------------------------------------------ FP32-accurate products from BF16 pieces
// An FP32 value splits exactly into three BF16 pieces x = h + m + l (h the
// rounding of x, m that of x - h, l that of the rest; each subtraction is
// exact).  Of the nine piece products of a b, the six with piece indices
// summing to at most 2 are kept: the dropped m l, l m, l l are below
// 2^-24 |a b| each, so A B^T is formed to about FP32 accuracy by ONE GEMM
// over a K dimension six times as long: A' = [h h m h m l](A) and
// B' = [h m h l m h](B), each laid out as six segments of W columns
// (split3_piece gives the piece of each segment).
constexpr int kSplit3 = 6;
__host__ __device__ constexpr int split3_piece(int side, int seg) {
    // side 0 (A): h h m h m l; side 1 (B): h m h l m h -- pairs (h,h) (h,m) (m,h) (h,l) (m,m) (l,h)
    return side == 0 ? (seg < 2 ? 0 : seg == 2 ? 1 : seg == 3 ? 0 : seg == 4 ? 1 : 2)
                     : (seg == 0 ? 0 : seg == 1 ? 1 : seg == 2 ? 0 : seg == 3 ? 2 : seg == 4 ? 1 : 0);
}

__device__ __forceinline__ __nv_bfloat16 split3_get(float x, int piece) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    if (piece == 0) return h;
    const float r1 = x - __bfloat162float(h);
    const __nv_bfloat16 m = __float2bfloat16_rn(r1);
    if (piece == 1) return m;
    return __float2bfloat16_rn(r1 - __bfloat162float(m));
}

// X holds R vectors of length `cols` as rows (row pitch ldx).  Writes the
// K-major operand out (cols x 6W BF16, row pitch ldo): out[c][seg W + r] =
// piece(seg) of X[r][c] for r < R, zero for R <= r < W.  32 x 32 tiles
// through shared memory: coalesced along c on the read, along r on the write.
static __global__ void __launch_bounds__(256) split3_t_kernel(const float *__restrict__ X, int R, int cols, int64_t ldx,
                                                       int W, int side, __nv_bfloat16 *__restrict__ out,
                                                       int64_t ldo) {
    __shared__ float tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    for (int j = ty; j < 32; j += 8) {
        const int r = r0 + j, c = c0 + tx;
        tile[j][tx] = (r < R && c < cols) ? X[(int64_t)r * ldx + c] : 0.0f;
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
        const int c = c0 + j, r = r0 + tx;
        if (c >= cols || r >= W) continue;
        const float x = tile[tx][j];
        __nv_bfloat16 *o = out + (int64_t)c * ldo + r;
#pragma unroll
        for (int seg = 0; seg < kSplit3; ++seg) o[(int64_t)seg * W] = split3_get(x, split3_piece(side, seg));
    }
}

// K-splits for a tile-starved F32 GEMM: as many as fit in one wave of CTAs,
// each split keeping at least 16 k-steps.  (Filling two whole waves instead,
// 43 row tiles x 7 splits at 5440 x 12000, measured 64 us against 42 us for
// 3 splits in one wave: each extra split adds a partial tile to write and
// reduce, and the second wave re-pays the pipeline fill.)
static int gemm_splits(int64_t M, int64_t N, int64_t K, int BN, int sms) {
    const int64_t tiles = std::max<int64_t>(1, ((M + kBM - 1) / kBM) * ((N + BN - 1) / BN));
    const int64_t nk = (K + kBK - 1) / kBK;
    int64_t z = sms / tiles;
    z = std::min<int64_t>(z, nk / 16);
    return (int)std::max<int64_t>(1, std::min<int64_t>(z, 16));
}

// C = A B^T for BF16 K-major A (M x K) and B (N x K), FP32 row-major C;
// blocking (reads the device error word after the launch).
// With A2 non-NULL: C = (A + A2) B^T (A2 the lo part of a split FP32 A,
// same shape and pitch as A).  With rscale non-NULL: row i of C is scaled by
// rscale[i].
template <int BN>
static int gemm_bf16_tn(const void *A, int64_t M, int64_t lda, const void *B, int64_t N, int64_t ldb, int64_t K,
                        float *C, int64_t ldc, cudaStream_t s, const void *A2 = nullptr,
                        const float *rscale = nullptr) {
    CUtensorMap ta, tb, ta2;
    MV_TRY(make_map_bf16(&ta, A, M, K, lda, kBM));
    MV_TRY(make_map_bf16(&tb, B, N, K, ldb, BN));
    if (A2) MV_TRY(make_map_bf16(&ta2, A2, M, K, lda, kBM));
    if (A2) MV_TRY((gemm_set_attrs<BN, kEpiF32, 2>()));
    else MV_TRY((gemm_set_attrs<BN, kEpiF32>()));
    int zero = 0;
    MV_CUDA_TRY(cudaMemcpyToSymbolAsync(g_gemm_err, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    if (A2)
        gemm_launch<BN, kEpiF32, 2>(ta, tb, M, N, K, C, ldc, nullptr, 0, s, 1, nullptr, nullptr, 1.0f, &ta2, rscale);
    else
        gemm_launch<BN, kEpiF32>(ta, tb, M, N, K, C, ldc, nullptr, 0, s, 1, nullptr, nullptr, 1.0f, nullptr, rscale);
    MV_CUDA_TRY(cudaGetLastError());
    int err = 0;
    MV_CUDA_TRY(cudaMemcpyFromSymbolAsync(&err, g_gemm_err, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    MV_CUDA_TRY(cudaStreamSynchronize(s));
    if (err != 0) {
        char msg[96];
        snprintf(msg, sizeof(msg), "tcgen05 GEMM pipeline wait timed out (stage code %d)", err);
        return record_message(MV_ERR_TIMEOUT, msg);
    }
    return MV_OK;
}

}  // namespace mv
