// Explicit covariance Sigma = L L^T (the classical model of Sec. 3's remark:
// NPGA with grad f(x) = 2 Sigma x, O(n^2) per iteration) formed once on the
// tcgen05 tensor cores.
//
// Sigma is symmetric, so only the 128 x 128 tiles (I, J) with I <= J are
// multiplied (one CTA per tile, nb (nb + 1) / 2 of them); the epilogue writes
// each tile and its mirror, so the stored Sigma is exactly symmetric.  On a
// diagonal tile only the entries with col >= row are kept and mirrored.
//
// Operands are BF16, K-major (row t of L along T), FP32 accumulation:
//   MV_BF16  L itself, one K-segment;
//   MV_FP8   Q expanded exactly to BF16 (e4m3 values are BF16 values) in
//            the workspace, one segment; the epilogue multiplies by
//            s_i s_j, since Sigma = diag(s) Q Q^T diag(s);
//   MV_F32   L = H + D with H = bf16(L), D = bf16(L - H) in the workspace;
//            Sigma ~= H H^T + H D^T + D H^T: each k-step stages the four
//            boxes H_I, D_I, H_J, D_J once and issues the three products
//            into one accumulator (the dropped D D^T and the rounding of D
//            are below 2^-16 |L_i| |L_j| per product term).
//
// Pipeline per CTA as in gemm.cuh: warp 0 (one thread) TMA producer over a
// 6-stage ring, warp 1 (one thread) MMA issuer (128 x 128 x 16 per
// instruction), warps 2..5 the epilogue, which also carries the running
// sum in FP32 registers (see the accumulation note below).  Every wait is bounded in time; a
// timeout is recorded in the device error word and the call returns
// MV_ERR_TIMEOUT.
#include "gemm.cuh"

namespace mv {

constexpr int kSigTile = 128;                 // BM = BN
constexpr uint32_t kSigBox = kSigTile * kBK * 2;   // one 128 x 64 BF16 operand box (16 KB)
// Stage geometry by number of products per k-step: one (BF16, FP8) = boxes
// A, B and 6 stages; three (FP32 split) = boxes H_I, D_I, H_J, D_J and 3 stages.
// A tensor-memory partial sums at most 64 MMAs (16 k-steps x 4, or 5 x 12).
template <int NSEG> struct SigGeo {
    static constexpr int BOXES = NSEG == 3 ? 4 : 2;
    static constexpr int S = NSEG == 3 ? 3 : 6;
    static constexpr uint32_t STAGE = BOXES * kSigBox;
    static constexpr int CHUNK = NSEG == 3 ? 5 : 16;
};
constexpr size_t kSigSmem = 1024 + 6 * (size_t)2 * kSigBox + (2 * 6 + 4) * 8 + 16;   // the larger of the two

// Tile order: the upper triangle is walked in super-blocks of kSigGroup x
// kSigGroup tiles (row-major inside each, super-blocks row-major over the
// upper triangle), so the ~150 CTAs that run at the same time share about
// 2 kSigGroup operand panels and read them from L2 rather than HBM.
constexpr int kSigGroup = 12;

__device__ __forceinline__ void tile_of(int t, int nb, int &I, int &J) {
    const int nsb = (nb + kSigGroup - 1) / kSigGroup;
    for (int P = 0; P < nsb; ++P) {
        const int i0 = P * kSigGroup, ri = min(nb, i0 + kSigGroup) - i0;
        for (int Q = P; Q < nsb; ++Q) {
            const int j0 = Q * kSigGroup, rj = min(nb, j0 + kSigGroup) - j0;
            if (Q == P) {                             // triangle of ri (ri + 1) / 2 tiles
                const int cnt = ri * (ri + 1) / 2;
                if (t < cnt) {
                    int a = 0;
                    while (t >= ri - a) {
                        t -= ri - a;
                        ++a;
                    }
                    I = i0 + a;
                    J = i0 + a + t;
                    return;
                }
                t -= cnt;
            } else {                                  // rectangle of ri x rj tiles
                const int cnt = ri * rj;
                if (t < cnt) {
                    I = i0 + t / rj;
                    J = j0 + t % rj;
                    return;
                }
                t -= cnt;
            }
        }
    }
    I = J = 0;                                        // not reached: t < nb (nb + 1) / 2
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Accumulation.  The tensor core adds each MMA's products into the FP32
// accumulator with a rounding that loses up to about an ulp of the running
// sum, with one sign when the terms have one sign (the diagonal of Sigma):
// over thousands of MMAs that is a bias of order 1e-4.  So a tile is
// accumulated in chunks of at most 64 MMAs (SigGeo::CHUNK k-steps), alternately into two
// 128-column tensor-memory buffers; the epilogue warps add every finished
// chunk into FP32 registers (round-to-nearest, fixed order) while the MMA
// warp fills the other buffer.
template <int NSEG>
__global__ void __launch_bounds__(kGemmThreads, 1)
sigma_gemm_kernel(const __grid_constant__ CUtensorMap tmH, const __grid_constant__ CUtensorMap tmD, int n, int K,
                  int nb, const float *__restrict__ rs, float *__restrict__ Sig, int64_t ldS) {
    using Geo = SigGeo<NSEG>;
    constexpr int S = Geo::S;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + S * Geo::STAGE);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * S + 4);
    const uint32_t full0 = umma::smem_u32(bars), empty0 = umma::smem_u32(bars + S);
    const uint32_t accf0 = umma::smem_u32(bars + 2 * S), acce0 = umma::smem_u32(bars + 2 * S + 2);
    // box b of stage s
    auto box = [&](int st, int b) { return umma::smem_u32(smem + (size_t)st * Geo::STAGE + (size_t)b * kSigBox); };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int I, J;
    tile_of(blockIdx.x, nb, I, J);
    const int m0 = I * kSigTile, n0 = J * kSigTile;
    const int steps = (K + kBK - 1) / kBK;
    const int nchunks = (steps + Geo::CHUNK - 1) / Geo::CHUNK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            umma::mbar_init(full0 + 8 * s, 1);
            umma::mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            umma::mbar_init(accf0 + 8 * b, 1);     // tcgen05.commit of a chunk
            umma::mbar_init(acce0 + 8 * b, 128);   // the four epilogue warps drained it
        }
        umma::mbar_fence_init();
    }
    if (warp == 1) {
        umma::tmem_alloc(umma::smem_u32(tmem_slot), 2 * kSigTile);
        umma::tmem_relinquish();
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            umma::prefetch_tensormap(&tmH);
            if (NSEG > 1) umma::prefetch_tensormap(&tmD);
            for (int g = 0; g < steps; ++g) {
                const int s = g % S;
                const uint32_t ph = (uint32_t)(g / S) & 1u;
                if (!umma::mbar_wait(empty0 + 8 * s, ph ^ 1u, kWaitNs)) {
                    atomicExch(&g_gemm_err, 1);
                    break;
                }
                const uint32_t fb = full0 + 8 * s;
                umma::mbar_arrive_expect_tx(fb, Geo::STAGE);
                if (NSEG == 3) {                       // H_I, D_I, H_J, D_J
                    umma::tma_load_2d(box(s, 0), &tmH, g * kBK, m0, fb);
                    umma::tma_load_2d(box(s, 1), &tmD, g * kBK, m0, fb);
                    umma::tma_load_2d(box(s, 2), &tmH, g * kBK, n0, fb);
                    umma::tma_load_2d(box(s, 3), &tmD, g * kBK, n0, fb);
                } else {                               // A_I, A_J
                    umma::tma_load_2d(box(s, 0), &tmH, g * kBK, m0, fb);
                    umma::tma_load_2d(box(s, 1), &tmH, g * kBK, n0, fb);
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = umma::idesc_bf16_f32(kBM, kSigTile);
            bool ok = true;
            for (int c = 0; c < nchunks && ok; ++c) {
                const int b = c & 1;
                if (c >= 2 && !umma::mbar_wait(acce0 + 8 * b, (uint32_t)((c >> 1) - 1) & 1u, 4 * kWaitNs)) {
                    atomicExch(&g_gemm_err, 4);
                    break;
                }
                umma::fence_after_sync();
                const uint32_t acc = tmem + (uint32_t)(b * kSigTile);
                const int g0 = c * Geo::CHUNK, g1 = min(steps, g0 + Geo::CHUNK);
                for (int g = g0; g < g1; ++g) {
                    const int s = g % S;
                    const uint32_t ph = (uint32_t)(g / S) & 1u;
                    if (!umma::mbar_wait(full0 + 8 * s, ph, kWaitNs)) {
                        atomicExch(&g_gemm_err, 2);
                        ok = false;
                        break;
                    }
                    umma::fence_after_sync();
                    if (NSEG == 3) {
                        // H_I H_J^T + H_I D_J^T + D_I H_J^T from the one stage
                        const uint64_t hi = umma::desc_kmajor_sw128(box(s, 0)), di = umma::desc_kmajor_sw128(box(s, 1));
                        const uint64_t hj = umma::desc_kmajor_sw128(box(s, 2)), dj = umma::desc_kmajor_sw128(box(s, 3));
#pragma unroll
                        for (int k = 0; k < kBK / 16; ++k) {
                            umma::mma_bf16(acc, hi + 2 * k, hj + 2 * k, idesc, (g != g0 || k != 0) ? 1u : 0u);
                            umma::mma_bf16(acc, hi + 2 * k, dj + 2 * k, idesc, 1u);
                            umma::mma_bf16(acc, di + 2 * k, hj + 2 * k, idesc, 1u);
                        }
                    } else {
                        const uint64_t da = umma::desc_kmajor_sw128(box(s, 0)), db = umma::desc_kmajor_sw128(box(s, 1));
#pragma unroll
                        for (int k = 0; k < kBK / 16; ++k)
                            umma::mma_bf16(acc, da + 2 * k, db + 2 * k, idesc, (g != g0 || k != 0) ? 1u : 0u);
                    }
                    umma::mma_commit(empty0 + 8 * s);
                }
                if (ok) umma::mma_commit(accf0 + 8 * b);
            }
        }
        __syncwarp();
    } else {
        const int lane_base = (warp & 3) * 32;
        const int row = m0 + lane_base + lane;
        const uint32_t tl = tmem + ((uint32_t)lane_base << 16);
        float acc[kSigTile];
#pragma unroll
        for (int j = 0; j < kSigTile; ++j) acc[j] = 0.f;
        bool ok = true;
        for (int c = 0; c < nchunks; ++c) {
            const int b = c & 1;
            if (!umma::mbar_wait(accf0 + 8 * b, (uint32_t)(c >> 1) & 1u, 4 * kWaitNs)) {
                ok = false;
                break;
            }
            umma::fence_after_sync();
#pragma unroll
            for (int q = 0; q < kSigTile / 32; ++q) {
                uint32_t r[32];
                umma::tmem_ld_32x32b_x32(tl + (uint32_t)(b * kSigTile + q * 32), r);
                umma::tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[q * 32 + j] += __uint_as_float(r[j]);
            }
            umma::fence_before_sync();
            mbar_arrive(acce0 + 8 * b);
        }
        if (ok) {
            const bool diag = I == J;
            const float sr = (rs != nullptr && row < n) ? rs[row] : 1.f;
            if (rs != nullptr) {
#pragma unroll
                for (int j = 0; j < kSigTile; ++j) acc[j] *= sr * (n0 + j < n ? __ldg(rs + n0 + j) : 0.f);
            }
            if (row < n) {
                float *srow = Sig + (int64_t)row * ldS;
                if (!diag && n0 + kSigTile <= n) {
#pragma unroll
                    for (int j = 0; j < kSigTile; j += 4)
                        *reinterpret_cast<float4 *>(srow + n0 + j) = make_float4(acc[j], acc[j + 1], acc[j + 2], acc[j + 3]);
                } else {
#pragma unroll
                    for (int j = 0; j < kSigTile; ++j)
                        if (n0 + j < n && (!diag || n0 + j >= row)) srow[n0 + j] = acc[j];
                }
            }
            // mirror: for fixed j the 32 lanes write 32 consecutive floats
#pragma unroll
            for (int j = 0; j < kSigTile; ++j)
                if (row < n && n0 + j < n && (!diag || n0 + j > row)) Sig[(int64_t)(n0 + j) * ldS + row] = acc[j];
        } else if (lane == 0) {
            atomicExch(&g_gemm_err, 3);
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (warp == 1) umma::tmem_dealloc(tmem, 2 * kSigTile);
}

// H = bf16(L), D = bf16(L - H), row by row (4 columns per thread step).
__global__ void split_hi_lo_kernel(const float *__restrict__ L, int64_t ld, int n, int T, __nv_bfloat16 *__restrict__ H,
                                   __nv_bfloat16 *__restrict__ D, int64_t ldo) {
    const int64_t quads = (T + 3) / 4;
    for (int64_t r = blockIdx.y; r < n; r += gridDim.y) {
        const float *src = L + r * ld;
        for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < quads; q += (int64_t)gridDim.x * blockDim.x) {
            const int64_t c = 4 * q;
            const float4 x = *reinterpret_cast<const float4 *>(src + c);   // c + 3 < ld: ld is a multiple of 4
            const float xs[4] = {x.x, x.y, x.z, x.w};
            __nv_bfloat16 h[4], d[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float v = c + j < T ? xs[j] : 0.f;
                h[j] = __float2bfloat16_rn(v);
                d[j] = __float2bfloat16_rn(v - __bfloat162float(h[j]));
            }
            *reinterpret_cast<uint2 *>(H + r * ldo + c) = *reinterpret_cast<const uint2 *>(h);
            *reinterpret_cast<uint2 *>(D + r * ldo + c) = *reinterpret_cast<const uint2 *>(d);
        }
    }
}

// Q (e4m3) -> BF16, exact (every e4m3 value is a BF16 value).
__global__ void expand_fp8_kernel(const uint8_t *__restrict__ Q, int64_t ld, int n, int T, __nv_bfloat16 *__restrict__ B,
                                  int64_t ldo) {
    const int64_t quads = (T + 3) / 4;
    for (int64_t r = blockIdx.y; r < n; r += gridDim.y) {
        const uint8_t *src = Q + r * ld;
        for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < quads; q += (int64_t)gridDim.x * blockDim.x) {
            const int64_t c = 4 * q;
            const uint32_t w = *reinterpret_cast<const uint32_t *>(src + c);   // c + 3 < ld: ld is a multiple of 16
            float f[4];
            Store<MV_FP8_E4M3>::four(w, f);
            __nv_bfloat16 b[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = __float2bfloat16_rn(c + j < T ? f[j] : 0.f);
            *reinterpret_cast<uint2 *>(B + r * ldo + c) = *reinterpret_cast<const uint2 *>(b);
        }
    }
}

static int64_t sigma_ldo(int64_t T) { return (T + 7) / 8 * 8; }   // BF16 row pitch: 16-byte rows

static int sigma_check(const mv_problem *P) {
    if (P == nullptr || P->L == nullptr) return MV_ERR_INVALID_ARG;
    if (P->dtype != MV_F32 && P->dtype != MV_BF16 && P->dtype != MV_FP8_E4M3) return MV_ERR_INVALID_ARG;
    if (P->layout != MV_LAYOUT_NT) return MV_ERR_INVALID_ARG;
    if (P->n < 1 || P->T < 1 || P->ld < P->T) return MV_ERR_INVALID_ARG;
    if (P->n > 32768 || P->T >= (1LL << 31))
        return record_message(MV_ERR_UNSUPPORTED, "mv_sigma_form: n must be <= 32768 and T below 2^31");
    const int es = dtype_size(P->dtype);
    if (((uintptr_t)P->L) % 16 != 0 || (P->ld * es) % 16 != 0) return MV_ERR_INVALID_ARG;
    if (P->dtype == MV_FP8_E4M3 && P->row_scale == nullptr) return MV_ERR_INVALID_ARG;
    return MV_OK;
}

static size_t sigma_ws_bytes(const mv_problem *P) {
    const size_t plane = align_up((size_t)P->n * (size_t)sigma_ldo(P->T) * 2, 256);
    if (P->dtype == MV_F32) return 2 * plane;
    if (P->dtype == MV_FP8_E4M3) return plane;
    return 256;
}

}  // namespace mv

using namespace mv;

extern "C" {

size_t mv_sigma_workspace_size(const mv_problem *P) {
    if (sigma_check(P) != MV_OK) return 0;
    return sigma_ws_bytes(P);
}

int mv_sigma_form(const mv_problem *P, float *d_Sigma, int64_t ldS, void *d_ws, size_t ws_bytes, mv_stream_t stream) {
    MV_TRY(sigma_check(P));
    if (d_Sigma == nullptr || ldS < P->n || (ldS & 3) != 0 || ((uintptr_t)d_Sigma) % 16 != 0) return MV_ERR_INVALID_ARG;
    const size_t need = sigma_ws_bytes(P);
    if (P->dtype != MV_BF16 && (d_ws == nullptr || ws_bytes < need || ((uintptr_t)d_ws) % 256 != 0))
        return MV_ERR_WORKSPACE;
    (void)cudaGetLastError();
    cudaStream_t s = (cudaStream_t)stream;
    const int n = (int)P->n, T = (int)P->T;
    const int nb = (n + kSigTile - 1) / kSigTile;
    const int64_t ldo = sigma_ldo(T);
    const size_t plane = align_up((size_t)n * (size_t)ldo * 2, 256);
    CUtensorMap tmH, tmD;
    int nseg = 1;
    const float *rs = nullptr;
    dim3 cgrid((unsigned)std::min<int64_t>((T / 4 + 255) / 256 + 1, 8), (unsigned)std::min(n, 4096));
    if (P->dtype == MV_BF16) {
        MV_TRY(make_map_bf16(&tmH, P->L, n, T, P->ld, kSigTile));
        tmD = tmH;
    } else if (P->dtype == MV_FP8_E4M3) {
        __nv_bfloat16 *B = reinterpret_cast<__nv_bfloat16 *>(d_ws);
        expand_fp8_kernel<<<cgrid, 256, 0, s>>>(reinterpret_cast<const uint8_t *>(P->L), P->ld, n, T, B, ldo);
        MV_TRY(make_map_bf16(&tmH, B, n, T, ldo, kSigTile));
        tmD = tmH;
        rs = P->row_scale;
    } else {
        __nv_bfloat16 *H = reinterpret_cast<__nv_bfloat16 *>(d_ws);
        __nv_bfloat16 *D = reinterpret_cast<__nv_bfloat16 *>(reinterpret_cast<char *>(d_ws) + plane);
        split_hi_lo_kernel<<<cgrid, 256, 0, s>>>(reinterpret_cast<const float *>(P->L), P->ld, n, T, H, D, ldo);
        MV_TRY(make_map_bf16(&tmH, H, n, T, ldo, kSigTile));
        MV_TRY(make_map_bf16(&tmD, D, n, T, ldo, kSigTile));
        nseg = 3;
    }
    MV_CUDA_TRY(cudaGetLastError());
    static int attrs = -1;
    if (attrs < 0)
        attrs = (cudaFuncSetAttribute(sigma_gemm_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kSigSmem) == cudaSuccess &&
                 cudaFuncSetAttribute(sigma_gemm_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kSigSmem) == cudaSuccess)
                    ? MV_OK
                    : MV_ERR_CUDA;
    if (attrs != MV_OK) return record_message(MV_ERR_CUDA, "sigma GEMM: shared-memory attribute refused");
    int zero = 0;
    MV_CUDA_TRY(cudaMemcpyToSymbolAsync(g_gemm_err, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    const unsigned tiles = (unsigned)((int64_t)nb * (nb + 1) / 2);
    if (nseg == 3)
        sigma_gemm_kernel<3><<<tiles, kGemmThreads, kSigSmem, s>>>(tmH, tmD, n, T, nb, rs, d_Sigma, ldS);
    else
        sigma_gemm_kernel<1><<<tiles, kGemmThreads, kSigSmem, s>>>(tmH, tmD, n, T, nb, rs, d_Sigma, ldS);
    MV_CUDA_TRY(cudaGetLastError());
    int err = 0;
    MV_CUDA_TRY(cudaMemcpyFromSymbolAsync(&err, g_gemm_err, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    MV_CUDA_TRY(cudaStreamSynchronize(s));
    if (err != 0) {
        char msg[96];
        snprintf(msg, sizeof(msg), "sigma GEMM pipeline wait timed out (stage code %d)", err);
        return record_message(MV_ERR_TIMEOUT, msg);
    }
    return MV_OK;
}

}  // extern "C"
