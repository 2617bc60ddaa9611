// Sketch stage of STR (Sec. 2.3 / 2.5, step 1): tilde L = L Phi as a BF16
// tcgen05 GEMM with FP32 accumulation in tensor memory (gemm.cuh), with
// A = L (n x T, row-major = K-major), B = Phi^T (s x T, one sketch column per
// row, K-major) and C = tilde L (n x s, FP32, row-major), accumulated in
// chunks of 256 k-columns (gemm_chunk.cuh) so that the tensor core's one-sided
// accumulator rounding does not shrink the result.  The factor may be
// stored in any of the three types: BF16 is read as is; FP32 is split into
// a BF16 hi + lo pair, both multiplied against each staged Phi tile into one
// accumulator (2^-18 relative per term); FP8 e4m3 is expanded exactly to
// BF16 and its row scales are applied in the epilogue.  Phi itself is drawn
// on the device from a seed (rng.cuh) or handed in.
#include "gemm_chunk.cuh"
#include "rng.cuh"

using namespace mv;

namespace mv {

// H = bf16(x), D = bf16(x - H) for an n x T FP32 block (row pitches ld / ldo).
__global__ void __launch_bounds__(256) split_hilo_kernel(const float *__restrict__ L, int n, int T, int64_t ld,
                                                         __nv_bfloat16 *__restrict__ H, __nv_bfloat16 *__restrict__ D,
                                                         int64_t ldo) {
    const int64_t per_row = (ldo + 3) / 4, total = (int64_t)n * per_row;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / per_row);
        const int t0 = 4 * (int)(idx - (int64_t)i * per_row);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int t = t0 + a;
            if (t >= ldo) break;
            const float x = t < T ? L[(int64_t)i * ld + t] : 0.0f;
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            H[(int64_t)i * ldo + t] = h;
            D[(int64_t)i * ldo + t] = __float2bfloat16_rn(x - __bfloat162float(h));
        }
    }
}

// e4m3 -> BF16, exact (every e4m3 value is a BF16 value).
__global__ void __launch_bounds__(256) fp8_bf16_kernel(const uint8_t *__restrict__ Q, int n, int T, int64_t ld,
                                                       __nv_bfloat16 *__restrict__ B, int64_t ldo) {
    const int64_t total = (int64_t)n * ldo;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / ldo), t = (int)(idx - (int64_t)i * ldo);
        float v = 0.0f;
        if (t < T) {
            __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)Q[(int64_t)i * ld + t], __NV_E4M3);
            v = __half2float(*reinterpret_cast<__half *>(&h));
        }
        B[idx] = __float2bfloat16_rn(v);
    }
}

static int64_t pitch8(int64_t T) { return (T + 7) / 8 * 8; }

}  // namespace mv

extern "C" int mv_sketch(const void *d_L, int64_t n, int64_t T, int64_t ldL, const void *d_Phi_t, int64_t m,
                         int64_t ldP, float *d_L_sketch, int64_t ldS, mv_stream_t stream) {
    if (d_L == nullptr || d_Phi_t == nullptr || d_L_sketch == nullptr) return MV_ERR_INVALID_ARG;
    if (n < 1 || T < 1 || m < 1 || ldL < T || ldP < T || ldS < m) return MV_ERR_INVALID_ARG;
    if (n >= (1LL << 31) || T >= (1LL << 31) || m >= (1LL << 31))
        return record_message(MV_ERR_UNSUPPORTED, "mv_sketch: n, T and m must be below 2^31");
    if (((uintptr_t)d_L) % 16 || ((uintptr_t)d_Phi_t) % 16 || ((uintptr_t)d_L_sketch) % 16) return MV_ERR_INVALID_ARG;
    if ((ldL * 2) % 16 || (ldP * 2) % 16) return MV_ERR_INVALID_ARG;
    (void)cudaGetLastError();
    cudaStream_t s = (cudaStream_t)stream;
    MV_TRY(gemm_err_clear(s));
    MV_TRY(gemmc<256>(d_L, nullptr, n, ldL, d_Phi_t, m, ldP, T, d_L_sketch, ldS, GemmEpi{}, s));
    return gemm_err_check(s, "mv_sketch");
}

extern "C" size_t mv_sketch_workspace_size(int32_t dtype, int64_t n, int64_t T) {
    if (n < 1 || T < 1) return 0;
    switch (dtype) {
        case MV_BF16: return 0;
        case MV_F32: return align_up(2 * (size_t)n * pitch8(T), 256) + align_up(2 * (size_t)n * pitch8(T), 256);
        case MV_FP8_E4M3: return align_up(2 * (size_t)n * pitch8(T), 256);
        default: return 0;
    }
}

extern "C" int mv_sketch_dtype(const void *d_L, int32_t dtype, const float *d_row_scale, int64_t n, int64_t T,
                               int64_t ldL, const void *d_Phi_t, int64_t m, int64_t ldP, float *d_L_sketch,
                               int64_t ldS, void *d_ws, size_t ws_bytes, mv_stream_t stream) {
    if (dtype == MV_BF16) return mv_sketch(d_L, n, T, ldL, d_Phi_t, m, ldP, d_L_sketch, ldS, stream);
    if (dtype != MV_F32 && dtype != MV_FP8_E4M3) return MV_ERR_INVALID_ARG;
    if (d_L == nullptr || d_Phi_t == nullptr || d_L_sketch == nullptr) return MV_ERR_INVALID_ARG;
    if (dtype == MV_FP8_E4M3 && d_row_scale == nullptr) return MV_ERR_INVALID_ARG;
    if (n < 1 || T < 1 || m < 1 || ldL < T || ldP < T || ldS < m) return MV_ERR_INVALID_ARG;
    if (n >= (1LL << 31) || T >= (1LL << 31) || m >= (1LL << 31))
        return record_message(MV_ERR_UNSUPPORTED, "mv_sketch_dtype: n, T and m must be below 2^31");
    if (((uintptr_t)d_Phi_t) % 16 || ((uintptr_t)d_L_sketch) % 16 || (ldP * 2) % 16) return MV_ERR_INVALID_ARG;
    const size_t need = mv_sketch_workspace_size(dtype, n, T);
    if (d_ws == nullptr || ws_bytes < need || ((uintptr_t)d_ws) % 256 != 0) return MV_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    (void)cudaGetLastError();
    const int64_t ldo = pitch8(T);
    const int grid = 152 * 8;
    __nv_bfloat16 *B0 = reinterpret_cast<__nv_bfloat16 *>(d_ws);
    if (dtype == MV_F32) {
        __nv_bfloat16 *B1 = reinterpret_cast<__nv_bfloat16 *>(reinterpret_cast<char *>(d_ws) +
                                                              align_up(2 * (size_t)n * ldo, 256));
        split_hilo_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const float *>(d_L), (int)n, (int)T, ldL, B0, B1, ldo);
        MV_CUDA_TRY(cudaGetLastError());
        MV_TRY(gemm_err_clear(s));
        MV_TRY(gemmc<256>(B0, B1, n, ldo, d_Phi_t, m, ldP, T, d_L_sketch, ldS, GemmEpi{}, s));
        return gemm_err_check(s, "mv_sketch_dtype");
    }
    fp8_bf16_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const uint8_t *>(d_L), (int)n, (int)T, ldL, B0, ldo);
    MV_CUDA_TRY(cudaGetLastError());
    GemmEpi e;
    e.rscale = d_row_scale;
    MV_TRY(gemm_err_clear(s));
    MV_TRY(gemmc<256>(B0, nullptr, n, ldo, d_Phi_t, m, ldP, T, d_L_sketch, ldS, e, s));
    return gemm_err_check(s, "mv_sketch_dtype");
}

extern "C" int mv_gaussian_sketch(uint64_t seed, int64_t m, int64_t T, void *d_Phi_t, int64_t ldP,
                                  mv_stream_t stream) {
    if (d_Phi_t == nullptr || m < 1 || T < 1 || ldP < T || ldP % 8 != 0 || ((uintptr_t)d_Phi_t) % 16 != 0)
        return MV_ERR_INVALID_ARG;
    if (m >= (1LL << 31) || T >= (1LL << 31) - 8)
        return record_message(MV_ERR_UNSUPPORTED, "mv_gaussian_sketch: m and T must be below 2^31");
    cudaStream_t s = (cudaStream_t)stream;
    (void)cudaGetLastError();
    const double scale = 1.0 / sqrt((double)m);
    gaussian_sketch_kernel<<<152 * 16, 256, 0, s>>>((uint32_t)seed, (uint32_t)(seed >> 32), (int)m, (int)T, ldP,
                                                   (float)scale, scale, reinterpret_cast<__nv_bfloat16 *>(d_Phi_t));
    MV_CUDA_TRY(cudaGetLastError());
    return MV_OK;
}

extern "C" int mv_countsketch_draw(uint64_t seed, int64_t T, int64_t m, int32_t *d_hash, int8_t *d_sign,
                                   mv_stream_t stream) {
    if (d_hash == nullptr || d_sign == nullptr || T < 1 || m < 1) return MV_ERR_INVALID_ARG;
    if (T >= (1LL << 31) || m >= (1LL << 30))
        return record_message(MV_ERR_UNSUPPORTED, "mv_countsketch_draw: T must be below 2^31 and m below 2^30");
    cudaStream_t s = (cudaStream_t)stream;
    (void)cudaGetLastError();
    countsketch_draw_kernel<<<(int)std::min<int64_t>((T + 255) / 256, 152 * 8), 256, 0, s>>>(
        (uint32_t)seed, (uint32_t)(seed >> 32), (int)T, (uint32_t)m, d_hash, d_sign);
    MV_CUDA_TRY(cudaGetLastError());
    return MV_OK;
}
