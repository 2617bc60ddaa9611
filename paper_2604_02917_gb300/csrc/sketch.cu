// Sketch stage of STR (Sec. 2.3 / 2.5, step 1): tilde L = L Phi as a BF16
// tcgen05 GEMM with FP32 accumulation in tensor memory (gemm.cuh), with
// A = L (n x T, row-major = K-major), B = Phi^T (m x T, one sketch column per
// row, K-major) and C = tilde L (n x m, FP32, row-major).
#include "gemm.cuh"


using namespace mv;

extern "C" int mv_sketch(const void *d_L, int64_t n, int64_t T, int64_t ldL, const void *d_Phi_t, int64_t m,
                         int64_t ldP, float *d_L_sketch, int64_t ldS, mv_stream_t stream) {
    if (d_L == nullptr || d_Phi_t == nullptr || d_L_sketch == nullptr) return MV_ERR_INVALID_ARG;
    if (n < 1 || T < 1 || m < 1 || ldL < T || ldP < T || ldS < m) return MV_ERR_INVALID_ARG;
    if (n >= (1LL << 31) || T >= (1LL << 31) || m >= (1LL << 31)) return MV_ERR_UNSUPPORTED;
    if (((uintptr_t)d_L) % 16 || ((uintptr_t)d_Phi_t) % 16 || ((uintptr_t)d_L_sketch) % 16) return MV_ERR_INVALID_ARG;
    if ((ldL * 2) % 16 || (ldP * 2) % 16) return MV_ERR_INVALID_ARG;
    (void)cudaGetLastError();
    return mv::gemm_bf16_tn<256>(d_L, n, ldL, d_Phi_t, m, ldP, T, d_L_sketch, ldS, (cudaStream_t)stream);
}
