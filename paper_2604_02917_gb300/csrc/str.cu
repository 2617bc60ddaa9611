// Truncate and ridge stages of STR (Sec. 2.5 steps 2-3, App. D.1-D.3).
//
// The thin SVD of tilde L (n x m) follows from the eigendecomposition of the
// n x n Gram matrix K = tilde L tilde L^T: its eigenvalues are sigma_i^2 and
// its eigenvectors are U.  The top-k pairs give the effective factor
// L_eff = U_k diag(sigma_k) (n x k), whose L_eff L_eff^T equals
// tilde L_k tilde L_k^T (App. D.3), and the ridge is gamma (or
// 1e-4 tr(Sigma)/n when the caller passes gamma < 0).  The pairs come from
// topk_eigen (trunc.cu): a Chebyshev-filtered subspace iteration whose
// products run on this library's tensor-core GEMMs, with a small FP64
// Rayleigh--Ritz eigenproblem at the end (a dense n x n eigensolver only
// for n <= 1024).  This file adds the knee rule of App. D.1 and the
// kappa-target ridge of App. D.2, and the whole STR build from a seed.
#include <stdio.h>

#include "mv_internal.cuh"
#include "trunc.h"

namespace mv {

// The knee rule of App. D.1 on lam (nonincreasing, cnt values):
// l = max{i < cnt : lam_i / lam_1 >= tau and lam_{i+1} / lam_i <= rho}
// (1-based; 0 if no i qualifies).  One block.
__global__ void knee_kernel(const double *__restrict__ lam, int cnt, double tau, double rho, int *out) {
    __shared__ int best;
    if (threadIdx.x == 0) best = 0;
    __syncthreads();
    const double lam1 = lam[0];
    int mine = 0;
    for (int i = 1 + threadIdx.x; i < cnt; i += blockDim.x) {
        const double li = lam[i - 1], lnext = lam[i];
        if (li / lam1 >= tau && lnext / li <= rho) mine = i;      // i grows along this thread's stride
    }
    if (mine > 0) atomicMax(&best, mine);
    __syncthreads();
    if (threadIdx.x == 0) *out = best;
}

// Columns k .. k_max-1 of L_eff and entries k .. k_max-1 of sigma set to zero.
__global__ void zero_tail_kernel(float *__restrict__ L_eff, int64_t ldE, int n, int k, int k_max,
                                 double *__restrict__ sigma) {
    const int w = k_max - k;
    const int64_t total = (int64_t)n * w;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / w), c = k + (int)(idx - (int64_t)i * w);
        L_eff[(int64_t)i * ldE + c] = 0.f;
        if (i == 0) sigma[c] = 0.0;
    }
}

// Workspace of a truncation: the eigen step's, then lam (max(n, 2k + 64))
// and the knee index.
static size_t lam_room(int64_t n, int64_t k) { return 8 * (size_t)std::max<int64_t>(n, 2 * k + 128); }

}  // namespace mv

using namespace mv;

extern "C" {

size_t mv_str_workspace_size(int64_t n, int64_t m, int64_t k) {
    const size_t e = topk_workspace_size(n, m, k);
    if (e == 0) return 0;
    return align_up(e, 256) + align_up(lam_room(n, k), 256) + 256;
}

int mv_str_truncate(const float *d_L_sketch, int64_t n, int64_t m, int64_t ldS, int64_t k, double gamma,
                    double trace_sigma, float *d_L_eff, int64_t ldE, double *d_sigma, double *h_gamma_out,
                    void *d_ws, size_t ws_bytes, mv_stream_t stream) {
    if (!d_L_sketch || !d_L_eff || !d_sigma) return MV_ERR_INVALID_ARG;
    if (n < 1 || m < 1 || k < 1 || k > n || ldS < m || ldE < k || n >= (1 << 30) || m >= (1 << 30))
        return MV_ERR_INVALID_ARG;
    const size_t need = mv_str_workspace_size(n, m, k);
    if (need == 0) return record_message(MV_ERR_UNSUPPORTED, "STR truncation: shape not supported");
    if (d_ws == nullptr || ws_bytes < need || ((uintptr_t)d_ws) % 256) return MV_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    (void)cudaGetLastError();
    const size_t e = align_up(topk_workspace_size(n, m, k), 256);
    double *lam = reinterpret_cast<double *>(reinterpret_cast<char *>(d_ws) + e);
    int64_t cnt = 0;
    MV_TRY(topk_eigen(d_L_sketch, n, m, ldS, k, d_L_eff, ldE, d_sigma, lam, &cnt, d_ws, e, s));
    if (h_gamma_out) *h_gamma_out = gamma >= 0.0 ? gamma : 1e-4 * trace_sigma / (double)n;
    return MV_OK;
}

int mv_str_truncate_knee(const float *d_L_sketch, int64_t n, int64_t m, int64_t ldS, double tau, double rho,
                         int64_t k_max, double kappa_target, double gamma, double trace_sigma, float *d_L_eff,
                         int64_t ldE, double *d_sigma, int64_t *h_k_out, double *h_gamma_out, void *d_ws,
                         size_t ws_bytes, mv_stream_t stream) {
    if (!d_L_sketch || !d_L_eff || !d_sigma || !h_k_out) return MV_ERR_INVALID_ARG;
    if (n < 2 || m < 1 || k_max < 1 || k_max > n || ldS < m || ldE < k_max || n >= (1 << 30) || m >= (1 << 30))
        return MV_ERR_INVALID_ARG;
    if (!(tau > 0.0) || !(rho > 0.0 && rho < 1.0) || !(kappa_target <= 0.0 || kappa_target > 1.0))
        return MV_ERR_INVALID_ARG;
    const size_t need = mv_str_workspace_size(n, m, k_max);
    if (need == 0) return record_message(MV_ERR_UNSUPPORTED, "STR truncation: shape not supported");
    if (d_ws == nullptr || ws_bytes < need || ((uintptr_t)d_ws) % 256) return MV_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    (void)cudaGetLastError();
    char *ws = reinterpret_cast<char *>(d_ws);
    const size_t e = align_up(topk_workspace_size(n, m, k_max), 256);
    double *lam = reinterpret_cast<double *>(ws + e);
    int *knee = reinterpret_cast<int *>(ws + e + align_up(lam_room(n, k_max), 256));
    int64_t cnt = 0;
    MV_TRY(topk_eigen(d_L_sketch, n, m, ldS, k_max, d_L_eff, ldE, d_sigma, lam, &cnt, ws, e, s));
    knee_kernel<<<1, 1024, 0, s>>>(lam, (int)cnt, tau, rho, knee);
    int hk = 0;
    double lam1 = 0.0;
    MV_CUDA_TRY(cudaMemcpyAsync(&hk, knee, sizeof(int), cudaMemcpyDeviceToHost, s));
    MV_CUDA_TRY(cudaMemcpyAsync(&lam1, lam, sizeof(double), cudaMemcpyDeviceToHost, s));
    MV_CUDA_TRY(cudaStreamSynchronize(s));
    if (hk < 1) return record_message(MV_ERR_NUMERIC, "knee rule: no index satisfies the tau and rho conditions");
    const int64_t k = hk < k_max ? hk : k_max;
    if (k < k_max) zero_tail_kernel<<<256, 256, 0, s>>>(d_L_eff, ldE, (int)n, (int)k, (int)k_max, d_sigma);
    MV_CUDA_TRY(cudaGetLastError());
    MV_CUDA_TRY(cudaStreamSynchronize(s));
    *h_k_out = k;
    if (h_gamma_out) {
        if (kappa_target > 1.0) *h_gamma_out = lam1 / (kappa_target - 1.0);   // App. D.2
        else *h_gamma_out = gamma >= 0.0 ? gamma : 1e-4 * trace_sigma / (double)n;
    }
    return MV_OK;
}

// Workspace of the whole STR build: tilde L (when the caller passes none),
// then either the sketch stage (Phi^T and the BF16 copy of L) or the
// truncation, which reuse the same bytes one after the other.
struct SkPlan {
    int64_t ldP, ldS;
    size_t o_ls, o_phi, o_conv, o_str, total;
};

static SkPlan sk_plan(int dtype, int64_t n, int64_t T, int64_t m, int64_t k, bool own_ls) {
    SkPlan p{};
    p.ldP = (T + 7) / 8 * 8;
    p.ldS = (m + 3) / 4 * 4;
    size_t off = 0;
    p.o_ls = off;
    if (own_ls) off = align_up(4 * (size_t)n * p.ldS, 256);
    p.o_phi = off;
    p.o_conv = align_up(p.o_phi + 2 * (size_t)m * p.ldP, 256);
    const size_t sketch_end = p.o_conv + mv_sketch_workspace_size(dtype, n, T);
    p.o_str = off;
    const size_t str_end = p.o_str + mv_str_workspace_size(n, m, k);
    p.total = align_up(sketch_end > str_end ? sketch_end : str_end, 256);
    return p;
}

size_t mv_sketch_str_workspace_size(int32_t dtype, int64_t n, int64_t T, int64_t m, int64_t k, int32_t own_sketch) {
    if (n < 1 || T < 1 || m < 1 || k < 1 || k > n || mv_str_workspace_size(n, m, k) == 0) return 0;
    if (dtype != MV_F32 && dtype != MV_BF16 && dtype != MV_FP8_E4M3) return 0;
    return sk_plan(dtype, n, T, m, k, own_sketch != 0).total;
}

int mv_sketch_str(const void *d_L, int32_t dtype, const float *d_row_scale, int64_t n, int64_t T, int64_t ldL,
                  int64_t m, uint64_t seed, int64_t k, double gamma, double trace_sigma, float *d_L_sketch,
                  int64_t ldS, float *d_L_eff, int64_t ldE, double *d_sigma, double *h_gamma_out, void *d_ws,
                  size_t ws_bytes, mv_stream_t stream) {
    if (!d_L || !d_L_eff || !d_sigma) return MV_ERR_INVALID_ARG;
    if (dtype != MV_F32 && dtype != MV_BF16 && dtype != MV_FP8_E4M3) return MV_ERR_INVALID_ARG;
    if (n < 1 || T < 1 || m < 1 || k < 1 || k > n || ldL < T || ldE < k) return MV_ERR_INVALID_ARG;
    if (d_L_sketch != nullptr && ldS < m) return MV_ERR_INVALID_ARG;
    const size_t need = mv_sketch_str_workspace_size(dtype, n, T, m, k, d_L_sketch == nullptr ? 1 : 0);
    if (need == 0) return MV_ERR_INVALID_ARG;
    if (d_ws == nullptr || ws_bytes < need || ((uintptr_t)d_ws) % 256) return MV_ERR_WORKSPACE;
    const SkPlan p = sk_plan(dtype, n, T, m, k, d_L_sketch == nullptr);
    char *ws = reinterpret_cast<char *>(d_ws);
    float *Ls = d_L_sketch ? d_L_sketch : reinterpret_cast<float *>(ws + p.o_ls);
    const int64_t lds = d_L_sketch ? ldS : p.ldS;
    // (1) Phi^T drawn from the seed, (2) tilde L = L Phi, (3) truncation + ridge
    MV_TRY(mv_gaussian_sketch(seed, m, T, ws + p.o_phi, p.ldP, stream));
    MV_TRY(mv_sketch_dtype(d_L, dtype, d_row_scale, n, T, ldL, ws + p.o_phi, m, p.ldP, Ls, lds, ws + p.o_conv,
                           need - p.o_conv, stream));
    return mv_str_truncate(Ls, n, m, lds, k, gamma, trace_sigma, d_L_eff, ldE, d_sigma, h_gamma_out, ws + p.o_str,
                           need - p.o_str, stream);
}

}  // extern "C"
