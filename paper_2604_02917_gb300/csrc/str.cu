// Truncate and ridge stages of STR (Sec. 2.5 steps 2-3, App. D.3), FP64.
//
// The thin SVD of tilde L (n x m) is obtained from the eigendecomposition of
// the n x n Gram matrix K = tilde L tilde L^T: its eigenvalues are sigma_i^2
// and its eigenvectors are U.  The top-k pairs give the effective factor
// L_eff = U_k diag(sigma_k) (n x k), whose L_eff L_eff^T equals
// tilde L_k tilde L_k^T (App. D.3), and the ridge is gamma (or
// 1e-4 tr(Sigma)/n when the caller passes gamma < 0).
//
// This one-time FP64 step uses two NVIDIA libraries, loaded at run time so
// that libmv itself loads without them: cuBLAS DSYRK for the Gram matrix (a
// plain library GEMM) and cuSOLVER DSYEVD for the eigenpairs (all n of them:
// on this GPU the full divide-and-conquer solver is several times faster
// than the selected-range one), of which the k largest are kept.
// Everything else (FP64 widening, assembling L_eff and sigma) is in the
// kernels below.
#include <dlfcn.h>
#include <stdio.h>

#include <mutex>

#include "mv_internal.cuh"

namespace mv {

// ------------------------------------------------------------------ runtime-loaded libraries
typedef int (*fn_cublasCreate)(void **);
typedef int (*fn_cublasSetStream)(void *, cudaStream_t);
typedef int (*fn_cublasDsyrk)(void *, int, int, int, int, const double *, const double *, int, const double *,
                              double *, int);
typedef int (*fn_cusolverCreate)(void **);
typedef int (*fn_cusolverSetStream)(void *, cudaStream_t);
typedef int (*fn_syevd_bs)(void *, int, int, int, const double *, int, const double *, int *);
typedef int (*fn_syevd)(void *, int, int, int, double *, int, double *, double *, int, int *);

constexpr int kOpT = 1, kFillLower = 0, kEigVector = 1;

struct Linalg {
    void *blas = nullptr, *solver = nullptr;
    void *hb = nullptr, *hs = nullptr;
    fn_cublasSetStream b_set_stream = nullptr;
    fn_cublasDsyrk dsyrk = nullptr;
    fn_cusolverSetStream s_set_stream = nullptr;
    fn_syevd_bs syevd_bs = nullptr;
    fn_syevd syevd = nullptr;
    bool ok = false;
};

static void *open_first(const char *const *names) {
    for (int i = 0; names[i]; ++i) {
        void *h = dlopen(names[i], RTLD_NOW | RTLD_GLOBAL);
        if (h) return h;
    }
    return nullptr;
}

static Linalg *linalg() {
    static Linalg L;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *blas_names[] = {"libcublas.so.13", "/usr/local/cuda/lib64/libcublas.so.13", "libcublas.so", nullptr};
        const char *solver_names[] = {"libcusolver.so.12", "/usr/local/cuda/lib64/libcusolver.so.12",
                                      "libcusolver.so", nullptr};
        void *lb = open_first(blas_names);
        void *ls = open_first(solver_names);
        if (!lb || !ls) return;
        auto bcreate = (fn_cublasCreate)dlsym(lb, "cublasCreate_v2");
        L.b_set_stream = (fn_cublasSetStream)dlsym(lb, "cublasSetStream_v2");
        L.dsyrk = (fn_cublasDsyrk)dlsym(lb, "cublasDsyrk_v2");
        auto screate = (fn_cusolverCreate)dlsym(ls, "cusolverDnCreate");
        L.s_set_stream = (fn_cusolverSetStream)dlsym(ls, "cusolverDnSetStream");
        L.syevd_bs = (fn_syevd_bs)dlsym(ls, "cusolverDnDsyevd_bufferSize");
        L.syevd = (fn_syevd)dlsym(ls, "cusolverDnDsyevd");
        if (!bcreate || !L.b_set_stream || !L.dsyrk || !screate || !L.s_set_stream || !L.syevd_bs ||
            !L.syevd)
            return;
        if (bcreate(&L.hb) != 0 || screate(&L.hs) != 0) return;
        L.ok = true;
    });
    return L.ok ? &L : nullptr;
}

// ------------------------------------------------------------------ kernels
__global__ void widen_kernel(const float *__restrict__ src, int n, int m, int64_t ld, double *__restrict__ dst) {
    const int64_t total = (int64_t)n * m;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / m, j = idx - i * m;
        dst[idx] = (double)src[i * ld + j];
    }
}

// Eigenpairs come back in ascending order in the first k columns of the
// column-major n x n array; column c of L_eff takes the (c+1)-th largest.
__global__ void leff_kernel(const double *__restrict__ U, const double *__restrict__ W, int n, int k,
                            float *__restrict__ L_eff, int64_t ldE, double *__restrict__ sigma) {
    const int64_t total = (int64_t)n * k;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / k), c = (int)(idx - (int64_t)i * k);
        const int src = k - 1 - c;
        const double s = sqrt(fmax(W[src], 0.0));
        L_eff[(int64_t)i * ldE + c] = (float)(U[(int64_t)src * n + i] * s);
        if (i == 0) sigma[c] = s;
    }
}

// The knee rule of App. D.1 on the eigenvalues W (ascending, n of them):
// with lam_i = W[n - i] (i = 1 .. n, nonincreasing), writes
// l = max{i < n : lam_i / lam_1 >= tau and lam_{i+1} / lam_i <= rho}
// (0 if no i qualifies).  One block.
__global__ void knee_kernel(const double *__restrict__ W, int n, double tau, double rho, int *out) {
    __shared__ int best;
    if (threadIdx.x == 0) best = 0;
    __syncthreads();
    const double lam1 = W[n - 1];
    int mine = 0;
    for (int i = 1 + threadIdx.x; i < n; i += blockDim.x) {
        const double li = W[n - i], lnext = W[n - i - 1];
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

struct StrPlan {
    size_t o_a, o_k, o_w, o_work, o_info, o_knee, total;
    int lwork;
};

static int str_plan(int64_t n, int64_t m, int64_t k, StrPlan *p) {
    Linalg *L = linalg();
    if (!L) return record_message(MV_ERR_UNSUPPORTED, "STR truncation needs cuBLAS and cuSOLVER (not found)");
    int lwork = 0;
    if (L->syevd_bs(L->hs, kEigVector, kFillLower, (int)n, nullptr, (int)n, nullptr, &lwork) != 0)
        return record_message(MV_ERR_CUDA, "cusolverDnDsyevd_bufferSize failed");
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    p->o_a = take(8 * (size_t)n * m);
    p->o_k = take(8 * (size_t)n * n);
    p->o_w = take(8 * (size_t)n);
    p->o_work = take(8 * (size_t)lwork);
    p->o_info = take(sizeof(int));
    p->o_knee = take(sizeof(int));
    p->total = off;
    p->lwork = lwork;
    return MV_OK;
}

}  // namespace mv

using namespace mv;

extern "C" {

size_t mv_str_workspace_size(int64_t n, int64_t m, int64_t k) {
    if (n < 1 || m < 1 || k < 1 || k > n || n >= (1 << 30) || m >= (1 << 30)) return 0;
    StrPlan p;
    if (str_plan(n, m, k, &p) != MV_OK) return 0;
    return p.total;
}

// FP64 Gram K = tilde L tilde L^T and all its eigenpairs (ascending) into the
// workspace: eigenvectors overwrite K (column-major), eigenvalues in W.
static int str_eigen(const float *d_L_sketch, int64_t n, int64_t m, int64_t ldS, const StrPlan &p, char *ws,
                     cudaStream_t s) {
    Linalg *L = linalg();
    double *A = reinterpret_cast<double *>(ws + p.o_a);
    double *K = reinterpret_cast<double *>(ws + p.o_k);
    double *W = reinterpret_cast<double *>(ws + p.o_w);
    double *work = reinterpret_cast<double *>(ws + p.o_work);
    int *info = reinterpret_cast<int *>(ws + p.o_info);
    widen_kernel<<<1024, 256, 0, s>>>(d_L_sketch, (int)n, (int)m, ldS, A);
    MV_CUDA_TRY(cudaGetLastError());
    // Row-major n x m tilde L is the column-major m x n matrix A; K = A^T A.
    if (L->b_set_stream(L->hb, s) != 0) return record_message(MV_ERR_CUDA, "cublasSetStream failed");
    const double one = 1.0, zero = 0.0;
    if (L->dsyrk(L->hb, kFillLower, kOpT, (int)n, (int)m, &one, A, (int)m, &zero, K, (int)n) != 0)
        return record_message(MV_ERR_CUDA, "cublasDsyrk failed");
    if (L->s_set_stream(L->hs, s) != 0) return record_message(MV_ERR_CUDA, "cusolverDnSetStream failed");
    if (L->syevd(L->hs, kEigVector, kFillLower, (int)n, K, (int)n, W, work, p.lwork, info) != 0)
        return record_message(MV_ERR_CUDA, "cusolverDnDsyevd failed");
    int hinfo = 0;
    MV_CUDA_TRY(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s));
    MV_CUDA_TRY(cudaStreamSynchronize(s));
    if (hinfo != 0) {
        char msg[96];
        snprintf(msg, sizeof(msg), "cusolverDnDsyevd: info=%d", hinfo);
        return record_message(MV_ERR_NUMERIC, msg);
    }
    return MV_OK;
}

int mv_str_truncate(const float *d_L_sketch, int64_t n, int64_t m, int64_t ldS, int64_t k, double gamma,
                    double trace_sigma, float *d_L_eff, int64_t ldE, double *d_sigma, double *h_gamma_out,
                    void *d_ws, size_t ws_bytes, mv_stream_t stream) {
    if (!d_L_sketch || !d_L_eff || !d_sigma) return MV_ERR_INVALID_ARG;
    if (n < 1 || m < 1 || k < 1 || k > n || ldS < m || ldE < k || n >= (1 << 30) || m >= (1 << 30))
        return MV_ERR_INVALID_ARG;
    StrPlan p;
    MV_TRY(str_plan(n, m, k, &p));
    if (d_ws == nullptr || ws_bytes < p.total || ((uintptr_t)d_ws) % 256) return MV_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    (void)cudaGetLastError();
    char *ws = reinterpret_cast<char *>(d_ws);
    MV_TRY(str_eigen(d_L_sketch, n, m, ldS, p, ws, s));
    double *K = reinterpret_cast<double *>(ws + p.o_k);
    double *W = reinterpret_cast<double *>(ws + p.o_w);
    // all n pairs come back ascending: the k largest are the last k columns
    leff_kernel<<<1024, 256, 0, s>>>(K + (size_t)(n - k) * n, W + (n - k), (int)n, (int)k, d_L_eff, ldE, d_sigma);
    MV_CUDA_TRY(cudaGetLastError());
    MV_CUDA_TRY(cudaStreamSynchronize(s));
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
    StrPlan p;
    MV_TRY(str_plan(n, m, k_max, &p));
    if (d_ws == nullptr || ws_bytes < p.total || ((uintptr_t)d_ws) % 256) return MV_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    (void)cudaGetLastError();
    char *ws = reinterpret_cast<char *>(d_ws);
    MV_TRY(str_eigen(d_L_sketch, n, m, ldS, p, ws, s));
    double *K = reinterpret_cast<double *>(ws + p.o_k);
    double *W = reinterpret_cast<double *>(ws + p.o_w);
    int *knee = reinterpret_cast<int *>(ws + p.o_knee);
    knee_kernel<<<1, 1024, 0, s>>>(W, (int)n, tau, rho, knee);
    int hk = 0;
    double lam1 = 0.0;
    MV_CUDA_TRY(cudaMemcpyAsync(&hk, knee, sizeof(int), cudaMemcpyDeviceToHost, s));
    MV_CUDA_TRY(cudaMemcpyAsync(&lam1, W + (n - 1), sizeof(double), cudaMemcpyDeviceToHost, s));
    MV_CUDA_TRY(cudaStreamSynchronize(s));
    if (hk < 1) return record_message(MV_ERR_NUMERIC, "knee rule: no index satisfies the tau and rho conditions");
    const int64_t k = hk < k_max ? hk : k_max;
    leff_kernel<<<1024, 256, 0, s>>>(K + (size_t)(n - k) * n, W + (n - k), (int)n, (int)k, d_L_eff, ldE, d_sigma);
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
