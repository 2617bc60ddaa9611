// Truncation stage of STR (Sec. 2.5, step (2)): the k largest eigenpairs of
// the Gram matrix K = tilde L tilde L^T (eigenvalues sigma_i^2, vectors U),
// computed as the paper's appendix on the complexity of STR suggests for
// large problems -- a partial decomposition by subspace iteration -- rather
// than by a dense eigensolver on all n pairs.
//
// Every product with K or with the n x b panels is a tensor-core GEMM of
// this library (gemm_chunk.cuh) on three-piece BF16 splits of its FP32
// operands (six piece products: FP32-accurate), accumulated in chunks so the
// tensor core's one-sided accumulator rounding does not bias the spectrum.
// The only library call is the symmetric eigensolver (cuSOLVER DSYEVD,
// loaded at run time) on the small b x b Rayleigh--Ritz matrices.
//
// Algorithm (block size b = max(2k, k + 512), rounded up to 64: the cut sits
// halfway down the unwanted part of the block, and a flat spectrum needs that
// part wide for the filter to separate the wanted eigenvalues):
//   1. K = tilde L tilde L^T (n x n FP32).
//   2. Q = orth(K^2 G), G an n x b Gaussian block.
//   3. Rayleigh--Ritz: the eigenvalues theta of Q^T K Q (b x b, FP32) give
//      the filter's cut c = theta_{(k+b)/2}, the Ritz value halfway down
//      the block's unwanted part: a lower bound of lambda_{(k+b)/2}, hence
//      below every wanted eigenvalue.
//   4. Chebyshev filtering: Y = T_d((K - e) / h) Q with e = h = c / 2, so
//      the unwanted eigenvalues [0, c] map to [-1, 1] and stay bounded while
//      the wanted ones above c grow like T_d; Q = orth(Y); repeated for the
//      degree schedule (5, 5, 3).  The three-term recurrence is fused into the GEMM
//      epilogue: Y_{j+1} = (2/h) K Y_j - (2e/h) Y_j - Y_{j-1}.
//   5. Final Rayleigh--Ritz: H = Q^T K Q in FP64, its eigenpairs (theta, V);
//      the k largest give sigma = sqrt(theta) and U = Q V.
// orth() is Lowdin's symmetric orthonormalisation Q = Y (Y^T Y)^{-1/2},
// with the inverse square root of the b x b Gram matrix (column-scaled to a
// unit diagonal and then by its Gershgorin bound) by the coupled
// Newton--Schulz iteration Y <- Y T, Z <- T Z, T = (3I - Z Y)/2 (Higham,
// "Functions of Matrices", 2008, Sec. 6.3), on the Gram matrix shifted by
// 1e-5 of its norm (the Gram matrix of an ill-conditioned panel in FP32 can
// have slightly negative eigenvalues, on which the iteration diverges); three
// passes with shifts 1e-5, 1e-7 and 0, the later ones restoring
// orthogonality to working precision.
//
// Small problems (n <= 1024, or b >= n) take the direct route: K and then
// all its eigenpairs by DSYEVD on the n x n matrix.
#include <dlfcn.h>
#include <math.h>
#include <cmath>
#include <stdio.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "gemm_chunk.cuh"
#include "rng.cuh"
#include "trunc.h"

namespace mv {

// ------------------------------------------------------------------ cuSOLVER (small dense eigenproblems)
typedef int (*fn_cusolverCreate)(void **);
typedef int (*fn_cusolverSetStream)(void *, cudaStream_t);
typedef int (*fn_syevd_bs)(void *, int, int, int, const double *, int, const double *, int *);
typedef int (*fn_syevd)(void *, int, int, int, double *, int, double *, double *, int, int *);
typedef int (*fn_ssyevd_bs)(void *, int, int, int, const float *, int, const float *, int *);
typedef int (*fn_ssyevd)(void *, int, int, int, float *, int, float *, float *, int, int *);

constexpr int kEigVector = 1, kEigNoVector = 0, kFillLower = 0;

struct EigLib {
    void *hs = nullptr;
    fn_cusolverSetStream set_stream = nullptr;
    fn_syevd_bs syevd_bs = nullptr;
    fn_syevd syevd = nullptr;
    fn_ssyevd_bs ssyevd_bs = nullptr;
    fn_ssyevd ssyevd = nullptr;
    bool ok = false;
};

static EigLib *eig_lib() {
    static EigLib L;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *names[] = {"libcusolver.so.12", "/usr/local/cuda/lib64/libcusolver.so.12", "libcusolver.so",
                               nullptr};
        void *h = nullptr;
        for (int i = 0; names[i] && !h; ++i) h = dlopen(names[i], RTLD_NOW | RTLD_GLOBAL);
        if (!h) return;
        auto create = (fn_cusolverCreate)dlsym(h, "cusolverDnCreate");
        L.set_stream = (fn_cusolverSetStream)dlsym(h, "cusolverDnSetStream");
        L.syevd_bs = (fn_syevd_bs)dlsym(h, "cusolverDnDsyevd_bufferSize");
        L.syevd = (fn_syevd)dlsym(h, "cusolverDnDsyevd");
        L.ssyevd_bs = (fn_ssyevd_bs)dlsym(h, "cusolverDnSsyevd_bufferSize");
        L.ssyevd = (fn_ssyevd)dlsym(h, "cusolverDnSsyevd");
        if (!create || !L.set_stream || !L.syevd_bs || !L.syevd || !L.ssyevd_bs || !L.ssyevd) return;
        if (create(&L.hs) != 0) return;
        L.ok = true;
    });
    return L.ok ? &L : nullptr;
}

// ------------------------------------------------------------------ small kernels
// FP32 standard normals (Philox4x32-10 + Box--Muller): the random start block.
static __global__ void randn_kernel(uint32_t k0, uint32_t k1, int R, int C, int64_t ld, float *__restrict__ out) {
    const int64_t total = (int64_t)R * C;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / C), c = (int)(idx - (int64_t)r * C);
        const Philox4 w = philox4x32_10((uint32_t)r, (uint32_t)c, 2u, 0u, k0, k1);
        const float u = (float)((w.w[0] >> 8) + 1u) * 5.9604644775390625e-8f;
        const float v = (float)(w.w[1] >> 8) * 5.9604644775390625e-8f;
        out[(int64_t)r * ld + c] = sqrtf(-2.0f * logf(u)) * cospif(2.0f * v);
    }
}

// Lowdin set-up on the b x b Gram matrix G: D_i = G_ii^{-1/2} and the
// Gershgorin row sums r_i = sum_j |D_i G_ij D_j| of the unit-diagonal D G D.
static __global__ void lowdin_rows_kernel(const float *__restrict__ G, int b, int64_t ld, float *__restrict__ D,
                                          float *__restrict__ rows) {
    const int i = blockIdx.x;
    __shared__ float red[32];
    const float di = rsqrtf(fmaxf(G[(int64_t)i * ld + i], 1e-30f));
    float acc = 0.0f;
    for (int j = threadIdx.x; j < b; j += blockDim.x)
        acc += fabsf(G[(int64_t)i * ld + j]) * rsqrtf(fmaxf(G[(int64_t)j * ld + j], 1e-30f));
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        D[i] = di;
        rows[i] = t * di;
    }
}

// A = (D G D / s + delta I) / (1 + delta) with s = max_i rows_i (>= the
// spectral radius of D G D), and Z = I: the start of the coupled
// Newton--Schulz iteration; *s_out = s (1 + delta), so that A ~ D G D / s_out.
// The shift delta keeps every eigenvalue of A at least delta / (1 + delta):
// the Gram matrix of a badly conditioned panel, formed in FP32, can have
// eigenvalues at the rounding level that come out slightly negative, and the
// iteration diverges on a negative one.  Directions that small carry no
// information; the shift only scales them down, and the second pass
// normalises what is left.  One grid.
static __global__ void lowdin_start_kernel(const float *__restrict__ G, int b, int64_t ld, const float *__restrict__ D,
                                           const float *__restrict__ rows, float delta, float *__restrict__ A,
                                           float *__restrict__ Z, float *__restrict__ s_out) {
    __shared__ float s_sh;
    if (threadIdx.x == 0) {
        float s = 1.0f;
        for (int i = 0; i < b; ++i) s = fmaxf(s, rows[i]);
        s_sh = s;
        if (blockIdx.x == 0) *s_out = s * (1.0f + delta);
    }
    __syncthreads();
    const float inv = 1.0f / s_sh, sh = 1.0f / (1.0f + delta);
    const int64_t total = (int64_t)b * b;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / b), j = (int)(idx - (int64_t)i * b);
        A[(int64_t)i * ld + j] = (D[i] * G[(int64_t)i * ld + j] * D[j] * inv + (i == j ? delta : 0.0f)) * sh;
        Z[(int64_t)i * ld + j] = i == j ? 1.0f : 0.0f;
    }
}

// T = 1.5 I - 0.5 P.
static __global__ void ns_t_kernel(const float *__restrict__ P, int b, int64_t ld, float *__restrict__ T) {
    const int64_t total = (int64_t)b * b;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / b), j = (int)(idx - (int64_t)i * b);
        T[(int64_t)i * ld + j] = (i == j ? 1.5f : 0.0f) - 0.5f * P[(int64_t)i * ld + j];
    }
}

// M = D Z / sqrt(s): Q = Y M is then Y (Y^T Y)^{-1/2} (Z ~ (D G D / s)^{-1/2}).
static __global__ void lowdin_m_kernel(const float *__restrict__ D, const float *__restrict__ Z, int b, int64_t ld,
                                       const float *__restrict__ s, float *__restrict__ M) {
    const float r = rsqrtf(*s);
    const int64_t total = (int64_t)b * b;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / b), j = (int)(idx - (int64_t)i * b);
        M[(int64_t)i * ld + j] = D[i] * Z[(int64_t)i * ld + j] * r;
    }
}

// H (b x b FP32, from a GEMM) -> FP64, symmetrised: (H + H^T) / 2.  The
// eigensolver reads the lower triangle of a column-major array, which for a
// symmetric matrix is the same bytes as row-major.
static __global__ void widen_sym_kernel(const float *__restrict__ H, int b, int64_t ld, double *__restrict__ Hd) {
    const int64_t total = (int64_t)b * b;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / b), j = (int)(idx - (int64_t)i * b);
        Hd[idx] = 0.5 * ((double)H[(int64_t)i * ld + j] + (double)H[(int64_t)j * ld + i]);
    }
}

// H (b x b FP32) -> contiguous FP32 (H + H^T) / 2: the input of the FP32
// eigensolver that only places the filter's cut.
static __global__ void sym_f32_kernel(const float *__restrict__ H, int b, int64_t ld, float *__restrict__ Hs) {
    const int64_t total = (int64_t)b * b;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / b), j = (int)(idx - (int64_t)i * b);
        Hs[idx] = 0.5f * (H[(int64_t)i * ld + j] + H[(int64_t)j * ld + i]);
    }
}

// From the eigensolver's output (W ascending, V column-major b x b): the k
// largest pairs in descending order -- Vt row c = eigenvector of the
// (c+1)-th largest (FP32, row pitch ldv, the B operand of U = Q V), sigma_c =
// sqrt(max(W, 0)) and lam_c = W (FP64, all b values descending).
static __global__ void pick_kernel(const double *__restrict__ V, const double *__restrict__ W, int b, int k,
                                   float *__restrict__ Vt, int64_t ldv, double *__restrict__ sigma,
                                   double *__restrict__ lam) {
    const int64_t total = (int64_t)k * b;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(idx / b), i = (int)(idx - (int64_t)c * b);
        const int src = b - 1 - c;
        Vt[(int64_t)c * ldv + i] = (float)V[(int64_t)src * b + i];
        if (i == 0) sigma[c] = sqrt(fmax(W[src], 0.0));
    }
    if (lam != nullptr)
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < b; c += gridDim.x * blockDim.x) lam[c] = W[b - 1 - c];
}

// L_eff column c = U column c times sigma_c (U n x k FP32 in place into L_eff).
static __global__ void scale_cols_kernel(const float *__restrict__ U, int64_t ldu, int n, int k,
                                         const double *__restrict__ sigma, float *__restrict__ L_eff, int64_t ldE) {
    const int64_t total = (int64_t)n * k;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / k), c = (int)(idx - (int64_t)i * k);
        L_eff[(int64_t)i * ldE + c] = (float)((double)U[(int64_t)i * ldu + c] * sigma[c]);
    }
}



// Direct route: V holds all n eigenvectors (column-major, ascending W);
// L_eff column c = eigenvector of the (c+1)-th largest times its sqrt, and
// lam = all n eigenvalues descending.
static __global__ void direct_leff_kernel(const double *__restrict__ V, const double *__restrict__ W, int n, int k,
                                          float *__restrict__ L_eff, int64_t ldE, double *__restrict__ sigma,
                                          double *__restrict__ lam) {
    const int64_t total = (int64_t)n * k;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / k), c = (int)(idx - (int64_t)i * k);
        const int src = n - 1 - c;
        const double sg = sqrt(fmax(W[src], 0.0));
        L_eff[(int64_t)i * ldE + c] = (float)(V[(int64_t)src * n + i] * sg);
        if (i == 0) sigma[c] = sg;
    }
    if (lam != nullptr)
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) lam[c] = W[n - 1 - c];
}

// ------------------------------------------------------------------ plan
struct TopkPlan {
    int64_t n, m, k, b;
    int64_t Wm, Wn, Wb;                 // piece segment widths (multiples of 64) along m, n and b
    bool direct;
    int lwork, lwork_s;
    size_t o_K, o_pl0, o_pl1;           // K (n x Wn FP32); pieces of tilde L (n x 6 Wm, both sides)
    size_t o_Kd, o_W;                   // direct route: FP64 copy of K, its eigenvalues
    size_t o_kp, o_y[3], o_yt0, o_yt1, o_xr;   // iterative route: K pieces, panels, panel pieces
    size_t o_sm[6], o_sp0, o_sp1;       // b x b work matrices and their pieces
    size_t o_D, o_rows, o_s, o_H, o_Wb, o_vt, o_u;
    size_t o_work, o_info, total;
};

static int64_t r64(int64_t x) { return (x + 63) / 64 * 64; }

static int topk_plan(int64_t n, int64_t m, int64_t k, TopkPlan *p) {
    EigLib *E = eig_lib();
    if (!E) return record_message(MV_ERR_UNSUPPORTED, "STR truncation needs cuSOLVER (not found)");
    *p = TopkPlan{};
    p->n = n;
    p->m = m;
    p->k = k;
    p->b = r64(std::max<int64_t>(2 * k, k + 512));
    p->direct = n <= 1024 || p->b >= n;
    if (p->direct) p->b = n;
    p->Wm = r64(m);
    p->Wn = r64(n);
    p->Wb = r64(p->b);
    const int64_t b = p->b;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    p->o_K = take(4 * (size_t)n * p->Wn);
    const size_t shared0 = off;                 // tilde L pieces, then (after K is formed) the rest
    p->o_pl0 = take(2 * (size_t)n * 6 * p->Wm);
    p->o_pl1 = take(2 * (size_t)n * 6 * p->Wm);
    const size_t end_pieces = off;
    off = shared0;
    int lwork = 0;
    if (p->direct) {
        p->o_Kd = take(8 * (size_t)n * n);
        p->o_W = take(8 * (size_t)n);
        if (E->syevd_bs(E->hs, kEigVector, kFillLower, (int)n, nullptr, (int)n, nullptr, &lwork) != 0)
            return record_message(MV_ERR_CUDA, "cusolverDnDsyevd_bufferSize failed");
    } else {
        p->o_kp = take(2 * (size_t)n * 6 * p->Wn);
        for (int i = 0; i < 3; ++i) p->o_y[i] = take(4 * (size_t)n * p->Wb);
        p->o_yt0 = take(2 * (size_t)b * 6 * p->Wn);
        p->o_yt1 = take(2 * (size_t)b * 6 * p->Wn);
        p->o_xr = take(2 * (size_t)n * 6 * p->Wb);
        for (int i = 0; i < 6; ++i) p->o_sm[i] = take(4 * (size_t)b * p->Wb);
        p->o_sp0 = take(2 * (size_t)b * 6 * p->Wb);
        p->o_sp1 = take(2 * (size_t)b * 6 * p->Wb);
        p->o_D = take(4 * (size_t)b);
        p->o_rows = take(4 * (size_t)b);
        p->o_s = take(16);
        p->o_H = take(8 * (size_t)b * b);
        p->o_Wb = take(8 * (size_t)b);
        p->o_vt = take(4 * (size_t)k * p->Wb);
        p->o_u = take(4 * (size_t)n * r64(k));
        if (E->syevd_bs(E->hs, kEigVector, kFillLower, (int)b, nullptr, (int)b, nullptr, &lwork) != 0)
            return record_message(MV_ERR_CUDA, "cusolverDnDsyevd_bufferSize failed");
        int lws = 0;
        if (E->ssyevd_bs(E->hs, kEigNoVector, kFillLower, (int)b, nullptr, (int)b, nullptr, &lws) != 0)
            return record_message(MV_ERR_CUDA, "cusolverDnSsyevd_bufferSize failed");
        p->lwork_s = lws;
        lwork = std::max(lwork, (lws + 1) / 2);
    }
    p->o_work = take(8 * (size_t)lwork);
    p->o_info = take(16);
    p->lwork = lwork;
    p->total = std::max(off, end_pieces);
    return MV_OK;
}

size_t topk_workspace_size(int64_t n, int64_t m, int64_t k) {
    if (n < 1 || m < 1 || k < 1 || k > n || n >= (1 << 30) || m >= (1 << 30)) return 0;
    TopkPlan p;
    if (topk_plan(n, m, k, &p) != MV_OK) return 0;
    return p.total;
}

// ------------------------------------------------------------------ driver
namespace {

struct Ctx {
    const TopkPlan &p;
    char *ws;
    cudaStream_t s;
    template <typename T>
    T *at(size_t off) const { return reinterpret_cast<T *>(ws + off); }
};

static int grid_for(int64_t total) { return (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 16)); }

// Pieces of X (R x cols FP32) as rows (side 0 or 1): R x 6W BF16.
static int split_rows(const Ctx &c, const float *X, int64_t R, int64_t cols, int64_t ldx, int64_t W, int side,
                      __nv_bfloat16 *out) {
    split3_rows_kernel<<<grid_for(R * W), 256, 0, c.s>>>(X, (int)R, (int)cols, ldx, (int)W, side, out, 6 * W);
    MV_CUDA_TRY(cudaGetLastError());
    return MV_OK;
}
// Pieces of X^T (X: R x cols FP32; out: cols x 6W with W >= R).
static int split_t(const Ctx &c, const float *X, int64_t R, int64_t cols, int64_t ldx, int64_t W, int side,
                   __nv_bfloat16 *out) {
    split3_t_kernel<<<dim3((unsigned)((cols + 31) / 32), (unsigned)((W + 31) / 32)), 256, 0, c.s>>>(
        X, (int)R, (int)cols, ldx, (int)W, side, out, 6 * W);
    MV_CUDA_TRY(cudaGetLastError());
    return MV_OK;
}
// C (M x N) = epilogue(A' B'^T) over piece operands of segment width W.
template <int BN>
static int gemm6(const Ctx &c, const __nv_bfloat16 *A, int64_t M, const __nv_bfloat16 *B, int64_t N, int64_t W,
                 float *C, int64_t ldc, const GemmEpi &e = GemmEpi{}) {
    return gemmc<BN>(A, nullptr, M, 6 * W, B, N, 6 * W, 6 * W, C, ldc, e, c.s);
}

// Q = Y (Y^T Y)^{-1/2} (n x b panels, row pitch Wb): Lowdin passes with the
// shifts and Newton--Schulz step counts of kOrthPasses.  Q may be Y.
struct OrthPass {
    float delta;
    int its;
};
constexpr OrthPass kOrthPasses[3] = {{1e-5f, 22}, {1e-7f, 14}, {0.0f, 8}};

static int orth(const Ctx &c, const float *Y, float *Q) {
    const TopkPlan &p = c.p;
    const int64_t n = p.n, b = p.b, Wb = p.Wb, Wn = p.Wn;
    float *G = c.at<float>(p.o_sm[0]), *A = c.at<float>(p.o_sm[1]), *Z = c.at<float>(p.o_sm[2]);
    float *P = c.at<float>(p.o_sm[3]), *Tm = c.at<float>(p.o_sm[4]), *A2 = c.at<float>(p.o_sm[5]);
    __nv_bfloat16 *yt0 = c.at<__nv_bfloat16>(p.o_yt0), *yt1 = c.at<__nv_bfloat16>(p.o_yt1);
    __nv_bfloat16 *sp0 = c.at<__nv_bfloat16>(p.o_sp0), *sp1 = c.at<__nv_bfloat16>(p.o_sp1);
    __nv_bfloat16 *xr = c.at<__nv_bfloat16>(p.o_xr);
    float *D = c.at<float>(p.o_D), *rows = c.at<float>(p.o_rows), *sc = c.at<float>(p.o_s);
    const float *src = Y;
    for (const OrthPass &ps : kOrthPasses) {
        // G = src^T src
        MV_TRY(split_t(c, src, n, b, Wb, Wn, 0, yt0));
        MV_TRY(split_t(c, src, n, b, Wb, Wn, 1, yt1));
        MV_TRY(gemm6<128>(c, yt0, b, yt1, b, Wn, G, Wb));
        lowdin_rows_kernel<<<(unsigned)b, 256, 0, c.s>>>(G, (int)b, Wb, D, rows);
        lowdin_start_kernel<<<grid_for(b * b), 256, 0, c.s>>>(G, (int)b, Wb, D, rows, ps.delta, A, Z, sc);
        MV_CUDA_TRY(cudaGetLastError());
        float *Ya = A, *Yb = A2;
        const int its = ps.its;
        for (int it = 0; it < its; ++it) {
            // P = Z Ya; T = (3I - P)/2; Yb = Ya T; Z <- T Z.  C = A B^T with A's rows and
            // the right factor's columns (its transposed pieces): no product relies on a
            // symmetry that rounding only keeps approximately.
            MV_TRY(split_rows(c, Z, b, b, Wb, Wb, 0, sp0));
            MV_TRY(split_t(c, Ya, b, b, Wb, Wb, 1, sp1));
            MV_TRY(gemm6<128>(c, sp0, b, sp1, b, Wb, P, Wb));
            ns_t_kernel<<<grid_for(b * b), 256, 0, c.s>>>(P, (int)b, Wb, Tm);
            MV_TRY(split_rows(c, Ya, b, b, Wb, Wb, 0, sp0));
            MV_TRY(split_t(c, Tm, b, b, Wb, Wb, 1, sp1));
            MV_TRY(gemm6<128>(c, sp0, b, sp1, b, Wb, Yb, Wb));
            MV_TRY(split_rows(c, Tm, b, b, Wb, Wb, 0, sp0));
            MV_TRY(split_t(c, Z, b, b, Wb, Wb, 1, sp1));
            MV_TRY(gemm6<128>(c, sp0, b, sp1, b, Wb, P, Wb));      // P = T Z
            std::swap(Ya, Yb);
            std::swap(Z, P);
        }
        // Q = src M, M = D Z / sqrt(s)
        lowdin_m_kernel<<<grid_for(b * b), 256, 0, c.s>>>(D, Z, (int)b, Wb, sc, Tm);
        MV_CUDA_TRY(cudaGetLastError());
        MV_TRY(split_rows(c, src, n, b, Wb, Wb, 0, xr));
        MV_TRY(split_t(c, Tm, b, b, Wb, Wb, 1, sp1));
        MV_TRY(gemm6<128>(c, xr, n, sp1, b, Wb, Q, Wb));   // reads only the pieces: Q may be src
        src = Q;
        Z = c.at<float>(p.o_sm[2]);                         // the swaps may have moved the names
        P = c.at<float>(p.o_sm[3]);
    }
    return MV_OK;
}

}  // namespace

namespace {

// The eigensolver on the b x b (or n x n) FP64 matrix Hd in place.
static int syevd(const TopkPlan &p, char *ws, double *Hd, int64_t dim, double *W, bool vectors, cudaStream_t s) {
    EigLib *E = eig_lib();
    int *info = reinterpret_cast<int *>(ws + p.o_info);
    if (E->syevd(E->hs, vectors ? kEigVector : kEigNoVector, kFillLower, (int)dim, Hd, (int)dim, W,
                 reinterpret_cast<double *>(ws + p.o_work), p.lwork, info) != 0)
        return record_message(MV_ERR_CUDA, "cusolverDnDsyevd failed");
    int hinfo = 0;
    MV_CUDA_TRY(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s));
    MV_CUDA_TRY(cudaStreamSynchronize(s));
    if (hinfo != 0) {
        char msg[96];
        snprintf(msg, sizeof(msg), "cusolverDnDsyevd: info=%d", hinfo);
        return record_message(MV_ERR_NUMERIC, msg);
    }
    // a non-finite entry upstream would otherwise reach sigma as sqrt(max(NaN, 0)) = 0
    std::vector<double> w((size_t)dim);
    MV_CUDA_TRY(cudaMemcpyAsync(w.data(), W, 8 * (size_t)dim, cudaMemcpyDeviceToHost, s));
    MV_CUDA_TRY(cudaStreamSynchronize(s));
    for (double v : w)
        if (!std::isfinite(v)) return record_message(MV_ERR_NUMERIC, "STR truncation: non-finite eigenvalue");
    return MV_OK;
}

// orth() is some 400 small launches; it is captured once per (workspace,
// shape, source, destination) into a CUDA graph -- on a private stream, so
// that the caller's stream may be the legacy default one -- and replayed.
struct OrthKey {
    const void *ws, *src, *dst;
    int64_t n, b, Wn, Wb;
    int dev;
    bool operator==(const OrthKey &o) const {
        return ws == o.ws && src == o.src && dst == o.dst && n == o.n && b == o.b && Wn == o.Wn && Wb == o.Wb &&
               dev == o.dev;
    }
};
static std::mutex g_orth_mu;
static std::vector<std::pair<OrthKey, cudaGraphExec_t>> g_orth_graphs;

static int orth_graph(const Ctx &c, const float *Y, float *Q) {
    int dev = 0;
    MV_CUDA_TRY(cudaGetDevice(&dev));
    const OrthKey key{c.ws, Y, Q, c.p.n, c.p.b, c.p.Wn, c.p.Wb, dev};
    std::lock_guard<std::mutex> lock(g_orth_mu);
    cudaGraphExec_t exec = nullptr;
    for (auto &kv : g_orth_graphs)
        if (kv.first == key) exec = kv.second;
    if (exec == nullptr) {
        MV_TRY((gemmc_set_attrs<128, 1>()));
        cudaStream_t cs;
        MV_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaStreamDestroy(cs);
            return record_message(MV_ERR_CUDA, "STR truncation: stream capture refused");
        }
        const Ctx cc{c.p, c.ws, cs};
        const int st = orth(cc, Y, Q);
        cudaGraph_t graph;
        const cudaError_t e = cudaStreamEndCapture(cs, &graph);
        cudaStreamDestroy(cs);
        if (st != MV_OK) {
            if (e == cudaSuccess) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return record_cuda_error(e, "cudaStreamEndCapture", __FILE__, __LINE__);
        const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) return record_cuda_error(ei, "cudaGraphInstantiate", __FILE__, __LINE__);
        if (g_orth_graphs.size() >= 16) {
            for (auto &kv : g_orth_graphs) cudaGraphExecDestroy(kv.second);
            g_orth_graphs.clear();
        }
        g_orth_graphs.emplace_back(key, exec);
    }
    MV_CUDA_TRY(cudaGraphLaunch(exec, c.s));
    return MV_OK;
}

// Eigenvalues only, in FP32, of the b x b matrix in H (row pitch Wb): they
// place the Chebyshev filter's cut, which needs no more accuracy.
static int ssyevd_values(const TopkPlan &p, char *ws, const float *H, float *Wout, cudaStream_t s) {
    EigLib *E = eig_lib();
    float *Hs = reinterpret_cast<float *>(ws + p.o_H);
    sym_f32_kernel<<<grid_for(p.b * p.b), 256, 0, s>>>(H, (int)p.b, p.Wb, Hs);
    MV_CUDA_TRY(cudaGetLastError());
    int *info = reinterpret_cast<int *>(ws + p.o_info);
    if (E->ssyevd(E->hs, kEigNoVector, kFillLower, (int)p.b, Hs, (int)p.b, Wout,
                  reinterpret_cast<float *>(ws + p.o_work), p.lwork_s, info) != 0)
        return record_message(MV_ERR_CUDA, "cusolverDnSsyevd failed");
    int hinfo = 0;
    MV_CUDA_TRY(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s));
    MV_CUDA_TRY(cudaStreamSynchronize(s));
    if (hinfo != 0) {
        char msg[96];
        snprintf(msg, sizeof(msg), "cusolverDnSsyevd: info=%d", hinfo);
        return record_message(MV_ERR_NUMERIC, msg);
    }
    return MV_OK;
}

// Rayleigh--Ritz matrix of the orthonormal panel Q: KQ into Wk, then
// H = Q^T (K Q) widened to FP64 (symmetrised) in p.o_H.
static int rayleigh(const Ctx &c, const float *Q, float *Wk) {
    const TopkPlan &p = c.p;
    const int64_t n = p.n, b = p.b, Wb = p.Wb, Wn = p.Wn;
    __nv_bfloat16 *kp = c.at<__nv_bfloat16>(p.o_kp);
    __nv_bfloat16 *yt0 = c.at<__nv_bfloat16>(p.o_yt0), *yt1 = c.at<__nv_bfloat16>(p.o_yt1);
    MV_TRY(split_t(c, Q, n, b, Wb, Wn, 1, yt1));
    MV_TRY(gemm6<128>(c, kp, n, yt1, b, Wn, Wk, Wb));
    MV_TRY(split_t(c, Q, n, b, Wb, Wn, 0, yt0));
    MV_TRY(split_t(c, Wk, n, b, Wb, Wn, 1, yt1));
    float *H = c.at<float>(p.o_sm[0]);
    MV_TRY(gemm6<128>(c, yt0, b, yt1, b, Wn, H, Wb));
    widen_sym_kernel<<<grid_for(b * b), 256, 0, c.s>>>(H, (int)b, Wb, c.at<double>(p.o_H));
    MV_CUDA_TRY(cudaGetLastError());
    return MV_OK;
}

constexpr int kDegrees[] = {5, 5, 3};             // Chebyshev degree schedule

}  // namespace

int topk_eigen(const float *Ls, int64_t n, int64_t m, int64_t ldS, int64_t k, float *L_eff, int64_t ldE,
               double *sigma, double *lam, int64_t *n_lam, void *d_ws, size_t ws_bytes, cudaStream_t s) {
    TopkPlan p;
    MV_TRY(topk_plan(n, m, k, &p));
    if (d_ws == nullptr || ws_bytes < p.total || ((uintptr_t)d_ws) % 256) return MV_ERR_WORKSPACE;
    EigLib *E = eig_lib();
    if (E->set_stream(E->hs, s) != 0) return record_message(MV_ERR_CUDA, "cusolverDnSetStream failed");
    char *ws = reinterpret_cast<char *>(d_ws);
    const Ctx c{p, ws, s};
    const int64_t b = p.b, Wb = p.Wb, Wn = p.Wn;
    MV_TRY(gemm_err_clear(s));
    // 1. K = tilde L tilde L^T
    float *K = c.at<float>(p.o_K);
    __nv_bfloat16 *pl0 = c.at<__nv_bfloat16>(p.o_pl0), *pl1 = c.at<__nv_bfloat16>(p.o_pl1);
    MV_TRY(split_rows(c, Ls, n, m, ldS, p.Wm, 0, pl0));
    MV_TRY(split_rows(c, Ls, n, m, ldS, p.Wm, 1, pl1));
    MV_TRY(gemm6<256>(c, pl0, n, pl1, n, p.Wm, K, Wn));
    if (p.direct) {
        double *Kd = c.at<double>(p.o_Kd), *W = c.at<double>(p.o_W);
        widen_sym_kernel<<<grid_for(n * n), 256, 0, s>>>(K, (int)n, Wn, Kd);
        MV_CUDA_TRY(cudaGetLastError());
        MV_TRY(syevd(p, ws, Kd, n, W, true, s));
        direct_leff_kernel<<<grid_for(n * k), 256, 0, s>>>(Kd, W, (int)n, (int)k, L_eff, ldE, sigma, lam);
        MV_CUDA_TRY(cudaGetLastError());
        if (n_lam) *n_lam = n;
        return gemm_err_check(s, "STR truncation");
    }
    // 2. random start (a Gaussian block is well conditioned as it stands); two power steps
    float *Y[3] = {c.at<float>(p.o_y[0]), c.at<float>(p.o_y[1]), c.at<float>(p.o_y[2])};
    __nv_bfloat16 *kp = c.at<__nv_bfloat16>(p.o_kp), *yt1 = c.at<__nv_bfloat16>(p.o_yt1);
    MV_TRY(split_rows(c, K, n, n, Wn, Wn, 0, kp));
    randn_kernel<<<grid_for(n * b), 256, 0, s>>>(0x5EEDu, 0x57Au, (int)n, (int)b, Wb, Y[0]);
    MV_CUDA_TRY(cudaGetLastError());
    for (int it = 0; it < 2; ++it) {
        float *src = Y[it & 1], *dst = Y[(it + 1) & 1];
        MV_TRY(split_t(c, src, n, b, Wb, Wn, 1, yt1));
        MV_TRY(gemm6<128>(c, kp, n, yt1, b, Wn, dst, Wb));
    }
    MV_TRY(orth_graph(c, Y[0], Y[0]));
    // 3. the cut from the Ritz values
    double *Wv = c.at<double>(p.o_Wb);
    MV_TRY(rayleigh(c, Y[0], Y[1]));
    float *Wf = reinterpret_cast<float *>(Wv);
    MV_TRY(ssyevd_values(p, ws, c.at<float>(p.o_sm[0]), Wf, s));
    std::vector<float> theta(b);
    MV_CUDA_TRY(cudaMemcpyAsync(theta.data(), Wf, 4 * (size_t)b, cudaMemcpyDeviceToHost, s));
    MV_CUDA_TRY(cudaStreamSynchronize(s));
    const double cut = theta[b - 1 - (k + b) / 2];       // ascending order: index from the top
    if (!(cut > 0.0)) return record_message(MV_ERR_NUMERIC, "STR truncation: non-positive Ritz value at the cut");
    const double e = 0.5 * cut, h = 0.5 * cut;
    // 4. Chebyshev filtering on [0, cut]
    for (int d : kDegrees) {
        float *prev = Y[0], *cur = Y[1], *nxt = Y[2];
        GemmEpi e1;
        e1.alpha = (float)(1.0 / h);
        e1.X1 = prev;
        e1.ld1 = Wb;
        e1.beta = (float)(-e / h);
        MV_TRY(split_t(c, prev, n, b, Wb, Wn, 1, yt1));
        MV_TRY(gemm6<128>(c, kp, n, yt1, b, Wn, cur, Wb, e1));
        for (int j = 1; j < d; ++j) {
            GemmEpi e2;
            e2.alpha = (float)(2.0 / h);
            e2.X1 = cur;
            e2.ld1 = Wb;
            e2.beta = (float)(-2.0 * e / h);
            e2.X2 = prev;
            e2.ld2 = Wb;
            e2.gamma = -1.0f;
            MV_TRY(split_t(c, cur, n, b, Wb, Wn, 1, yt1));
            MV_TRY(gemm6<128>(c, kp, n, yt1, b, Wn, nxt, Wb, e2));
            float *t = prev;
            prev = cur;
            cur = nxt;
            nxt = t;
        }
        MV_TRY(orth_graph(c, cur, Y[0]));
    }
    // 5. final Rayleigh--Ritz
    MV_TRY(rayleigh(c, Y[0], Y[1]));
    double *Hd = c.at<double>(p.o_H);
    MV_TRY(syevd(p, ws, Hd, b, Wv, true, s));
    float *Vt = c.at<float>(p.o_vt);
    pick_kernel<<<grid_for(k * b), 256, 0, s>>>(Hd, Wv, (int)b, (int)k, Vt, Wb, sigma, lam);
    MV_CUDA_TRY(cudaGetLastError());
    __nv_bfloat16 *xr = c.at<__nv_bfloat16>(p.o_xr), *sp1 = c.at<__nv_bfloat16>(p.o_sp1);
    float *U = c.at<float>(p.o_u);
    MV_TRY(split_rows(c, Y[0], n, b, Wb, Wb, 0, xr));
    MV_TRY(split_rows(c, Vt, k, b, Wb, Wb, 1, sp1));
    MV_TRY(gemm6<128>(c, xr, n, sp1, k, Wb, U, r64(k)));
    scale_cols_kernel<<<grid_for(n * k), 256, 0, s>>>(U, r64(k), (int)n, (int)k, sigma, L_eff, ldE);
    MV_CUDA_TRY(cudaGetLastError());
    if (n_lam) *n_lam = b;
    return gemm_err_check(s, "STR truncation");
}

}  // namespace mv
