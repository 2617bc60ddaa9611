// Efficient frontier (batched NPGA over many targets sharing one factor)
// and its FP32 refinement.
#include "solve_internal.cuh"

using namespace mv;

// ---------------------------------------------------------------------------
// Efficient frontier: B targets R_b share one factor L (BF16, or FP8 e4m3
// with row scales s: then the GEMMs read FP8 tiles expanded to BF16 in
// shared memory (gemm_q8.cuh), s multiplies the split Y operand, since
// L^T Y = L_q^T (s o Y), and the rows of G, since L Z = s o (L_q Z)).  The two
// half-products of all B gradients become skinny tensor-core GEMMs:
//   Z (T x B) = L^T Y,   G (n x B) = L Z,
// run on tcgen05 (gemm.cuh) with the n x B and T x B operands carried as a
// BF16 hi + lo pair (2B columns; the GEMM epilogue adds each pair), so the
// only rounding beyond FP32 accumulation is the BF16 storage of L itself.
// L^T is materialised once per call in the workspace so that both GEMMs
// read K-major operands.  Each target then takes its own NPGA step (a
// cluster per target) with its own KKT test and stops independently.
namespace mv {

struct FState {
    int k, done, converged, status;
    int proj_fail, proj_steps, pad0, pad1;
    double t, beta_prev, kkt, nu, tau, nu_kkt, tau_kkt, objective;
};

struct FArgs {
    FState *fs;
    const SolveState *st;       // alpha, mu_min, mu_max of the shared factor
    const float *G;             // n x 2B: hi and lo halves of L Z
    int ldG, B;
    double *X, *Y, *GX;         // B x n (row b = target b)
    __nv_bfloat16 *Ysplit;      // 2B x ldY: BF16 hi rows 0..B-1, lo rows B..2B-1
    int64_t ldY;
    const float *row_scale;     // FP8 factor: n scales (else null)
    const double *mu, *Rt;
    int n, mode, kkt_every, max_iter;
    double gamma, eps;
};

__device__ __forceinline__ void write_split(__nv_bfloat16 *Ys, int64_t ldY, int B, int b, int i, double y,
                                            const float *rs = nullptr) {
    const float yf = (float)(rs != nullptr ? y * (double)rs[i] : y);
    const __nv_bfloat16 hi = __float2bfloat16_rn(yf);
    Ys[(int64_t)b * ldY + i] = hi;
    Ys[(int64_t)(B + b) * ldY + i] = __float2bfloat16_rn(yf - __bfloat162float(hi));
}

template <int CL>
__global__ void __launch_bounds__(kProjNT) frontier_init_kernel(FArgs a) {
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ ProjSmem psm;
    const int b = blockIdx.x / CL, rank = cluster_rank<CL>();
    const int n = a.n, nl = (n + CL - 1) / CL, r0 = min(n, rank * nl), r1 = min(n, r0 + nl);
    ProjElems el = carve_elems(dsm, nl);
    el.n = r1 - r0;
    proj_smem_init(&psm);
    for (int i = threadIdx.x; i < el.n; i += kProjNT) {
        el.v[i] = 1.0 / n;
        el.mu[i] = a.mu[r0 + i];
    }
    __syncthreads();
    ClusterProj<CL> P{&psm, el};
    P.prepare();
    const ProjOut o = P.solve(a.Rt[b], a.mode, a.st->mu_min, a.st->mu_max, 0.0, -INFINITY, kProjBudget);
    const bool bad = (o.status == MV_ERR_INFEASIBLE || o.status == MV_ERR_NUMERIC);
    for (int i = threadIdx.x; i < el.n; i += kProjNT) {
        const int gi = r0 + i;
        const double xi = bad ? 0.0 : fmax(fma(o.nu, el.mu[i], el.v[i]) - o.tau, 0.0);
        a.X[(int64_t)b * n + gi] = xi;
        a.Y[(int64_t)b * n + gi] = xi;
        write_split(a.Ysplit, a.ldY, a.B, b, gi, xi, a.row_scale);
    }
    if (rank == 0 && threadIdx.x == 0) {
        FState f{};
        f.t = 1.0;
        f.nu = f.nu_kkt = o.nu;
        f.tau = f.tau_kkt = o.tau;
        f.kkt = INFINITY;
        f.status = bad ? o.status : (a.st->status != MV_OK ? a.st->status : MV_OK);
        f.done = (f.status != MV_OK) ? 1 : 0;
        a.fs[b] = f;
    }
    cluster_barrier<CL>();
}

template <int CL>
__global__ void __launch_bounds__(kProjNT) frontier_step_kernel(FArgs a) {
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ ProjSmem psm;
    __shared__ double sc[4];
    const int b = blockIdx.x / CL, rank = cluster_rank<CL>();
    FState *fs = a.fs + b;
    if (*(volatile int *)&fs->done) return;      // uniform over the cluster (see npga_step_kernel)
    const int n = a.n, nl = (n + CL - 1) / CL, r0 = min(n, rank * nl), r1 = min(n, r0 + nl);
    const int k = fs->k;
    const double beta_prev = fs->beta_prev, t = fs->t, alpha = a.st->alpha;
    const double mn = a.st->mu_min, mx = a.st->mu_max;
    const double nu0 = fs->nu, tau0 = fs->tau;
    const double gamma = a.gamma, R = a.Rt[b];
    if (threadIdx.x == 0) {
        sc[0] = 1.0 / (1.0 + beta_prev);
        const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        sc[1] = tn;
        sc[2] = (t - 1.0) / tn;
    }
    ProjElems el = carve_elems(dsm, nl);
    el.n = r1 - r0;
    proj_smem_init(&psm);
    const double inv1pb = sc[0], tn = sc[1], beta = sc[2];
    const bool check = (a.kkt_every > 0 && k % a.kkt_every == 0) || (k >= a.max_iter);
    double *Xb = a.X + (int64_t)b * n, *Yb = a.Y + (int64_t)b * n, *GXb = a.GX + (int64_t)b * n;
    for (int i = threadIdx.x; i < el.n; i += kProjNT) {
        const int gi = r0 + i;
        el.mu[i] = a.mu[gi];
        const double gyi = ((double)a.G[(int64_t)gi * a.ldG + b] + (double)a.G[(int64_t)gi * a.ldG + a.B + b]) *
                           (a.row_scale != nullptr ? (double)a.row_scale[gi] : 1.0);
        const double gxi = (k == 0) ? gyi : (gyi + beta_prev * GXb[gi]) * inv1pb;
        GXb[gi] = gxi;
        if (check) {
            const double xi = Xb[gi];
            el.v[i] = xi - alpha * (2.0 * gxi + 2.0 * gamma * xi);
        }
    }
    __syncthreads();
    ClusterProj<CL> P{&psm, el};
    if (check) {
        P.prepare();
        const ProjOut o = P.solve(R, a.mode, mn, mx, nu0, tau0, kProjBudget);   // see npga_step_body
        double r2 = 0.0;
        for (int i = threadIdx.x; i < el.n; i += kProjNT) {
            const double p = fmax(fma(o.nu, el.mu[i], el.v[i]) - o.tau, 0.0);
            const double d = p - Xb[r0 + i];
            r2 = fma(d, d, r2);
        }
        r2 = P.reduce_double(r2);
        const bool conv = r2 <= a.eps * a.eps;
        const bool stop = conv || k >= a.max_iter || !(r2 == r2);
        if (rank == 0 && threadIdx.x == 0) {
            fs->kkt = sqrt(r2);
            fs->nu_kkt = o.nu;
            fs->tau_kkt = o.tau;
            fs->proj_steps += o.steps;
            if (o.status != MV_OK) fs->proj_fail += 1;
            if (stop) {
                fs->done = 1;
                fs->converged = conv ? 1 : 0;
                fs->status = conv ? MV_OK : (!(r2 == r2) ? MV_ERR_NUMERIC : MV_ERR_NOT_CONVERGED);
            }
        }
        if (stop) {
            cluster_barrier<CL>();
            return;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < el.n; i += kProjNT) {
        const int gi = r0 + i;
        const double gyi = ((double)a.G[(int64_t)gi * a.ldG + b] + (double)a.G[(int64_t)gi * a.ldG + a.B + b]) *
                           (a.row_scale != nullptr ? (double)a.row_scale[gi] : 1.0);
        const double yi = Yb[gi];
        el.v[i] = yi - alpha * (2.0 * gyi + 2.0 * gamma * yi);
    }
    __syncthreads();
    P.prepare();
    const ProjOut o = P.solve(R, a.mode, mn, mx, nu0, tau0, kProjBudget);
    for (int i = threadIdx.x; i < el.n; i += kProjNT) {
        const int gi = r0 + i;
        const double xn = fmax(fma(o.nu, el.mu[i], el.v[i]) - o.tau, 0.0);
        const double xo = Xb[gi];
        const double yn = xn + beta * (xn - xo);
        Xb[gi] = xn;
        Yb[gi] = yn;
        write_split(a.Ysplit, a.ldY, a.B, b, gi, yn, a.row_scale);
    }
    if (rank == 0 && threadIdx.x == 0) {
        fs->t = tn;
        fs->beta_prev = beta;
        fs->k = k + 1;
        fs->nu = o.nu;
        fs->tau = o.tau;
        fs->proj_steps += o.steps;
        if (o.status != MV_OK) fs->proj_fail += 1;
        if (o.status == MV_ERR_INFEASIBLE || o.status == MV_ERR_NUMERIC) {
            fs->done = 1;
            fs->status = o.status;
        }
    }
    cluster_barrier<CL>();
}

// L (n x T, ld ldL) -> L^T (T x n, ld ldT), BF16, 32x32 tiles through shared memory.
template <typename E>
__global__ void transpose_elem_kernel(const E *__restrict__ L, int n, int T, int64_t ldL, E *__restrict__ Lt,
                                      int64_t ldT) {
    __shared__ E tile[32][33];
    const int t0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = i0 + r, t = t0 + threadIdx.x;
        tile[r][threadIdx.x] = (i < n && t < T) ? L[(int64_t)i * ldL + t] : E{};
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int t = t0 + r, i = i0 + threadIdx.x;
        if (t < T && i < n) Lt[(int64_t)t * ldT + i] = tile[threadIdx.x][r];
    }
}

// The FP32 factor as a BF16 pair: H = bf16(L), D = bf16(L - H), so that
// H + D carries L to 2^-18 of each entry (n x T, row pitches ld and ldo).
__global__ void hilo_kernel(const float *__restrict__ L, int n, int T, int64_t ld, __nv_bfloat16 *__restrict__ H,
                            __nv_bfloat16 *__restrict__ D, int64_t ldo) {
    const int64_t total = (int64_t)n * ldo;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / ldo), t = (int)(idx - (int64_t)i * ldo);
        const float x = t < T ? L[(int64_t)i * ld + t] : 0.0f;
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        H[idx] = h;
        D[idx] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
}

// Restart of every unfinished target from its current x (the refinement
// phase): y = x, t = 1, k = 0, the split operand rewritten from y (no row
// scales: the refined model is the FP32 factor itself).  Targets whose first
// phase failed (infeasible, numeric) keep their status.  One block per target.
__global__ void frontier_warm_kernel(FState *fs, const double *__restrict__ X, double *__restrict__ Y, int n, int B,
                                     __nv_bfloat16 *__restrict__ Ys, int64_t ldY) {
    const int b = blockIdx.x;
    const bool failed = fs[b].status == MV_ERR_INFEASIBLE || fs[b].status == MV_ERR_NUMERIC;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double x = X[(int64_t)b * n + i];
        Y[(int64_t)b * n + i] = x;
        write_split(Ys, ldY, B, b, i, x, nullptr);
    }
    if (threadIdx.x == 0 && !failed) {
        FState &f = fs[b];
        f.k = 0;
        f.done = 0;
        f.converged = 0;
        f.status = MV_OK;
        f.t = 1.0;
        f.beta_prev = 0.0;
        f.kkt = INFINITY;
    }
}

// Rows of X (B x n, FP64) -> the BF16 hi/lo operand rows (2B x ldY).
__global__ void split_rows_kernel(const double *__restrict__ X, int B, int n, __nv_bfloat16 *__restrict__ Ys,
                                  int64_t ldY, const float *__restrict__ rs) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)B * n) return;
    const int b = (int)(idx / n), i = (int)(idx - (int64_t)b * n);
    write_split(Ys, ldY, B, b, i, X[idx], rs);
}

// f_b = ||L^T x_b||^2 + gamma ||x_b||^2 from Z = L^T X carried as BF16 hi + lo rows.
__global__ void __launch_bounds__(kStepThreads)
frontier_objective_kernel(const __nv_bfloat16 *__restrict__ Zt, int64_t ldZ, int B, int T,
                          const double *__restrict__ X, int n, double gamma, FState *fs) {
    __shared__ double red[(kStepThreads / kWarp + 1) * 5];
    const int b = blockIdx.x;
    float s = 0.f, c = 0.f;
    for (int t = threadIdx.x; t < T; t += kStepThreads) {
        const float z = __bfloat162float(Zt[(int64_t)b * ldZ + t]) + __bfloat162float(Zt[(int64_t)(B + b) * ldZ + t]);
        const float y = fmaf(z, z, -c);
        const float u = s + y;
        c = (u - s) - y;
        s = u;
    }
    double v[2] = {(double)s - (double)c, 0.0};
    if (gamma != 0.0)
        for (int i = threadIdx.x; i < n; i += kStepThreads) v[1] = fma(X[(int64_t)b * n + i], X[(int64_t)b * n + i], v[1]);
    block_sum<2, kStepThreads>(v, red);
    if (threadIdx.x == 0) fs[b].objective = v[0] + gamma * v[1];
}

template <int CL>
static cudaError_t launch_frontier_kernel(bool init, const FArgs &a, int B, int n, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(B * CL));
    cfg.blockDim = dim3(kProjNT);
    cfg.dynamicSmemBytes = proj_elem_bytes((n + CL - 1) / CL);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (init) return cudaLaunchKernelEx(&cfg, frontier_init_kernel<CL>, a);
    return cudaLaunchKernelEx(&cfg, frontier_step_kernel<CL>, a);
}

static cudaError_t launch_frontier(bool init, int CL, const FArgs &a, cudaStream_t s) {
    switch (CL) {
        case 1: return launch_frontier_kernel<1>(init, a, a.B, a.n, s);
        case 2: return launch_frontier_kernel<2>(init, a, a.B, a.n, s);
        case 4: return launch_frontier_kernel<4>(init, a, a.B, a.n, s);
        case 8: return launch_frontier_kernel<8>(init, a, a.B, a.n, s);
        default: return launch_frontier_kernel<16>(init, a, a.B, a.n, s);
    }
}

static int frontier_attrs() {
    static std::once_flag once;
    static int st = MV_OK;
    std::call_once(once, [] {
        bool ok = cluster_attrs(frontier_init_kernel<1>, 1) && cluster_attrs(frontier_init_kernel<2>, 2) &&
                  cluster_attrs(frontier_init_kernel<4>, 4) && cluster_attrs(frontier_init_kernel<8>, 8) &&
                  cluster_attrs(frontier_init_kernel<16>, 16) && cluster_attrs(frontier_step_kernel<1>, 1) &&
                  cluster_attrs(frontier_step_kernel<2>, 2) && cluster_attrs(frontier_step_kernel<4>, 4) &&
                  cluster_attrs(frontier_step_kernel<8>, 8) && cluster_attrs(frontier_step_kernel<16>, 16);
        ok = ok && gemm_set_attrs<64, kEpiF32>() == MV_OK && gemm_set_attrs<128, kEpiF32>() == MV_OK &&
             gemm_set_attrs<256, kEpiF32>() == MV_OK && gemm_set_attrs<64, kEpiPairSplitT>() == MV_OK &&
             gemm_set_attrs<128, kEpiPairSplitT>() == MV_OK && gemm_set_attrs<256, kEpiPairSplitT>() == MV_OK;
        ok = ok && gemm_set_attrs<64, kEpiF32, 2>() == MV_OK && gemm_set_attrs<128, kEpiF32, 2>() == MV_OK &&
             gemm_set_attrs<256, kEpiF32, 2>() == MV_OK && gemm_set_attrs<64, kEpiPairSplitT, 2>() == MV_OK &&
             gemm_set_attrs<128, kEpiPairSplitT, 2>() == MV_OK && gemm_set_attrs<256, kEpiPairSplitT, 2>() == MV_OK;
        ok = ok && gemm_q8_set_attrs<64, kEpiF32>() == MV_OK && gemm_q8_set_attrs<128, kEpiF32>() == MV_OK &&
             gemm_q8_set_attrs<256, kEpiF32>() == MV_OK && gemm_q8_set_attrs<64, kEpiPairSplitT>() == MV_OK &&
             gemm_q8_set_attrs<128, kEpiPairSplitT>() == MV_OK && gemm_q8_set_attrs<256, kEpiPairSplitT>() == MV_OK;
        if (!ok) st = record_cuda_error(cudaGetLastError(), "frontier kernel attributes", __FILE__, __LINE__);
    });
    return st;
}

struct FPlan {
    int B;          // padded target count (32, 64 or 128)
    int BN;         // 2B: GEMM tile width
    int splits;     // K-splits of G = L Z (43 row tiles at n = 5440 would leave SMs idle)
    int64_t ldLt, ldY, ldZ;
    size_t o_lt, o_y, o_z, o_g, o_x, o_yd, o_gx, o_fs, o_rt, o_gpart, o_gtick;
    // FP32 refinement: BF16 hi and lo parts of the FP32 factor, n x ldH, and their transposes
    int64_t ldH;
    size_t o_h, o_d, o_ht, o_dt;
    size_t total;
};

static FPlan make_fplan(const Plan &p, int64_t nb, bool refine = false) {
    // The power method runs on the transposed copy: its plan's scratch comes first too.
    const Plan pt = make_plan(p.dt, p.n, p.T, (p.n + 15) / 16 * 16, 0, true, true);
    FPlan f{};
    f.B = nb <= 32 ? 32 : (nb <= 64 ? 64 : 128);
    f.BN = 2 * f.B;
    f.ldLt = (p.n + 15) / 16 * 16;                    // row pitch a multiple of 16 bytes for BF16 and FP8
    f.ldY = f.ldLt;
    f.ldZ = ((int64_t)p.T + 7) / 8 * 8;
    size_t off = std::max(p.total, pt.total);
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    f.o_lt = take((size_t)p.esize * p.T * f.ldLt);
    f.o_y = take(2 * (size_t)f.BN * f.ldY);
    f.o_z = take(2 * (size_t)f.BN * f.ldZ);
    f.o_g = take(4 * (size_t)p.n * f.BN);
    f.o_x = take(8 * (size_t)f.B * p.n);
    f.o_yd = take(8 * (size_t)f.B * p.n);
    f.o_gx = take(8 * (size_t)f.B * p.n);
    f.o_fs = take(sizeof(FState) * (size_t)f.B);
    f.o_rt = take(8 * (size_t)f.B);
    f.splits = gemm_splits(p.n, f.BN, p.T, f.BN, sm_count());
    f.o_gpart = take(4 * (size_t)f.splits * p.n * f.BN);
    f.o_gtick = take(4 * (size_t)((p.n + kBM - 1) / kBM) + 64);
    f.ldH = ((int64_t)p.T + 7) / 8 * 8;
    if (refine) {
        f.o_h = take(2 * (size_t)p.n * f.ldH);
        f.o_d = take(2 * (size_t)p.n * f.ldH);
        f.o_ht = take(2 * (size_t)p.T * f.ldLt);
        f.o_dt = take(2 * (size_t)p.T * f.ldLt);
    }
    f.total = off;
    return f;
}

template <int BN>
static void frontier_gemms(const CUtensorMap &tLt, const CUtensorMap &tY, const CUtensorMap &tL, const CUtensorMap &tZ,
                           const Plan &p, const FPlan &f, void *ws, cudaStream_t s) {
    float *gpart = at<float>(ws, f.o_gpart);
    unsigned *gtick = at<unsigned>(ws, f.o_gtick);
    if (p.dt == MV_FP8_E4M3) {
        gemm_q8_launch<BN, kEpiPairSplitT>(tLt, tY, p.T, f.BN, p.n, nullptr, 0, at<__nv_bfloat16>(ws, f.o_z), f.ldZ,
                                           s);
        gemm_q8_launch<BN, kEpiF32>(tL, tZ, p.n, f.BN, p.T, at<float>(ws, f.o_g), f.BN, nullptr, 0, s, f.splits,
                                    gpart, gtick);
        return;
    }
    gemm_launch<BN, kEpiPairSplitT>(tLt, tY, p.T, f.BN, p.n, nullptr, 0, at<__nv_bfloat16>(ws, f.o_z), f.ldZ, s);
    gemm_launch<BN, kEpiF32>(tL, tZ, p.n, f.BN, p.T, at<float>(ws, f.o_g), f.BN, nullptr, 0, s, f.splits, gpart,
                             gtick);
}

// The FP32-accurate pair: A = hi + lo (maps[0] + maps[4] for L^T, maps[2] + maps[5] for L).
template <int BN>
static void frontier_gemms2(const CUtensorMap *maps, const Plan &p, const FPlan &f, void *ws, cudaStream_t s) {
    gemm_launch<BN, kEpiPairSplitT, 2>(maps[0], maps[1], p.T, f.BN, p.n, nullptr, 0, at<__nv_bfloat16>(ws, f.o_z),
                                       f.ldZ, s, 1, nullptr, nullptr, 1.0f, &maps[4]);
    gemm_launch<BN, kEpiF32, 2>(maps[2], maps[3], p.n, f.BN, p.T, at<float>(ws, f.o_g), f.BN, nullptr, 0, s, f.splits,
                                at<float>(ws, f.o_gpart), at<unsigned>(ws, f.o_gtick), 1.0f, &maps[5]);
}

static void frontier_gemm_pair(const CUtensorMap *maps, const Plan &p, const FPlan &f, void *ws, cudaStream_t s,
                               bool two = false) {
    if (two) {
        if (f.BN == 64) frontier_gemms2<64>(maps, p, f, ws, s);
        else if (f.BN == 128) frontier_gemms2<128>(maps, p, f, ws, s);
        else frontier_gemms2<256>(maps, p, f, ws, s);
        return;
    }
    if (f.BN == 64) frontier_gemms<64>(maps[0], maps[1], maps[2], maps[3], p, f, ws, s);
    else if (f.BN == 128) frontier_gemms<128>(maps[0], maps[1], maps[2], maps[3], p, f, ws, s);
    else frontier_gemms<256>(maps[0], maps[1], maps[2], maps[3], p, f, ws, s);
}

// L^T X for the objectives, X already written as the split operand.
static void frontier_ltx(const CUtensorMap *maps, const Plan &p, const FPlan &f, void *ws, cudaStream_t s,
                         bool two = false) {
    __nv_bfloat16 *Zt = at<__nv_bfloat16>(ws, f.o_z);
    if (two) {
        if (f.BN == 64)
            gemm_launch<64, kEpiPairSplitT, 2>(maps[0], maps[1], p.T, f.BN, p.n, nullptr, 0, Zt, f.ldZ, s, 1, nullptr,
                                               nullptr, 1.0f, &maps[4]);
        else if (f.BN == 128)
            gemm_launch<128, kEpiPairSplitT, 2>(maps[0], maps[1], p.T, f.BN, p.n, nullptr, 0, Zt, f.ldZ, s, 1,
                                                nullptr, nullptr, 1.0f, &maps[4]);
        else
            gemm_launch<256, kEpiPairSplitT, 2>(maps[0], maps[1], p.T, f.BN, p.n, nullptr, 0, Zt, f.ldZ, s, 1,
                                                nullptr, nullptr, 1.0f, &maps[4]);
        return;
    }
    if (p.dt == MV_FP8_E4M3) {
        if (f.BN == 64) gemm_q8_launch<64, kEpiPairSplitT>(maps[0], maps[1], p.T, f.BN, p.n, nullptr, 0, Zt, f.ldZ, s);
        else if (f.BN == 128)
            gemm_q8_launch<128, kEpiPairSplitT>(maps[0], maps[1], p.T, f.BN, p.n, nullptr, 0, Zt, f.ldZ, s);
        else gemm_q8_launch<256, kEpiPairSplitT>(maps[0], maps[1], p.T, f.BN, p.n, nullptr, 0, Zt, f.ldZ, s);
        return;
    }
    if (f.BN == 64) gemm_launch<64, kEpiPairSplitT>(maps[0], maps[1], p.T, f.BN, p.n, nullptr, 0, Zt, f.ldZ, s);
    else if (f.BN == 128) gemm_launch<128, kEpiPairSplitT>(maps[0], maps[1], p.T, f.BN, p.n, nullptr, 0, Zt, f.ldZ, s);
    else gemm_launch<256, kEpiPairSplitT>(maps[0], maps[1], p.T, f.BN, p.n, nullptr, 0, Zt, f.ldZ, s);
}

}  // namespace mv

namespace mv {

// The frontier solve; with P_hi (the FP32 factor, MV_LAYOUT_NT) a second
// phase continues every target from the first phase's answer on the BF16
// hi + lo pair of P_hi (FP32-accurate products) to opts->eps, after the
// first phase on P (BF16 or FP8) has stopped at eps_lo.
static int frontier_solve(const mv_problem *P, const mv_problem *P_hi, const double *d_R_targets, int64_t n_targets,
                          const mv_solve_opts *O_in, double eps_lo, double *d_X, mv_solve_info *h_infos, void *d_ws,
                          size_t ws_bytes, cudaStream_t s) {
    MV_TRY(validate_problem(P));
    MV_TRY(require_nt(P, "frontier solve"));
    if (P->dtype == MV_F32)
        return record_message(MV_ERR_UNSUPPORTED, "frontier solve: L must be BF16 or FP8 (the tensor-core operand)");
    if (d_R_targets == nullptr || d_X == nullptr || h_infos == nullptr || n_targets < 1 || n_targets > 128)
        return MV_ERR_INVALID_ARG;
    if (P_hi) {
        MV_TRY(validate_problem(P_hi));
        MV_TRY(require_nt(P_hi, "frontier refinement"));
        if (P_hi->dtype != MV_F32 || P_hi->n != P->n || P_hi->T != P->T || P_hi->mu != P->mu ||
            P_hi->gamma != P->gamma || P_hi->mode != P->mode || !(eps_lo >= 0.0))
            return MV_ERR_INVALID_ARG;
    }
    mv_solve_opts O;
    if (O_in) O = *O_in; else mv_solve_opts_default(&O);
    if (O.max_iter < 0 || O.kkt_every < 0 || O.power_iters < 0 || !(O.eps >= 0.0)) return MV_ERR_INVALID_ARG;
    if (O.momentum != 0 || O.backtrack != 0)
        return record_message(MV_ERR_UNSUPPORTED, "frontier solve: fixed step and FISTA momentum only");
    if (O.lanczos != 0 && O.lanczos != 1) return MV_ERR_INVALID_ARG;
    const bool lanczos = O.lanczos == 1 && !(O.alpha > 0.0);
    if (lanczos && (O.power_iters < 1 || O.power_iters > kMaxLanczos))
        return record_message(MV_ERR_INVALID_ARG, "Lanczos step size: power_iters must be in 1..512");
    const Plan p = make_plan(P->dtype, P->n, P->T, P->ld, 0, true);   // power method: fused pass
    const FPlan f = make_fplan(p, n_targets, P_hi != nullptr);
    MV_TRY(check_ws(d_ws, ws_bytes, f.total));
    MV_TRY(set_kernel_attrs());
    MV_TRY(frontier_attrs());
    (void)cudaGetLastError();
    SolveState *st = at<SolveState>(d_ws, p.o_state);
    float *y32 = at<float>(d_ws, p.o_y32);
    const int B = f.B, nt = (int)n_targets;

    // Targets: the caller's n_targets, padded to B by repeating the last one (padded targets are ignored).
    double *Rt = at<double>(d_ws, f.o_rt);
    MV_CUDA_TRY(cudaMemcpyAsync(Rt, d_R_targets, 8 * (size_t)nt, cudaMemcpyDeviceToDevice, s));
    for (int b = nt; b < B; ++b)
        MV_CUDA_TRY(cudaMemcpyAsync(Rt + b, d_R_targets + nt - 1, 8, cudaMemcpyDeviceToDevice, s));

    // L^T (T x n) once per call: the A operand of Z = L^T Y, and the stored
    // layout in which the power method's fused pass streams fastest.
    const dim3 tgrid((unsigned)((p.T + 31) / 32), (unsigned)((p.n + 31) / 32));
    if (P->dtype == MV_FP8_E4M3)
        transpose_elem_kernel<uint8_t><<<tgrid, dim3(32, 8), 0, s>>>(
            reinterpret_cast<const uint8_t *>(P->L), p.n, p.T, P->ld, at<uint8_t>(d_ws, f.o_lt), f.ldLt);
    else
        transpose_elem_kernel<__nv_bfloat16><<<tgrid, dim3(32, 8), 0, s>>>(
            reinterpret_cast<const __nv_bfloat16 *>(P->L), p.n, p.T, P->ld, at<__nv_bfloat16>(d_ws, f.o_lt), f.ldLt);
    mv_problem Pt = *P;
    Pt.L = at<void>(d_ws, f.o_lt);
    Pt.ld = f.ldLt;
    Pt.layout = MV_LAYOUT_TN;
    const Plan pt = make_plan(P->dtype, P->n, P->T, f.ldLt, 0, true, true);

    // Shared step size from the power method (or Lanczos steps) on L, the
    // fused pass over L^T; the Lanczos vectors use the transposed plan's x
    // and y buffers, which the frontier leaves unused.
    MV_CUDA_TRY(cudaMemsetAsync(at<char>(d_ws, pt.o_tick_t), 0, 4 * (size_t)pt.t_blocks, s));
    MV_CUDA_TRY(cudaMemsetAsync(at<char>(d_ws, pt.o_tick_n), 0, 4 * (size_t)pt.n_groups, s));
    const float *rs = P->dtype == MV_FP8_E4M3 ? P->row_scale : nullptr;
    launch_setup(st, P->mu, P->power_start, rs, y32, p.n, s, lanczos ? at<float>(d_ws, pt.o_x) : nullptr,
                 lanczos ? at<double>(d_ws, pt.o_lan) : nullptr);
    if (pt.use_llt) {
        MV_CUDA_TRY(cudaMemsetAsync(llt_scratch(at<char>(d_ws, pt.o_llt), p.n).tickets, 0, llt_ticket_bytes(), s));
        MV_CUDA_TRY(cudaMemsetAsync(at<char>(d_ws, pt.o_err), 0, 16, s));
    }
    const int est_iters = (O.alpha > 0.0) ? 0 : O.power_iters;
    float *qv[2] = {at<float>(d_ws, pt.o_x), at<float>(d_ws, pt.o_y)};
    for (int it = 0; it < est_iters; ++it) {
        if (pt.use_llt)
            MV_TRY(launch_llt(pt, &Pt, y32, d_ws, nullptr, at<double>(d_ws, pt.o_gy), at<float>(d_ws, pt.o_g32), s));
        else
            gemv_pair(pt, &Pt, y32, d_ws, nullptr, at<double>(d_ws, pt.o_gy), s, at<float>(d_ws, pt.o_g32));
        if (lanczos)
            launch_lanczos_step(at<float>(d_ws, pt.o_g32), qv[it & 1], qv[(it + 1) & 1], at<double>(d_ws, pt.o_lan),
                                rs, y32, p.n, it, s);
        else
            launch_power_norm(at<float>(d_ws, pt.o_g32), rs, y32, p.n, s);
    }
    if (lanczos) {
        launch_lanczos_step_size(st, at<double>(d_ws, pt.o_lan), P->gamma, O.power_safety, O.alpha, s);
    } else {
        if (est_iters > 0) gemv_t_only(pt, &Pt, y32, d_ws, s);
        launch_step_size(st, at<float>(d_ws, pt.o_z), est_iters == 0 ? 0 : p.T, P->gamma, O.power_safety, O.alpha,
                         s);
    }
    MV_CUDA_TRY(cudaMemsetAsync(at<char>(d_ws, f.o_y), 0, 2 * (size_t)f.BN * f.ldY, s));
    MV_CUDA_TRY(cudaMemsetAsync(at<char>(d_ws, f.o_gtick), 0, 4 * (size_t)((p.n + kBM - 1) / kBM) + 64, s));
    MV_CUDA_TRY(cudaGetLastError());
    // Cluster size of the per-target projections: the smallest that holds n,
    // widened towards the single problem's while all B clusters still fit in
    // half a wave (B targets x 16 CTAs would queue in several waves).
    int fcl = 1;
    while ((p.n + fcl - 1) / fcl > kProjMaxLocal) fcl *= 2;
    while (fcl < p.cl && B * fcl * 4 <= sm_count()) fcl *= 2;

    FArgs a;
    a.fs = at<FState>(d_ws, f.o_fs);
    a.st = st;
    a.G = at<float>(d_ws, f.o_g);
    a.ldG = f.BN;
    a.B = B;
    a.X = at<double>(d_ws, f.o_x);
    a.Y = at<double>(d_ws, f.o_yd);
    a.GX = at<double>(d_ws, f.o_gx);
    a.Ysplit = at<__nv_bfloat16>(d_ws, f.o_y);
    a.ldY = f.ldY;
    a.row_scale = rs;
    a.mu = P->mu;
    a.Rt = Rt;
    a.n = p.n;
    a.mode = P->mode;
    a.kkt_every = O.kkt_every;
    a.max_iter = O.max_iter;
    a.gamma = P->gamma;
    a.eps = P_hi ? eps_lo : O.eps;
    MV_CUDA_TRY(launch_frontier(true, fcl, a, s));

    CUtensorMap maps[6];
    if (P->dtype == MV_FP8_E4M3) {
        MV_TRY(make_map_u8(&maps[0], at<void>(d_ws, f.o_lt), p.T, p.n, f.ldLt, kBM));
        MV_TRY(make_map_u8(&maps[2], P->L, p.n, p.T, P->ld, kBM));
    } else {
        MV_TRY(make_map_bf16(&maps[0], at<void>(d_ws, f.o_lt), p.T, p.n, f.ldLt, kBM));
        MV_TRY(make_map_bf16(&maps[2], P->L, p.n, p.T, P->ld, kBM));
    }
    MV_TRY(make_map_bf16(&maps[1], at<void>(d_ws, f.o_y), f.BN, p.n, f.ldY, f.BN));
    MV_TRY(make_map_bf16(&maps[3], at<void>(d_ws, f.o_z), f.BN, p.T, f.ldZ, f.BN));
    int zero = 0;
    MV_CUDA_TRY(cudaMemcpyToSymbolAsync(g_gemm_err, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));

    const int chunk = O.kkt_every > 0 ? O.kkt_every : 8;
    int launches = 3 + 3 * est_iters + (lanczos ? 0 : 1) + 2;
    std::vector<FState> hf(B);
    // One phase: chunks of kkt_every iterations (a cached-per-call graph) until every target is done.
    auto run_phase = [&](const CUtensorMap *mp, bool two) -> int {
        cudaGraphExec_t exec = nullptr;
        if (O.use_graph) {
            cudaStream_t cs;
            MV_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t graph;
            if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                for (int c = 0; c < chunk; ++c) {
                    frontier_gemm_pair(mp, p, f, d_ws, cs, two);
                    launch_frontier(false, fcl, a, cs);
                }
                if (cudaStreamEndCapture(cs, &graph) == cudaSuccess) {
                    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) exec = nullptr;
                    cudaGraphDestroy(graph);
                }
            }
            cudaStreamDestroy(cs);
            (void)cudaGetLastError();
        }
        const int64_t max_chunks = ((int64_t)O.max_iter + 1 + chunk - 1) / chunk + 1;
        int st_ = MV_OK;
        for (int64_t c = 0; c < max_chunks; ++c) {
            if (exec) {
                if (cudaGraphLaunch(exec, s) != cudaSuccess) {
                    st_ = record_cuda_error(cudaGetLastError(), "cudaGraphLaunch", __FILE__, __LINE__);
                    break;
                }
            } else {
                for (int i = 0; i < chunk; ++i) {
                    frontier_gemm_pair(mp, p, f, d_ws, s, two);
                    launch_frontier(false, fcl, a, s);
                }
            }
            launches += 3 * chunk;
            if (cudaMemcpyAsync(hf.data(), a.fs, sizeof(FState) * B, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                st_ = record_cuda_error(cudaGetLastError(), "frontier loop", __FILE__, __LINE__);
                break;
            }
            bool all = true;
            for (int b = 0; b < nt; ++b) all = all && hf[b].done;
            if (all) break;
        }
        if (exec) cudaGraphExecDestroy(exec);
        return st_;
    };
    MV_TRY(run_phase(maps, false));
    std::vector<int> iters1(B);
    for (int b = 0; b < B; ++b) iters1[b] = hf[b].k;
    bool two = false;
    if (P_hi) {
        // Phase 2 on the FP32 factor: BF16 hi + lo pair and its transposes, a step 1 % smaller.
        __nv_bfloat16 *H = at<__nv_bfloat16>(d_ws, f.o_h), *D = at<__nv_bfloat16>(d_ws, f.o_d);
        __nv_bfloat16 *Ht = at<__nv_bfloat16>(d_ws, f.o_ht), *Dt = at<__nv_bfloat16>(d_ws, f.o_dt);
        hilo_kernel<<<152 * 8, 256, 0, s>>>(reinterpret_cast<const float *>(P_hi->L), p.n, p.T, P_hi->ld, H, D, f.ldH);
        transpose_elem_kernel<__nv_bfloat16><<<tgrid, dim3(32, 8), 0, s>>>(H, p.n, p.T, f.ldH, Ht, f.ldLt);
        transpose_elem_kernel<__nv_bfloat16><<<tgrid, dim3(32, 8), 0, s>>>(D, p.n, p.T, f.ldH, Dt, f.ldLt);
        CUtensorMap m2[6];
        MV_TRY(make_map_bf16(&m2[0], Ht, p.T, p.n, f.ldLt, kBM));
        MV_TRY(make_map_bf16(&m2[4], Dt, p.T, p.n, f.ldLt, kBM));
        MV_TRY(make_map_bf16(&m2[2], H, p.n, p.T, f.ldH, kBM));
        MV_TRY(make_map_bf16(&m2[5], D, p.n, p.T, f.ldH, kBM));
        m2[1] = maps[1];
        m2[3] = maps[3];
        SolveState hs1{};
        MV_CUDA_TRY(cudaMemcpyAsync(&hs1, st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        MV_CUDA_TRY(cudaStreamSynchronize(s));
        const double alpha2 = hs1.alpha / 1.01;
        MV_CUDA_TRY(cudaMemcpyAsync(&st->alpha, &alpha2, sizeof(double), cudaMemcpyHostToDevice, s));
        frontier_warm_kernel<<<B, 256, 0, s>>>(a.fs, a.X, a.Y, p.n, B, a.Ysplit, a.ldY);
        MV_CUDA_TRY(cudaGetLastError());
        a.row_scale = nullptr;
        a.eps = O.eps;
        for (int i = 0; i < 6; ++i) maps[i] = m2[i];
        two = true;
        launches += 4;
        MV_TRY(run_phase(maps, true));
    }
    // Objectives: one more L^T X product with X written as the split operand.
    split_rows_kernel<<<(unsigned)((B * (int64_t)p.n + 255) / 256), 256, 0, s>>>(a.X, B, p.n, a.Ysplit, f.ldY,
                                                                               a.row_scale);
    frontier_ltx(maps, p, f, d_ws, s, two);
    frontier_objective_kernel<<<B, kStepThreads, 0, s>>>(at<__nv_bfloat16>(d_ws, f.o_z), f.ldZ, B, p.T, a.X, p.n,
                                                         P->gamma, a.fs);
    launches += 3;
    MV_CUDA_TRY(cudaGetLastError());
    MV_CUDA_TRY(cudaMemcpyAsync(hf.data(), a.fs, sizeof(FState) * B, cudaMemcpyDeviceToHost, s));
    int err = 0;
    MV_CUDA_TRY(cudaMemcpyFromSymbolAsync(&err, g_gemm_err, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    MV_CUDA_TRY(cudaMemcpy2DAsync(d_X, 8 * (size_t)p.n, a.X, 8 * (size_t)p.n, 8 * (size_t)p.n, (size_t)nt,
                                  cudaMemcpyDeviceToDevice, s));
    SolveState hs{};
    MV_CUDA_TRY(cudaMemcpyAsync(&hs, st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    MV_CUDA_TRY(cudaStreamSynchronize(s));
    if (err != 0) return record_message(MV_ERR_TIMEOUT, "frontier GEMM pipeline wait timed out");
    int worst = MV_OK;
    for (int b = 0; b < nt; ++b) {
        mv_solve_info &I = h_infos[b];
        I = mv_solve_info{};
        I.iterations = P_hi ? iters1[b] + hf[b].k : hf[b].k;
        I.refine_iterations = P_hi ? hf[b].k : 0;
        I.status = hf[b].done ? hf[b].status : MV_ERR_NOT_CONVERGED;
        I.converged = hf[b].converged;
        I.proj_failures = hf[b].proj_fail;
        I.proj_steps = hf[b].proj_steps;
        I.kkt = hf[b].kkt;
        I.objective = hf[b].objective;
        I.alpha = hs.alpha;
        I.lambda_hat = hs.lambda_hat;
        I.nu = hf[b].nu;
        I.launches = launches;
        if (I.status != MV_OK && worst == MV_OK) worst = I.status;
    }
    return worst;
}

}  // namespace mv

extern "C" {

size_t mv_frontier_workspace_size(const mv_problem *P, int64_t n_targets) {
    if (validate_problem(P) != MV_OK || P->layout != MV_LAYOUT_NT || P->dtype == MV_F32 || n_targets < 1 ||
        n_targets > 128)
        return 0;
    const Plan p = make_plan(P->dtype, P->n, P->T, P->ld, 0, true);
    return make_fplan(p, n_targets).total;
}

int mv_npga_solve_frontier(const mv_problem *P, const double *d_R_targets, int64_t n_targets,
                           const mv_solve_opts *O_in, double *d_X, mv_solve_info *h_infos, void *d_ws, size_t ws_bytes,
                           mv_stream_t stream) {
    return frontier_solve(P, nullptr, d_R_targets, n_targets, O_in, 0.0, d_X, h_infos, d_ws, ws_bytes,
                          (cudaStream_t)stream);
}

size_t mv_frontier_refined_workspace_size(const mv_problem *P_lo, const mv_problem *P_hi, int64_t n_targets) {
    if (mv_frontier_workspace_size(P_lo, n_targets) == 0 || validate_problem(P_hi) != MV_OK ||
        P_hi->dtype != MV_F32 || P_hi->layout != MV_LAYOUT_NT)
        return 0;
    const Plan p = make_plan(P_lo->dtype, P_lo->n, P_lo->T, P_lo->ld, 0, true);
    return make_fplan(p, n_targets, true).total;
}

int mv_npga_solve_frontier_refined(const mv_problem *P_lo, const mv_problem *P_hi, const double *d_R_targets,
                                   int64_t n_targets, const mv_solve_opts *O_in, double eps_lo, double *d_X,
                                   mv_solve_info *h_infos, void *d_ws, size_t ws_bytes, mv_stream_t stream) {
    if (P_hi == nullptr) return MV_ERR_INVALID_ARG;
    return frontier_solve(P_lo, P_hi, d_R_targets, n_targets, O_in, eps_lo, d_X, h_infos, d_ws, ws_bytes,
                          (cudaStream_t)stream);
}

}  // extern "C"
