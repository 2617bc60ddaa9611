// NPGA solve (Algorithm 1, fixed step of Sec. 3.1) on one GPU.
//
// Per iteration three kernels run back to back on one stream:
//   gemv_t  z = L^T y^k                 (all SMs, HBM-bound)
//   gemv_n  g = L z                     (all SMs, HBM-bound)
//   step    one block: grad f(x^k) by linearity, KKT check every kkt_every
//           iterations, v = y^k - alpha (2g + 2 gamma y^k), x^{k+1} = Pi_F(v)
//           (FP64, warm-started), FISTA momentum and extrapolation.
// A chunk of kkt_every iterations is captured once into a CUDA graph and
// replayed; every kernel returns at once when the device-side `done` flag is
// set, so a chunk that overruns convergence costs only empty launches.  The
// host reads the flag once per chunk.
#include <stdlib.h>

#include <mutex>
#include <unordered_map>
#include <vector>

#include "gemm.cuh"
#include "gemm_q8.cuh"
#include "gemv.cuh"
#include "llt_api.h"
#include "project.cuh"
#include "symv.cuh"

namespace mv {

constexpr int kStepThreads = 512;
constexpr int kProjBudget = 100;

struct SolveState {
    int k, done, converged, status;
    int proj_fail, proj_steps, pad1, pad2;
    double t, beta_prev;
    double alpha, lambda_hat;
    double kkt, nu, tau, nu_kkt, tau_kkt;
    double mu_min, mu_max;
    double objective;
    double beta_c;                         // constant momentum (momentum = 1)
    int bt_started, backtracks, dykstra, pad3;
};

struct Plan {
    int dt, vec, esize;
    int n, T;
    int64_t ld;
    bool tn;                               // L stored transposed (T x n)
    int gr, gc;                            // rows and columns of the stored matrix
    int cl;                                // cluster size of the step kernel
    int t_blocks, t_splits, t_rows;        // gemv_t grid
    int n_groups, n_splits, n_cols;        // gemv_n grid
    bool use_llt;                          // fused single-pass L L^T y (llt.cuh)
    bool want_z;                           // the loop's fused pass also writes z = L^T y to o_z
    LltPlan lp;
    bool sig;                              // explicit Sigma (symv.cuh) instead of a factor
    int snb;                               // Sigma tile rows
    size_t o_spart, o_stick, o_gobj;
    size_t o_dyk, o_gd, o_xp;              // Dykstra scratch; backtracking L L^T d and candidate
    // workspace offsets (bytes)
    size_t o_state, o_x, o_y, o_gx, o_gy, o_g32, o_y32, o_z, o_zpart, o_gpart, o_tick_t, o_tick_n;
    size_t o_llt, o_err, o_zd;
    int64_t zstride;                       // row pitch (floats) of the gemv_t partials
    size_t total;
};

static int sm_count() {
    static int cached = 0;
    if (cached == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        int c = 0;
        cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
        cached = c > 0 ? c : 148;
    }
    return cached;
}

static constexpr int kRW = 4;   // rows per warp in gemv_n

// The fused pass pays a cluster exchange per 128-byte column block, so it is
// used where a block holds many rows and there are many blocks.
// gemv_t (column sums) and gemv_n (row dots) run over the stored matrix:
// L (n x T) for MV_LAYOUT_NT, where z = L^T y is gemv_t and g = L z is
// gemv_n; L^T (T x n) for MV_LAYOUT_TN, where the two swap roles.
static Plan make_plan(int dt, int64_t n, int64_t T, int64_t ld, int grouped_rows = 0, bool fused = false,
                      bool tn = false, int n_bytes = 16384) {
    Plan p{};
    p.dt = dt;
    p.esize = dtype_size(dt);
    p.vec = 16 / p.esize;
    p.n = (int)n;
    p.T = (int)T;
    p.ld = ld;
    p.tn = tn;
    const int64_t gr = tn ? T : n, gc = tn ? n : T;
    p.gr = (int)gr;
    p.gc = (int)gc;
    p.cl = proj_cluster_size(n);
    // Tuning override of the step kernel's cluster size (1, 2, 4, 8 or 16).
    if (const char *env = getenv("MV_STEP_CLUSTER")) {
        const int c = atoi(env);
        if ((c == 1 || c == 2 || c == 4 || c == 8 || c == 16) && (n + c - 1) / c <= kProjMaxLocal) p.cl = c;
    }
    const int sms = sm_count();
    // gemv_t: strips of 256*VEC columns; rows split so the grid covers
    // several waves of the machine (4 resident blocks per SM assumed).
    const int strip = kGemvThreads * p.vec;
    p.t_blocks = (int)((gc + strip - 1) / strip);
    const int slots = sms * 4;
    int splits = (slots * 3 + p.t_blocks - 1) / p.t_blocks;
    splits = (int)std::max<int64_t>(1, std::min<int64_t>(splits, (gr + 63) / 64));
    if (grouped_rows > 0) splits = (int)((gr + grouped_rows - 1) / grouped_rows);   // many problems share the GPU
    int rows = (int)((gr + splits - 1) / splits);
    if (rows > kMaxRowsPerSplit) rows = kMaxRowsPerSplit;
    p.t_rows = rows;
    p.t_splits = (int)((gr + rows - 1) / rows);
    // gemv_n: 32 rows per block, column splits of 16 KB of the matrix per row.
    const int rows_per_block = (kGemvThreads / kWarp) * kRW;
    p.n_groups = (int)((gr + rows_per_block - 1) / rows_per_block);
    p.n_cols = n_bytes / p.esize;                        // 16 KB per row per split by default
    if (p.n_cols > gc) p.n_cols = (int)((gc + 32 * p.vec - 1) / (32 * p.vec) * (32 * p.vec));
    p.n_splits = (int)((gc + p.n_cols - 1) / p.n_cols);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    p.o_state = take(sizeof(SolveState));
    p.o_x = take(8 * (size_t)n);
    p.o_y = take(8 * (size_t)n);
    p.o_gx = take(8 * (size_t)n);
    p.o_gy = take(8 * (size_t)n);
    p.o_g32 = take(4 * (size_t)n);
    p.o_y32 = take(4 * (size_t)n);
    p.o_z = take(4 * (size_t)T + 64);
    p.zstride = (gc + 15) / 16 * 16;
    p.o_zpart = take(4 * (size_t)p.zstride * p.t_splits);
    p.o_gpart = take(4 * (size_t)gr * p.n_splits);
    p.o_zd = tn ? take(8 * (size_t)T) : 0;
    p.o_tick_t = take(4 * (size_t)p.t_blocks);
    p.o_tick_n = take(4 * (size_t)p.n_groups);
    p.use_llt = false;
    p.lp = LltPlan{};
    if (fused && llt_plan(dt, n, T, false, tn).ok) {
        // The scratch is sized without the device query, so the workspace
        // size does not depend on the device.
        p.o_llt = take(llt_scratch_bytes(n));
        p.lp = llt_plan(dt, n, T, true, tn);
        p.use_llt = p.lp.ok;
    }
    const int nl = (int)((n + p.cl - 1) / p.cl);
    p.o_dyk = take(8 * 4 * (size_t)nl * p.cl);
    p.o_gd = take(8 * (size_t)n);
    p.o_xp = take(8 * (size_t)n);
    p.o_err = take(16);
    p.total = off;
    return p;
}

// Explicit Sigma (n x n FP32): the product is one symmetric pass (symv.cuh).
static Plan make_plan_sigma(int64_t n, int64_t ld) {
    Plan p{};
    p.dt = MV_F32;
    p.esize = 4;
    p.vec = 4;
    p.n = (int)n;
    p.T = 0;
    p.ld = ld;
    p.gr = p.gc = (int)n;
    p.sig = true;
    p.cl = proj_cluster_size(n);
    if (const char *env = getenv("MV_STEP_CLUSTER")) {
        const int c = atoi(env);
        if ((c == 1 || c == 2 || c == 4 || c == 8 || c == 16) && (n + c - 1) / c <= kProjMaxLocal) p.cl = c;
    }
    p.snb = (int)((n + kSymTile - 1) / kSymTile);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    p.o_state = take(sizeof(SolveState));
    p.o_x = take(8 * (size_t)n);
    p.o_y = take(8 * (size_t)n);
    p.o_gx = take(8 * (size_t)n);
    p.o_gy = take(8 * (size_t)n);
    p.o_g32 = take(4 * (size_t)n);
    p.o_y32 = take(4 * (size_t)n);
    p.o_gobj = take(8 * (size_t)n);
    p.o_spart = take(symv_part_bytes((int)n));
    p.o_stick = take(4 * (size_t)p.snb);
    p.o_z = p.o_zpart = p.o_gpart = p.o_tick_t = p.o_tick_n = p.o_g32;   // unused by this form
    const int nl = (int)((n + p.cl - 1) / p.cl);
    p.o_dyk = take(8 * 4 * (size_t)nl * p.cl);
    p.o_gd = take(8 * (size_t)n);
    p.o_xp = take(8 * (size_t)n);
    p.o_err = take(16);
    p.total = off;
    return p;
}

template <typename T_>
static T_ *at(void *ws, size_t off) {
    return reinterpret_cast<T_ *>(reinterpret_cast<char *>(ws) + off);
}

// ------------------------------------------------------------------ kernels
// This block's slice of the Dykstra scratch (4 arrays of nl doubles).
__device__ __forceinline__ double *dyk_slice(double *base, int rank, int nl) {
    return base ? base + (size_t)rank * 4 * nl : nullptr;
}

__device__ __forceinline__ void setup_body(SolveState *st, const double *__restrict__ mu, const double *__restrict__ r0,
             const float *__restrict__ row_scale, float *__restrict__ y32, int n) {
    __shared__ double red[(kStepThreads / kWarp + 1) * 5];
    double mn = INFINITY, mx = -INFINITY, ss = 0.0;
    for (int i = threadIdx.x; i < n; i += kStepThreads) {
        const double m = mu[i];
        mn = fmin(mn, m);
        mx = fmax(mx, m);
        const double r = r0 ? r0[i] : 1.0;
        ss += r * r;
        if (!(m == m)) mx = NAN;
    }
    block_minmax<kStepThreads>(mn, mx, red);
    __syncthreads();
    double v1[1] = {ss};
    block_sum<1, kStepThreads>(v1, red);
    const double inv = v1[0] > 0.0 ? 1.0 / sqrt(v1[0]) : 0.0;
    for (int i = threadIdx.x; i < n; i += kStepThreads) {
        const double r = r0 ? r0[i] : 1.0;
        const double s = row_scale ? (double)row_scale[i] : 1.0;
        y32[i] = (float)(r * inv * s);
    }
    if (threadIdx.x == 0) {
        SolveState z{};
        z.mu_min = mn;
        z.mu_max = mx;
        z.t = 1.0;
        z.status = (mx == mx && mn == mn) ? MV_OK : MV_ERR_NUMERIC;
        *st = z;
    }
}

__global__ void __launch_bounds__(kStepThreads)
setup_kernel(SolveState *st, const double *__restrict__ mu, const double *__restrict__ r0,
             const float *__restrict__ row_scale, float *__restrict__ y32, int n) {
    setup_body(st, mu, r0, row_scale, y32, n);
}

// u <- g / ||g|| (power method) from the FP32 copy of g, written as the FP32
// gemv input (row-scaled).  FP32 arithmetic: u only sets the direction.
__device__ __forceinline__ void power_norm_body(const float *__restrict__ g32, const float *__restrict__ row_scale, float *__restrict__ y32,
                  int n) {
    __shared__ float red[kStepThreads / kWarp + 1];
    float ss = 0.f;
    for (int i = threadIdx.x; i < n; i += kStepThreads) ss = fmaf(g32[i], g32[i], ss);
    ss = warp_sumf(ss);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x < 32) {
        float t = threadIdx.x < kStepThreads / kWarp ? red[threadIdx.x] : 0.f;
        t = warp_sumf(t);
        if (threadIdx.x == 0) red[kStepThreads / kWarp] = t;
    }
    __syncthreads();
    const float tot = red[kStepThreads / kWarp];
    const float inv = tot > 0.f ? rsqrtf(tot) : 0.f;
    for (int i = threadIdx.x; i < n; i += kStepThreads)
        y32[i] = g32[i] * inv * (row_scale ? row_scale[i] : 1.f);
}

__global__ void __launch_bounds__(kStepThreads)
power_norm_kernel(const float *__restrict__ g32, const float *__restrict__ row_scale, float *__restrict__ y32,
                  int n) {
    power_norm_body(g32, row_scale, y32, n);
}

// Compensated FP32 sum of squares of an FP32 vector; FP64 only across threads.
__device__ __forceinline__ double sumsq_f32(const float *__restrict__ z, int T, double *red) {
    float s = 0.f, c = 0.f;
    for (int t = threadIdx.x; t < T; t += kStepThreads) {
        const float y = fmaf(z[t], z[t], -c);
        const float u = s + y;
        c = (u - s) - y;
        s = u;
    }
    double v[1] = {(double)s - (double)c};
    block_sum<1, kStepThreads>(v, red);
    return v[0];
}

// alpha = 1 / (2 (lambda_hat (1 + safety) + gamma)), or the override.
__device__ __forceinline__ void set_step(SolveState *st, double lam, double gamma, double safety, double alpha_override) {
    st->lambda_hat = lam;
    double a = alpha_override;
    if (!(a > 0.0)) {
        const double lf = 2.0 * (lam * (1.0 + safety) + gamma);
        a = lf > 0.0 ? 1.0 / lf : 1.0;
    }
    st->alpha = a;
    if (!(a == a) || !isfinite(a)) st->status = MV_ERR_NUMERIC;
}

// lambda_hat = ||L^T u||^2.
__device__ __forceinline__ void step_size_body(SolveState *st, const float *__restrict__ z, int T, double gamma, double safety,
                 double alpha_override) {
    __shared__ double red[(kStepThreads / kWarp + 1) * 5];
    const double lam = sumsq_f32(z, T, red);
    if (threadIdx.x == 0) set_step(st, lam, gamma, safety, alpha_override);
}

__global__ void __launch_bounds__(kStepThreads)
step_size_kernel(SolveState *st, const float *__restrict__ z, int T, double gamma, double safety,
                 double alpha_override) {
    step_size_body(st, z, T, gamma, safety, alpha_override);
}

// Explicit Sigma: lambda_hat = u^T (Sigma u), the Rayleigh quotient of the
// unit power vector u (equal to ||L^T u||^2 when Sigma = L L^T).
__global__ void __launch_bounds__(kStepThreads)
step_size_sigma_kernel(SolveState *st, const float *__restrict__ u, const double *__restrict__ su, int n, double gamma,
                       double safety, double alpha_override) {
    __shared__ double red[(kStepThreads / kWarp + 1) * 5];
    double v[1] = {0.0};
    for (int i = threadIdx.x; i < n; i += kStepThreads) v[0] = fma((double)u[i], su[i], v[0]);
    block_sum<1, kStepThreads>(v, red);
    if (threadIdx.x == 0) set_step(st, v[0], gamma, safety, alpha_override);
}

// x^0: Pi_F(1/n 1), or the caller's x^0 when warm-starting; y^0 = x^0.
// Runs as one cluster of CL blocks (the projection of project.cuh).
template <int CL>
__device__ __forceinline__ void init_x_body(SolveState *st, const double *__restrict__ mu,
                                            const double *__restrict__ x_in, double *__restrict__ x,
                                            double *__restrict__ y, float *__restrict__ y32,
                                            const float *__restrict__ row_scale, int n, double R, int mode,
                                            unsigned char *dsm, ProjSmem &psm, double *dyk = nullptr,
                                            int dyk_iters = 0, int budget = kProjBudget) {
    const int rank = cluster_rank<CL>();
    const int nl = (n + CL - 1) / CL;
    const int r0 = min(n, rank * nl);
    const int r1 = min(n, r0 + nl);
    const double mn = st->mu_min, mx = st->mu_max;
    if (x_in == nullptr) {
        ProjElems el = carve_elems(dsm, nl);
        el.n = r1 - r0;
        proj_smem_init(&psm);
        for (int i = threadIdx.x; i < el.n; i += kProjNT) {
            el.v[i] = 1.0 / n;
            el.mu[i] = mu[r0 + i];
        }
        __syncthreads();
        ClusterProj<CL> P{&psm, el};
        P.dyk = dyk_slice(dyk, rank, nl);
        P.dyk_iters = dyk_iters;
        P.prepare();
        const ProjOut o = P.solve(R, mode, mn, mx, 0.0, -INFINITY, budget);
        for (int i = threadIdx.x; i < el.n; i += kProjNT) {
            const double xi = o.status == MV_ERR_INFEASIBLE ? NAN : fmax(fma(o.nu, el.mu[i], el.v[i]) - o.tau, 0.0);
            x[r0 + i] = xi;
            y[r0 + i] = xi;
            y32[r0 + i] = (float)(xi * (row_scale ? (double)row_scale[r0 + i] : 1.0));
        }
        if (rank == 0 && threadIdx.x == 0) {
            if (o.status == MV_ERR_INFEASIBLE || o.status == MV_ERR_NUMERIC) st->status = o.status;
            st->nu = o.nu;
            st->tau = o.tau;
            st->nu_kkt = o.nu;
            st->tau_kkt = o.tau;
            st->dykstra += o.dykstra;
        }
        cluster_barrier<CL>();
    } else {
        for (int i = r0 + threadIdx.x; i < r1; i += kProjNT) {
            const double xi = x_in[i];
            x[i] = xi;
            y[i] = xi;
            y32[i] = (float)(xi * (row_scale ? (double)row_scale[i] : 1.0));
        }
        if (rank == 0 && threadIdx.x == 0) {
            st->nu = 0.0;
            st->tau = -INFINITY;
            st->nu_kkt = 0.0;
            st->tau_kkt = -INFINITY;
        }
    }
    if (rank == 0 && threadIdx.x == 0) {
        st->t = 1.0;
        st->beta_prev = 0.0;
        st->k = 0;
        st->done = (st->status != MV_OK) ? 1 : 0;
        st->converged = 0;
        st->proj_fail = 0;
        st->proj_steps = 0;
        st->kkt = INFINITY;
    }
}

template <int CL>
__global__ void __launch_bounds__(kProjNT)
init_x_kernel(SolveState *st, const double *__restrict__ mu, const double *__restrict__ x_in,
              double *__restrict__ x, double *__restrict__ y, float *__restrict__ y32,
              const float *__restrict__ row_scale, int n, double R, int mode, double *dyk, int dyk_iters,
              int budget) {
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ ProjSmem psm;
    init_x_body<CL>(st, mu, x_in, x, y, y32, row_scale, n, R, mode, dsm, psm, dyk, dyk_iters, budget);
}

struct StepArgs {
    SolveState *st;
    const double *gy;
    double *x, *y, *gx;
    float *y32;
    const double *mu;
    const float *row_scale;
    int n, mode, kkt_every, max_iter;
    double R, gamma, eps;
    // Sec. 3.1 variants and the projection safeguard
    double *dyk = nullptr;                 // 4 (n + CL) doubles of Dykstra scratch, or none
    int dyk_iters = 0;
    int budget = kProjBudget;
    int momentum = 0;                      // 1: beta fixed at st->beta_c
    int pad = 0;
    double bt_rho = 0.5;
    double m_f = 0.0;                      // curvature bound of the constant momentum
    double *gyw = nullptr;                 // backtracking: L L^T y (written), L L^T d, candidate x+
    const double *gd = nullptr;
    double *xp = nullptr;
};


// One NPGA step on a cluster of CL blocks; block r owns assets [r0, r1).
template <int CL>
__device__ __forceinline__ void npga_step_body(const StepArgs &a, unsigned char *dsm, ProjSmem &psm) {
    SolveState *st = a.st;
    // Every block reads the flag before the first cluster barrier; the flag is
    // only written after later barriers, so the whole cluster agrees.
    if (*(volatile int *)&st->done) return;
    const int n = a.n;
    const int rank = cluster_rank<CL>();
    const int nl = (n + CL - 1) / CL;
    const int r0 = min(n, rank * nl);
    const int r1 = min(n, r0 + nl);
    const int k = st->k;
    const double beta_prev = st->beta_prev, alpha = st->alpha, t = st->t;
    const double mn = st->mu_min, mx = st->mu_max;
    const double nu0 = st->nu, tau0 = st->tau, nuk0 = st->nu_kkt, tauk0 = st->tau_kkt;
    const double gamma = a.gamma;
    ProjElems el = carve_elems(dsm, nl);
    el.n = r1 - r0;
    // Scalars are computed once (FP64 is scarce on this part) and broadcast.
    __shared__ double sc[4];
    if (threadIdx.x == 0) {
        sc[0] = 1.0 / (1.0 + beta_prev);
        if (a.momentum == 1) {             // strongly convex specialisation: t unused, beta fixed
            sc[1] = t;
            sc[2] = st->beta_c;
        } else {
            const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
            sc[1] = tn;
            sc[2] = (t - 1.0) / tn;
        }
    }
    proj_smem_init(&psm);
    const double inv1pb = sc[0], tn = sc[1], beta = sc[2];
    const bool check = (a.kkt_every > 0 && k % a.kkt_every == 0) || (k >= a.max_iter);

    // L L^T x^k by linearity from the product at y^k; the point to project:
    // x - alpha grad f(x) on a KKT test, else the gradient step from y^k
    // (one pass over the vectors either way).
    for (int i = threadIdx.x; i < el.n; i += kProjNT) {
        const int gi = r0 + i;
        el.mu[i] = a.mu[gi];
        const double gyi = a.gy[gi];
        const double gxi = (k == 0) ? gyi : (gyi + beta_prev * a.gx[gi]) * inv1pb;
        a.gx[gi] = gxi;
        if (check) {
            const double xi = a.x[gi];
            el.v[i] = xi - alpha * (2.0 * gxi + 2.0 * gamma * xi);
        } else {
            const double yi = a.y[gi];
            el.v[i] = yi - alpha * (2.0 * gyi + 2.0 * gamma * yi);
        }
    }
    __syncthreads();
    ClusterProj<CL> P{&psm, el};
    P.dyk = dyk_slice(a.dyk, rank, nl);
    P.dyk_iters = a.dyk_iters;
    if (check) {
        P.prepare();
        const ProjOut o = P.solve(a.R, a.mode, mn, mx, nuk0, tauk0, a.budget);
        double r2 = 0.0;
        for (int i = threadIdx.x; i < el.n; i += kProjNT) {
            const double p = fmax(fma(o.nu, el.mu[i], el.v[i]) - o.tau, 0.0);
            const double d = p - a.x[r0 + i];
            r2 = fma(d, d, r2);
        }
        r2 = P.reduce_double(r2);          // identical in every block
        const bool conv = r2 <= a.eps * a.eps;
        const bool stop = conv || k >= a.max_iter || !(r2 == r2);
        if (rank == 0 && threadIdx.x == 0) {
            const double kkt = sqrt(r2);
            st->kkt = kkt;
            st->nu_kkt = o.nu;
            st->tau_kkt = o.tau;
            st->proj_steps += o.steps;
            st->dykstra += o.dykstra;
            if (o.status != MV_OK) st->proj_fail += 1;
            if (stop) {
                st->done = 1;
                st->converged = conv ? 1 : 0;
                st->status = conv ? MV_OK : (!(r2 == r2) ? MV_ERR_NUMERIC : MV_ERR_NOT_CONVERGED);
            }
        }
        if (stop) {
            cluster_barrier<CL>();
            return;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < el.n; i += kProjNT) {
            const int gi = r0 + i;
            const double yi = a.y[gi];
            el.v[i] = yi - alpha * (2.0 * a.gy[gi] + 2.0 * gamma * yi);
        }
        __syncthreads();
    }
    P.prepare();
    const ProjOut o = P.solve(a.R, a.mode, mn, mx, nu0, tau0, a.budget);
    for (int i = threadIdx.x; i < el.n; i += kProjNT) {
        const int gi = r0 + i;
        const double xn = fmax(fma(o.nu, el.mu[i], el.v[i]) - o.tau, 0.0);
        const double xo = a.x[gi];
        const double yn = xn + beta * (xn - xo);
        a.x[gi] = xn;
        a.y[gi] = yn;
        a.y32[gi] = (float)(yn * (a.row_scale ? (double)a.row_scale[gi] : 1.0));
    }
    if (rank == 0 && threadIdx.x == 0) {
        st->t = tn;
        st->beta_prev = beta;
        st->k = k + 1;
        st->nu = o.nu;
        st->tau = o.tau;
        if (o.status != MV_OK) st->proj_fail += 1;
        st->proj_steps += o.steps;
        st->dykstra += o.dykstra;
        if (o.status == MV_ERR_INFEASIBLE || o.status == MV_ERR_NUMERIC) {
            st->done = 1;
            st->status = o.status;
        }
    }
    cluster_barrier<CL>();   // no block leaves while a peer may still address its shared memory
}

template <int CL>
__global__ void __launch_bounds__(kProjNT) npga_step_kernel(StepArgs a) {
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ ProjSmem psm;
    npga_step_body<CL>(a, dsm, psm);
}

// Grouped form: cluster b runs the step of problem b.
template <int CL>
__global__ void __launch_bounds__(kProjNT) npga_step_grouped(const StepArgs *__restrict__ args) {
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ ProjSmem psm;
    const StepArgs a = args[blockIdx.x / CL];
    npga_step_body<CL>(a, dsm, psm);
}

// Sets up the Sec. 3.1 variants once alpha is known: the first backtracking
// trial step (alpha0, or the power-method step / rho^4 when alpha0 <= 0)
// and the constant momentum beta = (1 - q) / (1 + q), q = sqrt(alpha m_f)
// (clamped to q <= 1).
__device__ __forceinline__ double const_beta(double alpha, double m_f) {
    const double q = fmin(sqrt(alpha * m_f), 1.0);
    return (1.0 - q) / (1.0 + q);
}

__global__ void variant_setup_kernel(SolveState *st, int momentum, double m_f, int backtrack, double alpha0,
                                     double rho) {
    if (threadIdx.x != 0) return;
    if (backtrack) st->alpha = alpha0 > 0.0 ? alpha0 : st->alpha / (rho * rho * rho * rho);
    if (momentum) st->beta_c = const_beta(st->alpha, m_f);
    st->bt_started = 0;
}

// One backtracking step (Sec. 3.1, adaptive backtracking) on a cluster of
// CL blocks.  The pending candidate x+ = Pi_F(y - alpha grad f(y)) was
// projected by the previous launch, and the product between the two
// launches formed L L^T d for d = x+ - y.  The sufficient-decrease test
//     f(x+) <= f(y) + <grad f(y), d> + ||d||^2 / (2 alpha)
// is exactly d^T L L^T d + gamma ||d||^2 <= ||d||^2 / (2 alpha) for this
// quadratic f, evaluated in that form (the difference of objective values
// cancels to rounding noise near the solution).  Accepted: x <- x+,
// L L^T x <- L L^T y + L L^T d, the momentum step, and L L^T y for the new
// y by linearity, with the KKT test every kkt_every accepted iterations.
// Rejected: alpha <- rho alpha.  Either way the next candidate is projected
// from y and d is written as the next product's FP32 input.
template <int CL>
__device__ __forceinline__ void npga_bt_step_body(const StepArgs &a, unsigned char *dsm, ProjSmem &psm) {
    SolveState *st = a.st;
    if (*(volatile int *)&st->done) return;
    const int n = a.n;
    const int rank = cluster_rank<CL>();
    const int nl = (n + CL - 1) / CL;
    const int r0 = min(n, rank * nl);
    const int r1 = min(n, r0 + nl);
    const int k = st->k;
    const double t = st->t, mn = st->mu_min, mx = st->mu_max;
    const bool started = st->bt_started != 0;
    double alpha = st->alpha;
    const double gamma = a.gamma;
    ProjElems el = carve_elems(dsm, nl);
    el.n = r1 - r0;
    proj_smem_init(&psm);
    ClusterProj<CL> P{&psm, el};
    P.dyk = dyk_slice(a.dyk, rank, nl);
    P.dyk_iters = a.dyk_iters;
    __shared__ double sc[2];
    int kn = k;
    double tn = t, beta = st->beta_prev;
    bool accepted = false, rejected = false, numeric = false;
    for (int i = threadIdx.x; i < el.n; i += kProjNT) el.mu[i] = a.mu[r0 + i];
    if (started) {
        double s1 = 0.0, s2 = 0.0;
        for (int i = threadIdx.x; i < el.n; i += kProjNT) {
            const int gi = r0 + i;
            const double d = a.xp[gi] - a.y[gi];
            s1 = fma(d, a.gd[gi], s1);
            s2 = fma(d, d, s2);
        }
        s1 = P.reduce_double(s1);
        s2 = P.reduce_double(s2);
        const double q = s1 + gamma * s2;
        if (!(q == q) || !(s2 == s2)) {
            numeric = true;
        } else if (s2 == 0.0 || q <= s2 / (2.0 * alpha)) {
            accepted = true;
        } else {
            rejected = true;
        }
    }
    if (accepted) {
        if (threadIdx.x == 0) {
            if (a.momentum == 1) {
                sc[0] = t;
                sc[1] = st->beta_c;
            } else {
                const double tt = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
                sc[0] = tt;
                sc[1] = (t - 1.0) / tt;
            }
        }
        __syncthreads();
        tn = sc[0];
        beta = sc[1];
        for (int i = threadIdx.x; i < el.n; i += kProjNT) {
            const int gi = r0 + i;
            const double gxp = a.gyw[gi] + a.gd[gi];            // L L^T x+
            const double xo = a.x[gi], xn = a.xp[gi];
            a.gyw[gi] = (1.0 + beta) * gxp - beta * a.gx[gi];     // L L^T y_new
            a.x[gi] = xn;
            a.gx[gi] = gxp;
            a.y[gi] = xn + beta * (xn - xo);
        }
        kn = k + 1;
        const bool check = (a.kkt_every > 0 && kn % a.kkt_every == 0) || kn >= a.max_iter;
        if (check) {
            for (int i = threadIdx.x; i < el.n; i += kProjNT) {
                const int gi = r0 + i;
                const double xi = a.x[gi];
                el.v[i] = xi - alpha * (2.0 * a.gx[gi] + 2.0 * gamma * xi);
            }
            __syncthreads();
            P.prepare();
            const ProjOut o = P.solve(a.R, a.mode, mn, mx, st->nu_kkt, st->tau_kkt, a.budget);
            double r2 = 0.0;
            for (int i = threadIdx.x; i < el.n; i += kProjNT) {
                const double pi = fmax(fma(o.nu, el.mu[i], el.v[i]) - o.tau, 0.0);
                const double dd = pi - a.x[r0 + i];
                r2 = fma(dd, dd, r2);
            }
            r2 = P.reduce_double(r2);
            const bool conv = r2 <= a.eps * a.eps;
            const bool stop = conv || kn >= a.max_iter || !(r2 == r2);
            if (rank == 0 && threadIdx.x == 0) {
                st->kkt = sqrt(r2);
                st->nu_kkt = o.nu;
                st->tau_kkt = o.tau;
                st->proj_steps += o.steps;
                st->dykstra += o.dykstra;
                if (o.status != MV_OK) st->proj_fail += 1;
                st->k = kn;
                st->t = tn;
                st->beta_prev = beta;
                if (stop) {
                    st->done = 1;
                    st->converged = conv ? 1 : 0;
                    st->status = conv ? MV_OK : (!(r2 == r2) ? MV_ERR_NUMERIC : MV_ERR_NOT_CONVERGED);
                }
            }
            if (stop) {
                cluster_barrier<CL>();
                return;
            }
            __syncthreads();
        }
    }
    if (rejected) alpha *= a.bt_rho;
    if (numeric || !(alpha > 1e-300)) {
        if (rank == 0 && threadIdx.x == 0) {
            st->done = 1;
            st->status = MV_ERR_NUMERIC;
        }
        cluster_barrier<CL>();
        return;
    }
    // next candidate from y
    for (int i = threadIdx.x; i < el.n; i += kProjNT) {
        const int gi = r0 + i;
        const double yi = a.y[gi];
        el.v[i] = yi - alpha * (2.0 * a.gyw[gi] + 2.0 * gamma * yi);
    }
    __syncthreads();
    P.prepare();
    const ProjOut o = P.solve(a.R, a.mode, mn, mx, st->nu, st->tau, a.budget);
    for (int i = threadIdx.x; i < el.n; i += kProjNT) {
        const int gi = r0 + i;
        const double xpn = fmax(fma(o.nu, el.mu[i], el.v[i]) - o.tau, 0.0);
        a.xp[gi] = xpn;
        a.y32[gi] = (float)((xpn - a.y[gi]) * (a.row_scale ? (double)a.row_scale[gi] : 1.0));
    }
    if (rank == 0 && threadIdx.x == 0) {
        st->k = kn;
        st->t = tn;
        st->beta_prev = beta;
        st->alpha = alpha;
        if (rejected) {
            st->backtracks += 1;
            if (a.momentum == 1) st->beta_c = const_beta(alpha, a.m_f);
        }
        st->bt_started = 1;
        st->nu = o.nu;
        st->tau = o.tau;
        st->proj_steps += o.steps;
        st->dykstra += o.dykstra;
        if (o.status != MV_OK) st->proj_fail += 1;
        if (o.status == MV_ERR_INFEASIBLE || o.status == MV_ERR_NUMERIC) {
            st->done = 1;
            st->status = o.status;
        }
    }
    cluster_barrier<CL>();
}

template <int CL>
__global__ void __launch_bounds__(kProjNT) npga_bt_step_kernel(StepArgs a) {
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ ProjSmem psm;
    npga_bt_step_body<CL>(a, dsm, psm);
}

// FP64 n-vector -> scaled FP32 gemv input.
__global__ void to_y32_kernel(const double *__restrict__ x, const float *__restrict__ row_scale,
                              float *__restrict__ y32, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y32[i] = (float)(x[i] * (row_scale ? (double)row_scale[i] : 1.0));
}

// f(x) = ||z||^2 + gamma ||x||^2 with z = L^T x.
__device__ __forceinline__ void objective_body(SolveState *st, const float *__restrict__ z, int T, const double *__restrict__ x, int n,
                 double gamma) {
    __shared__ double red[(kStepThreads / kWarp + 1) * 5];
    const double zz = sumsq_f32(z, T, red);
    double s[1] = {0.0};
    if (gamma != 0.0)
        for (int i = threadIdx.x; i < n; i += kStepThreads) s[0] = fma(x[i], x[i], s[0]);
    block_sum<1, kStepThreads>(s, red);
    if (threadIdx.x == 0) st->objective = zz + gamma * s[0];
}

__global__ void __launch_bounds__(kStepThreads)
objective_kernel(SolveState *st, const float *__restrict__ z, int T, const double *__restrict__ x, int n,
                 double gamma) {
    objective_body(st, z, T, x, n, gamma);
}

// f(x) = x^T w + gamma ||x||^2 for w = Sigma x or w = L L^T x.
__global__ void __launch_bounds__(kStepThreads)
objective_dot_kernel(SolveState *st, const double *__restrict__ x, const double *__restrict__ sx, int n, double gamma) {
    __shared__ double red[(kStepThreads / kWarp + 1) * 5];
    double v[2] = {0.0, 0.0};
    for (int i = threadIdx.x; i < n; i += kStepThreads) {
        v[0] = fma(x[i], sx[i], v[0]);
        v[1] = fma(x[i], x[i], v[1]);
    }
    block_sum<2, kStepThreads>(v, red);
    if (threadIdx.x == 0) st->objective = v[0] + gamma * v[1];
}

// g = 2 (L z) + 2 gamma y   (gradient building block output).
__global__ void grad_finish_kernel(const double *__restrict__ lz, const double *__restrict__ y, double gamma,
                                   double *__restrict__ g, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) g[i] = 2.0 * lz[i] + 2.0 * gamma * y[i];
}

// ------------------------------------------------------------------ host
static int validate_problem(const mv_problem *P) {
    if (P == nullptr || P->L == nullptr || P->mu == nullptr) return MV_ERR_INVALID_ARG;
    if (P->dtype != MV_F32 && P->dtype != MV_BF16 && P->dtype != MV_FP8_E4M3) return MV_ERR_INVALID_ARG;
    if (P->mode != MV_RETURN_GE && P->mode != MV_RETURN_EQ) return MV_ERR_INVALID_ARG;
    if (P->layout != MV_LAYOUT_NT && P->layout != MV_LAYOUT_TN && P->layout != MV_LAYOUT_SIGMA)
        return MV_ERR_INVALID_ARG;
    if (P->layout == MV_LAYOUT_SIGMA && P->dtype != MV_F32) return MV_ERR_INVALID_ARG;
    if (P->n < 1 || P->T < 1 || P->ld < (P->layout == MV_LAYOUT_NT ? P->T : P->n)) return MV_ERR_INVALID_ARG;
    if (P->n > kProjMaxN || P->T > (1LL << 31) - 1)
        return record_message(MV_ERR_UNSUPPORTED, "problem: n must be <= 32768 and T below 2^31");
    const int es = dtype_size(P->dtype);
    if (((uintptr_t)P->L) % 16 != 0 || (P->ld * es) % 16 != 0) return MV_ERR_INVALID_ARG;
    if (P->dtype == MV_FP8_E4M3 && P->row_scale == nullptr) return MV_ERR_INVALID_ARG;
    if (!(P->gamma >= 0.0) || !(P->R_target == P->R_target)) return MV_ERR_INVALID_ARG;
    return MV_OK;
}

static bool is_tn(const mv_problem *P) { return P->layout == MV_LAYOUT_TN; }
static bool is_sigma(const mv_problem *P) { return P->layout == MV_LAYOUT_SIGMA; }

// The plan of a single-problem call: explicit Sigma, or a factor in either layout.
static Plan plan_for(const mv_problem *P, bool fused) {
    if (is_sigma(P)) return make_plan_sigma(P->n, P->ld);
    return make_plan(P->dtype, P->n, P->T, P->ld, 0, fused, is_tn(P));
}

// The calls that read L only through the NT-layout kernels.
static int require_nt(const mv_problem *P, const char *what) {
    if (P->layout == MV_LAYOUT_NT) return MV_OK;
    char msg[128];
    snprintf(msg, sizeof(msg), "%s: the factor must be stored n x T (MV_LAYOUT_NT)", what);
    return record_message(MV_ERR_UNSUPPORTED, msg);
}

static int check_ws(void *ws, size_t ws_bytes, size_t need) {
    if (need == 0) return MV_OK;
    if (ws == nullptr || ws_bytes < need || ((uintptr_t)ws) % 256 != 0) return MV_ERR_WORKSPACE;
    return MV_OK;
}

template <int DT>
static void launch_gemv_t(const Plan &p, const void *L, const float *w32, float *out32, double *out64,
                          const float *cscale, void *ws, const int *done, cudaStream_t s) {
    dim3 grid(p.t_blocks, p.t_splits);
    gemv_t_kernel<DT><<<grid, kGemvThreads, 0, s>>>(L, p.ld, p.gr, p.gc, w32, at<float>(ws, p.o_zpart), p.zstride,
                                                     out32, at<unsigned>(ws, p.o_tick_t), p.t_rows, done, out64, cscale);
}

template <int DT>
static void launch_gemv_n(const Plan &p, const void *L, const float *w32, const float *rscale, double *out64,
                          float *out32, void *ws, const int *done, cudaStream_t s) {
    dim3 grid(p.n_groups, p.n_splits);
    const size_t smem = (size_t)p.n_cols * 4;
    gemv_n_kernel<DT, kRW><<<grid, kGemvThreads, smem, s>>>(L, p.ld, p.gr, p.gc, w32, rscale, at<float>(ws, p.o_gpart),
                                                           out64, out32, at<unsigned>(ws, p.o_tick_n), p.n_cols, done);
}

// z = L^T y32 into the FP32 T-vector at o_z (y32 pre-multiplied by the FP8 scales).
template <int DT>
static void launch_z_t(const Plan &p, const mv_problem *P, const float *y32, void *ws, const int *done,
                       cudaStream_t s) {
    float *z = at<float>(ws, p.o_z);
    if (p.tn)
        launch_gemv_n<DT>(p, P->L, y32, nullptr, at<double>(ws, p.o_zd), z, ws, done, s);
    else
        launch_gemv_t<DT>(p, P->L, y32, z, nullptr, nullptr, ws, done, s);
}

// g = L z (FP64, FP8 scales applied) and optionally its FP32 copy g32.
template <int DT>
static void launch_g_t(const Plan &p, const mv_problem *P, const float *z, void *ws, const int *done, double *g,
                       float *g32, cudaStream_t s) {
    const float *rs = P->dtype == MV_FP8_E4M3 ? P->row_scale : nullptr;
    if (p.tn)
        launch_gemv_t<DT>(p, P->L, z, g32, g, rs, ws, done, s);
    else
        launch_gemv_n<DT>(p, P->L, z, rs, g, g32, ws, done, s);
}

static void launch_z(const Plan &p, const mv_problem *P, const float *y32, void *ws, const int *done, cudaStream_t s) {
    switch (p.dt) {
        case MV_F32: launch_z_t<MV_F32>(p, P, y32, ws, done, s); break;
        case MV_BF16: launch_z_t<MV_BF16>(p, P, y32, ws, done, s); break;
        default: launch_z_t<MV_FP8_E4M3>(p, P, y32, ws, done, s); break;
    }
}

static void launch_g(const Plan &p, const mv_problem *P, const float *z, void *ws, const int *done, double *g,
                     float *g32, cudaStream_t s) {
    switch (p.dt) {
        case MV_F32: launch_g_t<MV_F32>(p, P, z, ws, done, g, g32, s); break;
        case MV_BF16: launch_g_t<MV_BF16>(p, P, z, ws, done, g, g32, s); break;
        default: launch_g_t<MV_FP8_E4M3>(p, P, z, ws, done, g, g32, s); break;
    }
}

// g = L L^T y (row-scaled) in one pass over L; capturable (no synchronisation).
static int launch_llt(const Plan &p, const mv_problem *P, const float *y32, void *ws, const int *done, double *g_out,
                      float *g32, cudaStream_t s, float *z = nullptr) {
    LltScratch sc = llt_scratch(at<char>(ws, p.o_llt), p.n);
    sc.err = at<int>(ws, p.o_err);             // read back by the solve
    return llt_launch(p.lp, p.dt, P->L, p.n, p.T, p.ld, y32, P->dtype == MV_FP8_E4M3 ? P->row_scale : nullptr, sc,
                      done, g_out, g32, s, z);
}

// Kernel attributes are set once per process, before any stream capture.
template <typename Kern>
static bool cluster_attrs(Kern k, int CL) {
    const int smem = (int)proj_elem_bytes(kProjMaxLocal);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return false;
    if (CL > 8 && cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        return false;
    return true;
}

static int set_kernel_attrs() {
    static std::once_flag once;
    static int status = MV_OK;
    std::call_once(once, [] {
        const int big = 96 * 1024;
        bool ok = cudaFuncSetAttribute(gemv_n_kernel<MV_F32, kRW>, cudaFuncAttributeMaxDynamicSharedMemorySize, big) ==
                      cudaSuccess &&
                  cudaFuncSetAttribute(gemv_n_kernel<MV_BF16, kRW>, cudaFuncAttributeMaxDynamicSharedMemorySize, big) ==
                      cudaSuccess &&
                  cudaFuncSetAttribute(gemv_n_kernel<MV_FP8_E4M3, kRW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       big) == cudaSuccess;
        ok = ok && cluster_attrs(npga_step_kernel<1>, 1) && cluster_attrs(npga_step_kernel<2>, 2) &&
             cluster_attrs(npga_step_kernel<4>, 4) && cluster_attrs(npga_step_kernel<8>, 8) &&
             cluster_attrs(npga_step_kernel<16>, 16);
        ok = ok && cluster_attrs(npga_bt_step_kernel<1>, 1) && cluster_attrs(npga_bt_step_kernel<2>, 2) &&
             cluster_attrs(npga_bt_step_kernel<4>, 4) && cluster_attrs(npga_bt_step_kernel<8>, 8) &&
             cluster_attrs(npga_bt_step_kernel<16>, 16);
        ok = ok && cluster_attrs(init_x_kernel<1>, 1) && cluster_attrs(init_x_kernel<2>, 2) &&
             cluster_attrs(init_x_kernel<4>, 4) && cluster_attrs(init_x_kernel<8>, 8) &&
             cluster_attrs(init_x_kernel<16>, 16);
        if (!ok) status = record_cuda_error(cudaGetLastError(), "kernel attributes", __FILE__, __LINE__);
    });
    return status;
}

static void gemv_pair(const Plan &p, const mv_problem *P, const float *y32, void *ws, const int *done,
                      double *g_out, cudaStream_t s, float *g32 = nullptr) {
    launch_z(p, P, y32, ws, done, s);
    launch_g(p, P, at<float>(ws, p.o_z), ws, done, g_out, g32, s);
}

static void gemv_t_only(const Plan &p, const mv_problem *P, const float *y32, void *ws, cudaStream_t s) {
    launch_z(p, P, y32, ws, nullptr, s);
}

template <typename Kern, typename... Args>
static cudaError_t launch_cluster(Kern kern, int CL, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)CL);
    cfg.blockDim = dim3(kProjNT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

static size_t step_smem(int n, int CL) { return proj_elem_bytes((n + CL - 1) / CL); }

static void launch_step(const Plan &p, const mv_problem *P, const mv_solve_opts *O, void *ws, cudaStream_t s) {
    StepArgs a;
    a.st = at<SolveState>(ws, p.o_state);
    a.gy = at<double>(ws, p.o_gy);
    a.x = at<double>(ws, p.o_x);
    a.y = at<double>(ws, p.o_y);
    a.gx = at<double>(ws, p.o_gx);
    a.y32 = at<float>(ws, p.o_y32);
    a.mu = P->mu;
    a.row_scale = P->dtype == MV_FP8_E4M3 ? P->row_scale : nullptr;
    a.n = p.n;
    a.mode = P->mode;
    a.kkt_every = O->kkt_every;
    a.max_iter = O->max_iter;
    a.R = P->R_target;
    a.gamma = P->gamma;
    a.eps = O->eps;
    a.dyk = O->dykstra_iters > 0 ? at<double>(ws, p.o_dyk) : nullptr;
    a.dyk_iters = O->dykstra_iters;
    a.budget = O->proj_budget;
    a.momentum = O->momentum;
    a.bt_rho = O->bt_rho;
    a.m_f = O->m_f > 0.0 ? O->m_f : 2.0 * P->gamma;
    a.gyw = at<double>(ws, p.o_gy);
    a.gd = at<double>(ws, p.o_gd);
    a.xp = at<double>(ws, p.o_xp);
    const size_t sm = step_smem(p.n, p.cl);
    if (O->backtrack) {
        switch (p.cl) {
            case 1: launch_cluster(npga_bt_step_kernel<1>, 1, sm, s, a); break;
            case 2: launch_cluster(npga_bt_step_kernel<2>, 2, sm, s, a); break;
            case 4: launch_cluster(npga_bt_step_kernel<4>, 4, sm, s, a); break;
            case 8: launch_cluster(npga_bt_step_kernel<8>, 8, sm, s, a); break;
            default: launch_cluster(npga_bt_step_kernel<16>, 16, sm, s, a); break;
        }
        return;
    }
    switch (p.cl) {
        case 1: launch_cluster(npga_step_kernel<1>, 1, sm, s, a); break;
        case 2: launch_cluster(npga_step_kernel<2>, 2, sm, s, a); break;
        case 4: launch_cluster(npga_step_kernel<4>, 4, sm, s, a); break;
        case 8: launch_cluster(npga_step_kernel<8>, 8, sm, s, a); break;
        default: launch_cluster(npga_step_kernel<16>, 16, sm, s, a); break;
    }
}

static void launch_init_x(const Plan &p, const mv_problem *P, const mv_solve_opts *O, const double *x_in, void *ws,
                          cudaStream_t s) {
    SolveState *st = at<SolveState>(ws, p.o_state);
    const float *rs = P->dtype == MV_FP8_E4M3 ? P->row_scale : nullptr;
    double *x = at<double>(ws, p.o_x), *y = at<double>(ws, p.o_y);
    float *y32 = at<float>(ws, p.o_y32);
    double *dyk = O->dykstra_iters > 0 ? at<double>(ws, p.o_dyk) : nullptr;
    const int di = O->dykstra_iters, bud = O->proj_budget;
    const size_t sm = step_smem(p.n, p.cl);
#define MV_INIT_X(CL_) launch_cluster(init_x_kernel<CL_>, CL_, sm, s, st, P->mu, x_in, x, y, y32, rs, p.n, P->R_target, \
                                      P->mode, dyk, di, bud)
    switch (p.cl) {
        case 1: MV_INIT_X(1); break;
        case 2: MV_INIT_X(2); break;
        case 4: MV_INIT_X(4); break;
        case 8: MV_INIT_X(8); break;
        default: MV_INIT_X(16); break;
    }
#undef MV_INIT_X
}

// Sigma y32 -> out64 (and out32) over the upper tiles of Sigma.
static int launch_symv(const Plan &p, const mv_problem *P, const float *y32, void *ws, const int *done, double *out64,
                       float *out32, cudaStream_t s) {
    SymvArgs a;
    a.S = reinterpret_cast<const float *>(P->L);
    a.ld = P->ld;
    a.n = p.n;
    a.nb = p.snb;
    a.y = y32;
    a.part = at<float>(ws, p.o_spart);
    a.tickets = at<unsigned>(ws, p.o_stick);
    a.out64 = out64;
    a.out32 = out32;
    a.done = done;
    a.err = at<int>(ws, p.o_err);
    return symv_launch(a, s);
}

// L L^T y32 -> out64 by whichever product the plan uses (capturable).
static int launch_product(const Plan &p, const mv_problem *P, const float *y32, void *ws, double *out64,
                          cudaStream_t s) {
    if (p.sig) return launch_symv(p, P, y32, ws, nullptr, out64, nullptr, s);
    if (p.use_llt) return launch_llt(p, P, y32, ws, nullptr, out64, nullptr, s);
    gemv_pair(p, P, y32, ws, nullptr, out64, s);
    return MV_OK;
}

// One loop iteration.  With `ev` non-null, events ev[0..3] bracket gemv_t,
// gemv_n and the step kernel (ev[3] is the next iteration's ev[0]); with the
// fused pass, ev[0..1] bracket it and ev[1..2] is empty.
static int launch_iteration(const Plan &p, const mv_problem *P, const mv_solve_opts *O, void *ws,
                            cudaStream_t s, const cudaEvent_t *ev) {
    SolveState *st = at<SolveState>(ws, p.o_state);
    const float *y32 = at<float>(ws, p.o_y32);
    // the product: L L^T y for the step, L L^T d for a backtracking trial
    double *gy = O->backtrack ? at<double>(ws, p.o_gd) : at<double>(ws, p.o_gy);
    const int *done = &st->done;
    if (ev) cudaEventRecord(ev[0], s);
    if (p.use_llt || p.sig) {
        if (p.sig)
            MV_TRY(launch_symv(p, P, y32, ws, done, gy, nullptr, s));
        else
            MV_TRY(launch_llt(p, P, y32, ws, done, gy, nullptr, s, p.want_z ? at<float>(ws, p.o_z) : nullptr));
        if (ev) cudaEventRecord(ev[1], s);
        if (ev) cudaEventRecord(ev[2], s);
        launch_step(p, P, O, ws, s);
        if (ev) cudaEventRecord(ev[3], s);
        return MV_OK;
    }
    launch_z(p, P, y32, ws, done, s);
    if (ev) cudaEventRecord(ev[1], s);
    launch_g(p, P, at<float>(ws, p.o_z), ws, done, gy, nullptr, s);
    if (ev) cudaEventRecord(ev[2], s);
    launch_step(p, P, O, ws, s);
    if (ev) cudaEventRecord(ev[3], s);
    return MV_OK;
}

// Process-wide pool of timing events, reused so cached graphs stay valid.
static std::mutex g_ev_mu;
static std::vector<cudaEvent_t> g_events;
static int timing_events(int count, const cudaEvent_t **out) {
    std::lock_guard<std::mutex> lock(g_ev_mu);
    if ((int)g_events.size() < count) {
        while ((int)g_events.size() < count) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return MV_ERR_CUDA;
            g_events.push_back(e);
        }
    }
    *out = g_events.data();
    return MV_OK;
}

// One cached graph per distinct (problem, options, workspace) triple.
struct GraphKey {
    const void *L, *mu, *rs, *ws;
    int64_t n, T, ld;
    int dt, mode, kkt_every, max_iter, chunk, fused;
    double R, gamma, eps;
    const void *ev;
    int momentum, backtrack, budget, dyk_iters;
    double bt_rho, m_f;
    double aux = 0.0;                    // any further scalar baked into the graph (the adjoint's alpha)
    bool operator==(const GraphKey &o) const {
        return L == o.L && mu == o.mu && rs == o.rs && ws == o.ws && n == o.n && T == o.T && ld == o.ld &&
               dt == o.dt && mode == o.mode && kkt_every == o.kkt_every && max_iter == o.max_iter &&
               chunk == o.chunk && fused == o.fused && R == o.R && gamma == o.gamma && eps == o.eps && ev == o.ev &&
               momentum == o.momentum && backtrack == o.backtrack && budget == o.budget &&
               dyk_iters == o.dyk_iters && bt_rho == o.bt_rho && m_f == o.m_f && aux == o.aux;
    }
};
struct GraphKeyHash {
    size_t operator()(const GraphKey &k) const {
        size_t h = (size_t)k.L ^ ((size_t)k.ws << 1) ^ ((size_t)k.n * 1315423911u) ^ ((size_t)k.T << 7);
        h ^= std::hash<double>()(k.R) + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
        return h;
    }
};
static std::mutex g_graph_mu;
static std::unordered_map<GraphKey, cudaGraphExec_t, GraphKeyHash> g_graphs;

// Returns the cached executable graph of `key`, capturing `enqueue(stream)`
// into it on first use.
template <typename F>
static int cached_graph(const GraphKey &key, F &&enqueue, cudaGraphExec_t *out) {
    std::lock_guard<std::mutex> lock(g_graph_mu);
    auto it = g_graphs.find(key);
    if (it != g_graphs.end()) {
        *out = it->second;
        return MV_OK;
    }
    cudaStream_t cs;
    MV_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaStreamDestroy(cs);
        return MV_ERR_CUDA;
    }
    const int lst = enqueue(cs);
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (lst != MV_OK) {
        if (e == cudaSuccess) cudaGraphDestroy(graph);
        return lst;
    }
    if (e != cudaSuccess) return MV_ERR_CUDA;
    cudaGraphExec_t exec;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return MV_ERR_CUDA;
    if (g_graphs.size() > 32) {
        for (auto &kv : g_graphs) cudaGraphExecDestroy(kv.second);
        g_graphs.clear();
    }
    g_graphs.emplace(key, exec);
    *out = exec;
    return MV_OK;
}

static GraphKey graph_key(const Plan &p, const mv_problem *P, const mv_solve_opts *O, int chunk, const void *ev) {
    return GraphKey{P->L, P->mu, P->row_scale, nullptr, P->n, P->T, P->ld, P->dtype, P->mode, O->kkt_every,
                    O->max_iter, chunk, p.sig ? 2 : (p.use_llt ? (p.want_z ? 3 : 1) : 0), P->R_target, P->gamma, O->eps, ev,
                    O->momentum, O->backtrack, O->proj_budget, O->dykstra_iters, O->bt_rho, O->m_f};
}

static int get_chunk_graph(const Plan &p, const mv_problem *P, const mv_solve_opts *O, void *ws, int chunk,
                           const cudaEvent_t *ev, cudaGraphExec_t *out) {
    GraphKey key = graph_key(p, P, O, chunk, (const void *)ev);
    key.ws = ws;
    return cached_graph(key, [&](cudaStream_t cs) {
        int lst = MV_OK;
        for (int c = 0; c < chunk && lst == MV_OK; ++c) lst = launch_iteration(p, P, O, ws, cs, ev ? ev + 3 * c : nullptr);
        return lst;
    }, out);
}

// The power method of Sec. 3.1: u <- L L^T u / ||L L^T u|| power_iters
// times from the y32 that setup wrote, then the product that lambda_hat
// reads (z = L^T u, or Sigma u); capturable.  Adds the launches to *count.
static int launch_power(const Plan &p, const mv_problem *P, int power_iters, void *ws, cudaStream_t s, int *count) {
    const float *rs = P->dtype == MV_FP8_E4M3 ? P->row_scale : nullptr;
    float *y32 = at<float>(ws, p.o_y32);
    for (int it = 0; it < power_iters; ++it) {
        if (p.sig) {
            MV_TRY(launch_symv(p, P, y32, ws, nullptr, at<double>(ws, p.o_gy), at<float>(ws, p.o_g32), s));
            *count += 2;
        } else if (p.use_llt) {
            MV_TRY(launch_llt(p, P, y32, ws, nullptr, at<double>(ws, p.o_gy), at<float>(ws, p.o_g32), s));
            *count += 2;
        } else {
            gemv_pair(p, P, y32, ws, nullptr, at<double>(ws, p.o_gy), s, at<float>(ws, p.o_g32));
            *count += 3;
        }
        power_norm_kernel<<<1, kStepThreads, 0, s>>>(at<float>(ws, p.o_g32), rs, y32, p.n);
    }
    if (p.sig)
        MV_TRY(launch_symv(p, P, y32, ws, nullptr, at<double>(ws, p.o_gy), nullptr, s));
    else
        gemv_t_only(p, P, y32, ws, s);
    *count += 1;
    return cudaGetLastError() == cudaSuccess ? MV_OK : MV_ERR_CUDA;
}

static int get_power_graph(const Plan &p, const mv_problem *P, const mv_solve_opts *O, void *ws,
                           cudaGraphExec_t *out) {
    GraphKey key = graph_key(p, P, O, -1 - O->power_iters, nullptr);
    key.ws = ws;
    int dummy = 0;
    return cached_graph(key, [&](cudaStream_t cs) { return launch_power(p, P, O->power_iters, ws, cs, &dummy); },
                        out);
}

}  // namespace mv

using namespace mv;

extern "C" {

void mv_solve_opts_default(mv_solve_opts *o) {
    if (!o) return;
    o->max_iter = 10000;
    o->kkt_every = 5;
    o->power_iters = 50;
    o->warm_start = 0;
    o->eps = 1e-6;
    o->power_safety = 1e-3;
    o->alpha = 0.0;
    o->use_graph = 1;
    o->timing = 0;
    o->checkpoint_every = 50;
    o->two_pass = 0;
    o->momentum = 0;
    o->backtrack = 0;
    o->m_f = 0.0;
    o->bt_rho = 0.5;
    o->bt_alpha0 = 0.0;
    o->proj_budget = 100;
    o->dykstra_iters = 2000;
}

size_t mv_npga_workspace_size(const mv_problem *P) {
    if (validate_problem(P) != MV_OK) return 0;
    return plan_for(P, true).total;
}

int mv_gradient(const mv_problem *P, const double *d_y, float *d_z, double *d_g, void *d_ws, size_t ws_bytes,
                mv_stream_t stream) {
    MV_TRY(validate_problem(P));
    if (d_y == nullptr || d_g == nullptr || (is_sigma(P) && d_z != nullptr)) return MV_ERR_INVALID_ARG;
    const Plan p = plan_for(P, true);
    MV_TRY(check_ws(d_ws, ws_bytes, p.total));
    MV_TRY(set_kernel_attrs());
    (void)cudaGetLastError();
    cudaStream_t s = (cudaStream_t)stream;
    float *y32 = at<float>(d_ws, p.o_y32);
    double *lz = at<double>(d_ws, p.o_gy);
    MV_CUDA_TRY(cudaMemsetAsync(at<char>(d_ws, p.o_tick_t), 0, 4 * (size_t)p.t_blocks, s));
    MV_CUDA_TRY(cudaMemsetAsync(at<char>(d_ws, p.o_tick_n), 0, 4 * (size_t)p.n_groups, s));
    const float *rs = P->dtype == MV_FP8_E4M3 ? P->row_scale : nullptr;
    to_y32_kernel<<<(p.n + 255) / 256, 256, 0, s>>>(d_y, rs, y32, p.n);
    if (p.sig) {
        MV_CUDA_TRY(cudaMemsetAsync(at<char>(d_ws, p.o_stick), 0, 4 * (size_t)p.snb, s));
        MV_CUDA_TRY(cudaMemsetAsync(at<char>(d_ws, p.o_err), 0, 16, s));
        MV_TRY(launch_symv(p, P, y32, d_ws, nullptr, lz, nullptr, s));
    } else if (p.use_llt) {
        MV_CUDA_TRY(cudaMemsetAsync(llt_scratch(at<char>(d_ws, p.o_llt), p.n).tickets, 0, llt_ticket_bytes(), s));
        MV_CUDA_TRY(cudaMemsetAsync(at<char>(d_ws, p.o_err), 0, 16, s));
        MV_TRY(launch_llt(p, P, y32, d_ws, nullptr, lz, nullptr, s, d_z ? at<float>(d_ws, p.o_z) : nullptr));
    } else {
        gemv_pair(p, P, y32, d_ws, nullptr, lz, s);
    }
    grad_finish_kernel<<<(p.n + 255) / 256, 256, 0, s>>>(lz, d_y, P->gamma, d_g, p.n);
    if (d_z) MV_CUDA_TRY(cudaMemcpyAsync(d_z, at<float>(d_ws, p.o_z), 4 * (size_t)p.T, cudaMemcpyDeviceToDevice, s));
    MV_CUDA_TRY(cudaGetLastError());
    return MV_OK;
}

int mv_npga_solve(const mv_problem *P, const mv_solve_opts *O_in, double *d_x_inout, mv_solve_info *h_info,
                  void *d_ws, size_t ws_bytes, mv_stream_t stream) {
    MV_TRY(validate_problem(P));
    if (d_x_inout == nullptr || h_info == nullptr) return MV_ERR_INVALID_ARG;
    mv_solve_opts O;
    if (O_in) O = *O_in; else mv_solve_opts_default(&O);
    if (O.max_iter < 0 || O.kkt_every < 0 || O.power_iters < 0 || !(O.eps >= 0.0)) return MV_ERR_INVALID_ARG;
    if ((O.momentum != 0 && O.momentum != 1) || (O.backtrack != 0 && O.backtrack != 1) || O.proj_budget < 1 ||
        O.dykstra_iters < 0)
        return MV_ERR_INVALID_ARG;
    if (O.momentum == 1 && !(O.m_f > 0.0) && !(P->gamma > 0.0))
        return record_message(MV_ERR_INVALID_ARG, "constant momentum needs m_f > 0 or gamma > 0");
    if (O.backtrack == 1 && !(O.bt_rho > 0.0 && O.bt_rho < 1.0)) return MV_ERR_INVALID_ARG;
    const Plan p = plan_for(P, O.two_pass == 0);
    MV_TRY(check_ws(d_ws, ws_bytes, p.total));
    MV_TRY(set_kernel_attrs());
    (void)cudaGetLastError();   // start from a clean error state
    cudaStream_t s = (cudaStream_t)stream;
    SolveState *st = at<SolveState>(d_ws, p.o_state);
    float *y32 = at<float>(d_ws, p.o_y32);
    const float *rs = P->dtype == MV_FP8_E4M3 ? P->row_scale : nullptr;
    *h_info = mv_solve_info{};

    MV_CUDA_TRY(cudaMemsetAsync(at<char>(d_ws, p.o_tick_t), 0, 4 * (size_t)p.t_blocks, s));
    MV_CUDA_TRY(cudaMemsetAsync(at<char>(d_ws, p.o_tick_n), 0, 4 * (size_t)p.n_groups, s));
    MV_CUDA_TRY(cudaMemsetAsync(at<char>(d_ws, p.o_err), 0, 16, s));
    if (p.use_llt) MV_CUDA_TRY(cudaMemsetAsync(llt_scratch(at<char>(d_ws, p.o_llt), p.n).tickets, 0, llt_ticket_bytes(), s));
    if (p.sig) MV_CUDA_TRY(cudaMemsetAsync(at<char>(d_ws, p.o_stick), 0, 4 * (size_t)p.snb, s));
    setup_kernel<<<1, kStepThreads, 0, s>>>(st, P->mu, P->power_start, rs, y32, p.n);
    // Power method for ||L_eff||_2^2 (skipped when the step is given): one
    // cached graph of all its launches, or host-issued when graphs are off.
    int launches = 4;
    if (!(O.alpha > 0.0)) {
        if (O.use_graph && !O.timing) {
            cudaGraphExec_t pexec = nullptr;
            MV_TRY(get_power_graph(p, P, &O, d_ws, &pexec));
            MV_CUDA_TRY(cudaGraphLaunch(pexec, s));
            int cnt = 0;
            for (int it = 0; it < O.power_iters; ++it) cnt += (p.sig || p.use_llt) ? 2 : 3;
            launches += cnt + 1;
        } else {
            MV_TRY(launch_power(p, P, O.power_iters, d_ws, s, &launches));
        }
    }
    if (p.sig)
        step_size_sigma_kernel<<<1, kStepThreads, 0, s>>>(st, y32, at<double>(d_ws, p.o_gy), (O.alpha > 0.0) ? 0 : p.n,
                                                          P->gamma, O.power_safety, O.alpha);
    else
        step_size_kernel<<<1, kStepThreads, 0, s>>>(st, at<float>(d_ws, p.o_z), (O.alpha > 0.0) ? 0 : p.T, P->gamma,
                                                    O.power_safety, O.alpha);
    if (O.momentum || O.backtrack) {
        variant_setup_kernel<<<1, 32, 0, s>>>(st, O.momentum, O.m_f > 0.0 ? O.m_f : 2.0 * P->gamma, O.backtrack,
                                              O.bt_alpha0, O.bt_rho);
        launches += 1;
    }
    launch_init_x(p, P, &O, O.warm_start ? d_x_inout : nullptr, d_ws, s);
    if (O.backtrack) {
        // L L^T y^0 (= L L^T x^0), then the first trial candidate
        MV_TRY(launch_product(p, P, y32, d_ws, at<double>(d_ws, p.o_gy), s));
        MV_CUDA_TRY(cudaMemcpyAsync(at<double>(d_ws, p.o_gx), at<double>(d_ws, p.o_gy), 8 * (size_t)p.n,
                                    cudaMemcpyDeviceToDevice, s));
        launch_step(p, P, &O, d_ws, s);
        launches += 3;
    }
    MV_CUDA_TRY(cudaGetLastError());

    const int chunk = O.kkt_every > 0 ? O.kkt_every : 8;
    const int per_iter = (p.use_llt || p.sig) ? 2 : 3;
    const cudaEvent_t *ev = nullptr;
    if (O.timing) MV_TRY(timing_events(3 * chunk + 1, &ev));
    // Events recorded by graph nodes cannot be timed, so a timed solve issues
    // its kernels from the host (same kernels, same order).
    cudaGraphExec_t exec = nullptr;
    if (O.use_graph && !O.timing) MV_TRY(get_chunk_graph(p, P, &O, d_ws, chunk, nullptr, &exec));
    // max_iter + 1 iterations may run: the last one only evaluates the KKT residual.
    int64_t max_chunks = ((int64_t)O.max_iter + 1 + chunk - 1) / chunk + 1;
    // rejected trial steps take loop slots without advancing k; the step only
    // shrinks, so rejections are few (log(alpha0 / alpha) / log(1 / rho))
    if (O.backtrack) max_chunks += 64 / chunk + 2;
    SolveState hs{};
    int k_prev = 0, timed = 0;
    double t_t = 0.0, t_n = 0.0, t_s = 0.0;
    for (int64_t c = 0; c < max_chunks; ++c) {
        if (exec) {
            MV_CUDA_TRY(cudaGraphLaunch(exec, s));
        } else {
            for (int i = 0; i < chunk; ++i) MV_TRY(launch_iteration(p, P, &O, d_ws, s, ev ? ev + 3 * i : nullptr));
            MV_CUDA_TRY(cudaGetLastError());
        }
        launches += per_iter * chunk;
        MV_CUDA_TRY(cudaMemcpyAsync(&hs, st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        MV_CUDA_TRY(cudaStreamSynchronize(s));
        if (ev) {
            // Iterations that did real work in this chunk: the completed steps
            // plus, on the chunk that converged, the final checking iteration.
            int pairs = hs.k - k_prev + (hs.done ? 1 : 0);
            pairs = pairs < 0 ? 0 : (pairs > chunk ? chunk : pairs);
            for (int i = 0; i < pairs; ++i) {
                float a = 0.f, b = 0.f, d = 0.f;
                MV_CUDA_TRY(cudaEventElapsedTime(&a, ev[3 * i], ev[3 * i + 1]));
                MV_CUDA_TRY(cudaEventElapsedTime(&b, ev[3 * i + 1], ev[3 * i + 2]));
                MV_CUDA_TRY(cudaEventElapsedTime(&d, ev[3 * i + 2], ev[3 * i + 3]));
                t_t += a;
                t_n += b;
                t_s += d;
            }
            timed += pairs;
        }
        k_prev = hs.k;
        if (hs.done) break;
    }
    // Objective of the returned iterate.  A solve that stopped at a KKT test
    // returns the iterate that test evaluated, and the step kept L L^T x
    // there (gx, by linearity from the products at y): f = x^T gx +
    // gamma ||x||^2 with no further pass over L.  Otherwise (an error stop,
    // the iteration budget of the host loop, backtracking) one more pass
    // z = L^T x (or Sigma x).
    const bool at_test = hs.done && !O.backtrack && (hs.status == MV_OK || hs.status == MV_ERR_NOT_CONVERGED);
    if (at_test) {
        objective_dot_kernel<<<1, kStepThreads, 0, s>>>(st, at<double>(d_ws, p.o_x), at<double>(d_ws, p.o_gx), p.n,
                                                        P->gamma);
        launches += 1;
    } else {
        launches += 3;
        to_y32_kernel<<<(p.n + 255) / 256, 256, 0, s>>>(at<double>(d_ws, p.o_x), rs, y32, p.n);
        if (p.sig) {
            MV_TRY(launch_symv(p, P, y32, d_ws, nullptr, at<double>(d_ws, p.o_gobj), nullptr, s));
            objective_dot_kernel<<<1, kStepThreads, 0, s>>>(st, at<double>(d_ws, p.o_x), at<double>(d_ws, p.o_gobj),
                                                            p.n, P->gamma);
        } else {
            gemv_t_only(p, P, y32, d_ws, s);
            objective_kernel<<<1, kStepThreads, 0, s>>>(st, at<float>(d_ws, p.o_z), p.T, at<double>(d_ws, p.o_x), p.n,
                                                        P->gamma);
        }
    }
    MV_CUDA_TRY(cudaMemcpyAsync(d_x_inout, at<double>(d_ws, p.o_x), 8 * (size_t)p.n, cudaMemcpyDeviceToDevice, s));
    MV_CUDA_TRY(cudaMemcpyAsync(&hs, st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    int xerr = 0;
    MV_CUDA_TRY(cudaMemcpyAsync(&xerr, at<int>(d_ws, p.o_err), sizeof(int), cudaMemcpyDeviceToHost, s));
    MV_CUDA_TRY(cudaStreamSynchronize(s));
    MV_CUDA_TRY(cudaGetLastError());
    h_info->iterations = hs.k;
    h_info->status = hs.done ? hs.status : MV_ERR_NOT_CONVERGED;
    if (xerr != 0) {
        char msg[96];
        snprintf(msg, sizeof(msg), "single-pass product: a bounded wait timed out (code %d)", xerr);
        h_info->status = record_message(MV_ERR_TIMEOUT, msg);
    }
    h_info->converged = hs.converged;
    h_info->proj_failures = hs.proj_fail;
    h_info->kkt = hs.kkt;
    h_info->objective = hs.objective;
    h_info->alpha = hs.alpha;
    h_info->lambda_hat = hs.lambda_hat;
    h_info->nu = hs.nu;
    h_info->launches = launches;
    h_info->timed_pairs = timed;
    const bool one_pass = p.use_llt || p.sig;
    h_info->t_gemv_t_ms = one_pass ? 0.0 : t_t;
    h_info->t_gemv_n_ms = one_pass ? 0.0 : t_n;
    h_info->t_fused_ms = one_pass ? t_t : 0.0;
    h_info->fused = p.sig ? 2 : (p.use_llt ? 1 : 0);
    h_info->t_step_ms = t_s;
    h_info->proj_steps = hs.proj_steps;
    h_info->backtracks = hs.backtracks;
    h_info->dykstra = hs.dykstra;
    return h_info->status;
}

}  // extern "C"

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
    const double nu0 = fs->nu, tau0 = fs->tau, nuk0 = fs->nu_kkt, tauk0 = fs->tau_kkt;
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
        const ProjOut o = P.solve(R, a.mode, mn, mx, nuk0, tauk0, kProjBudget);
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
    size_t o_lt, o_y, o_z, o_g, o_x, o_yd, o_gx, o_fs, o_rt, o_gpart, o_gtick, total;
};

static FPlan make_fplan(const Plan &p, int64_t nb) {
    FPlan f{};
    f.B = nb <= 32 ? 32 : (nb <= 64 ? 64 : 128);
    f.BN = 2 * f.B;
    f.ldLt = (p.n + 15) / 16 * 16;                    // row pitch a multiple of 16 bytes for BF16 and FP8
    f.ldY = f.ldLt;
    f.ldZ = ((int64_t)p.T + 7) / 8 * 8;
    size_t off = p.total;
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

static void frontier_gemm_pair(const CUtensorMap *maps, const Plan &p, const FPlan &f, void *ws, cudaStream_t s) {
    if (f.BN == 64) frontier_gemms<64>(maps[0], maps[1], maps[2], maps[3], p, f, ws, s);
    else if (f.BN == 128) frontier_gemms<128>(maps[0], maps[1], maps[2], maps[3], p, f, ws, s);
    else frontier_gemms<256>(maps[0], maps[1], maps[2], maps[3], p, f, ws, s);
}

// L^T X for the objectives, X already written as the split operand.
static void frontier_ltx(const CUtensorMap *maps, const Plan &p, const FPlan &f, void *ws, cudaStream_t s) {
    __nv_bfloat16 *Zt = at<__nv_bfloat16>(ws, f.o_z);
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
    MV_TRY(validate_problem(P));
    MV_TRY(require_nt(P, "frontier solve"));
    if (P->dtype == MV_F32)
        return record_message(MV_ERR_UNSUPPORTED, "frontier solve: L must be BF16 or FP8 (the tensor-core operand)");
    if (d_R_targets == nullptr || d_X == nullptr || h_infos == nullptr || n_targets < 1 || n_targets > 128)
        return MV_ERR_INVALID_ARG;
    mv_solve_opts O;
    if (O_in) O = *O_in; else mv_solve_opts_default(&O);
    if (O.max_iter < 0 || O.kkt_every < 0 || O.power_iters < 0 || !(O.eps >= 0.0)) return MV_ERR_INVALID_ARG;
    if (O.momentum != 0 || O.backtrack != 0)
        return record_message(MV_ERR_UNSUPPORTED, "frontier solve: fixed step and FISTA momentum only");
    const Plan p = make_plan(P->dtype, P->n, P->T, P->ld, 0, true);   // power method: fused pass
    const FPlan f = make_fplan(p, n_targets);
    MV_TRY(check_ws(d_ws, ws_bytes, f.total));
    MV_TRY(set_kernel_attrs());
    MV_TRY(frontier_attrs());
    (void)cudaGetLastError();
    cudaStream_t s = (cudaStream_t)stream;
    SolveState *st = at<SolveState>(d_ws, p.o_state);
    float *y32 = at<float>(d_ws, p.o_y32);
    const int B = f.B, nt = (int)n_targets;

    // Targets: the caller's n_targets, padded to B by repeating the last one (padded targets are ignored).
    double *Rt = at<double>(d_ws, f.o_rt);
    MV_CUDA_TRY(cudaMemcpyAsync(Rt, d_R_targets, 8 * (size_t)nt, cudaMemcpyDeviceToDevice, s));
    for (int b = nt; b < B; ++b)
        MV_CUDA_TRY(cudaMemcpyAsync(Rt + b, d_R_targets + nt - 1, 8, cudaMemcpyDeviceToDevice, s));

    // Shared step size from the power method on L (the single-problem GEMV path).
    MV_CUDA_TRY(cudaMemsetAsync(at<char>(d_ws, p.o_tick_t), 0, 4 * (size_t)p.t_blocks, s));
    MV_CUDA_TRY(cudaMemsetAsync(at<char>(d_ws, p.o_tick_n), 0, 4 * (size_t)p.n_groups, s));
    const float *rs = P->dtype == MV_FP8_E4M3 ? P->row_scale : nullptr;
    setup_kernel<<<1, kStepThreads, 0, s>>>(st, P->mu, P->power_start, rs, y32, p.n);
    if (p.use_llt) {
        MV_CUDA_TRY(cudaMemsetAsync(llt_scratch(at<char>(d_ws, p.o_llt), p.n).tickets, 0, llt_ticket_bytes(), s));
        MV_CUDA_TRY(cudaMemsetAsync(at<char>(d_ws, p.o_err), 0, 16, s));
    }
    for (int it = 0; it < O.power_iters; ++it) {
        if (p.use_llt)
            MV_TRY(launch_llt(p, P, y32, d_ws, nullptr, at<double>(d_ws, p.o_gy), at<float>(d_ws, p.o_g32), s));
        else
            gemv_pair(p, P, y32, d_ws, nullptr, at<double>(d_ws, p.o_gy), s, at<float>(d_ws, p.o_g32));
        power_norm_kernel<<<1, kStepThreads, 0, s>>>(at<float>(d_ws, p.o_g32), rs, y32, p.n);
    }
    if (O.power_iters > 0) gemv_t_only(p, P, y32, d_ws, s);
    step_size_kernel<<<1, kStepThreads, 0, s>>>(st, at<float>(d_ws, p.o_z), (O.alpha > 0.0 || O.power_iters == 0) ? 0 : p.T,
                                                P->gamma, O.power_safety, O.alpha);
    const dim3 tgrid((unsigned)((p.T + 31) / 32), (unsigned)((p.n + 31) / 32));
    if (P->dtype == MV_FP8_E4M3)
        transpose_elem_kernel<uint8_t><<<tgrid, dim3(32, 8), 0, s>>>(
            reinterpret_cast<const uint8_t *>(P->L), p.n, p.T, P->ld, at<uint8_t>(d_ws, f.o_lt), f.ldLt);
    else
        transpose_elem_kernel<__nv_bfloat16><<<tgrid, dim3(32, 8), 0, s>>>(
            reinterpret_cast<const __nv_bfloat16 *>(P->L), p.n, p.T, P->ld, at<__nv_bfloat16>(d_ws, f.o_lt), f.ldLt);
    MV_CUDA_TRY(cudaMemsetAsync(at<char>(d_ws, f.o_y), 0, 2 * (size_t)f.BN * f.ldY, s));
    MV_CUDA_TRY(cudaMemsetAsync(at<char>(d_ws, f.o_gtick), 0, 4 * (size_t)((p.n + kBM - 1) / kBM) + 64, s));
    MV_CUDA_TRY(cudaGetLastError());

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
    a.eps = O.eps;
    MV_CUDA_TRY(launch_frontier(true, p.cl, a, s));

    CUtensorMap maps[4];
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
    int launches = 3 + 3 * O.power_iters + 1 + 2;
    cudaGraphExec_t exec = nullptr;
    if (O.use_graph) {
        cudaStream_t cs;
        MV_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            for (int c = 0; c < chunk; ++c) {
                frontier_gemm_pair(maps, p, f, d_ws, cs);
                launch_frontier(false, p.cl, a, cs);
            }
            if (cudaStreamEndCapture(cs, &graph) == cudaSuccess) {
                if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) exec = nullptr;
                cudaGraphDestroy(graph);
            }
        }
        cudaStreamDestroy(cs);
        (void)cudaGetLastError();
    }
    std::vector<FState> hf(B);
    const int64_t max_chunks = ((int64_t)O.max_iter + 1 + chunk - 1) / chunk + 1;
    for (int64_t c = 0; c < max_chunks; ++c) {
        if (exec) {
            MV_CUDA_TRY(cudaGraphLaunch(exec, s));
        } else {
            for (int i = 0; i < chunk; ++i) {
                frontier_gemm_pair(maps, p, f, d_ws, s);
                MV_CUDA_TRY(launch_frontier(false, p.cl, a, s));
            }
        }
        launches += 3 * chunk;
        MV_CUDA_TRY(cudaMemcpyAsync(hf.data(), a.fs, sizeof(FState) * B, cudaMemcpyDeviceToHost, s));
        MV_CUDA_TRY(cudaStreamSynchronize(s));
        bool all = true;
        for (int b = 0; b < nt; ++b) all = all && hf[b].done;
        if (all) break;
    }
    if (exec) cudaGraphExecDestroy(exec);
    // Objectives: one more L^T X product with X written as the split operand.
    split_rows_kernel<<<(unsigned)((B * (int64_t)p.n + 255) / 256), 256, 0, s>>>(a.X, B, p.n, a.Ysplit, f.ldY, rs);
    frontier_ltx(maps, p, f, d_ws, s);
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
        I.iterations = hf[b].k;
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

}  // extern "C"

// ---------------------------------------------------------------------------
// Adjoint of the unrolled solve (reverse sweep with checkpointed recompute).
namespace mv {

// Cluster-wide FP64 sums of NV values per thread, added in a fixed order.
template <int CL, int NV>
__device__ void cluster_sums(ProjSmem *sh, double (&v)[NV], double *dslots /* [2][CL][NV] smem */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ double wsum[kProjNT / kWarp][NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) wsum[warp][k] = v[k];
    __syncthreads();
    const int par = sh->parity;
    if (threadIdx.x == 0) {
        double t[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) t[k] = 0.0;
        for (int w = 0; w < kProjNT / kWarp; ++w)
#pragma unroll
            for (int k = 0; k < NV; ++k) t[k] += wsum[w][k];
        const int me = cluster_rank<CL>();
        for (int r = 0; r < CL; ++r) {
            double *dst = dslots + ((size_t)par * CL + me) * NV;
            if constexpr (CL > 1) dst = cg::this_cluster().map_shared_rank(dst, r);
#pragma unroll
            for (int k = 0; k < NV; ++k) dst[k] = t[k];
        }
    }
    cluster_barrier<CL>();
    __shared__ double res[NV];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double a = 0.0;
            for (int r = 0; r < CL; ++r) a += dslots[((size_t)par * CL + r) * NV + k];
            res[k] = a;
        }
        sh->parity = par ^ 1;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = res[k];
    __syncthreads();
}

struct AdjArgs {
    const double *x1;          // x_{k+1} (support and values)
    // nu_j (the return-row multiplier of that projection) and beta_{k0 + j}
    // are read on the device, so a captured segment replays for any k0
    const double *nu_tape;     // segment tape of nu
    const double *betas;       // beta_k, k = 0 .. K-1
    const int *k0;             // first iteration of the segment
    int j;                     // position in the segment
    int eq;                    // 1: equality mode (the return row always tight)
    double *xbar, *ybar, *mubar;
    double *vbar;              // out: v_bar (FP64)
    float *vbar32;             // out: v_bar as the gemv input
    float *vrec;               // out: v_bar row of the dL update
    const double *mu;
    int n;
};

// One backward step through the projection and the momentum update.
template <int CL>
__global__ void __launch_bounds__(kProjNT) adj_proj_kernel(AdjArgs a) {
    __shared__ ProjSmem psm;
    __shared__ double dsl[2 * kProjMaxCL * 5];
    const int rank = cluster_rank<CL>();
    const int n = a.n, nl = (n + CL - 1) / CL, r0 = min(n, rank * nl), r1 = min(n, r0 + nl);
    const double nu = a.nu_tape[a.j], beta = a.betas[*a.k0 + a.j];
    const bool active = a.eq || nu != 0.0;
    proj_smem_init(&psm);
    double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};   // |S|, sum mu, sum mu^2, sum a, sum mu a
    for (int i = r0 + threadIdx.x; i < r1; i += kProjNT) {
        if (a.x1[i] > 0.0) {
            const double m = a.mu[i], ab = a.xbar[i] + (1.0 + beta) * a.ybar[i];
            s[0] += 1.0;
            s[1] += m;
            s[2] = fma(m, m, s[2]);
            s[3] += ab;
            s[4] = fma(m, ab, s[4]);
        }
    }
    cluster_sums<CL, 5>(&psm, s, dsl);
    double c1 = 0.0, c2 = 0.0;
    const double det = s[0] * s[2] - s[1] * s[1];
    // With mu constant on S (or |S| = 1) the return row adds nothing to the
    // budget row: project on span(1) only (x does not move with mu there).
    const bool two = active && det > 1e-14 * s[0] * s[2];
    if (two) {
        c1 = (s[2] * s[3] - s[1] * s[4]) / det;
        c2 = (s[0] * s[4] - s[1] * s[3]) / det;
    } else if (s[0] > 0.0) {
        c1 = s[3] / s[0];
    }
    for (int i = r0 + threadIdx.x; i < r1; i += kProjNT) {
        const double ab = a.xbar[i] + (1.0 + beta) * a.ybar[i];
        const double xi = a.x1[i];
        double vb = 0.0;
        if (xi > 0.0) {
            vb = ab - c1 - c2 * a.mu[i];
            if (two) a.mubar[i] += nu * vb - xi * c2;
        }
        a.xbar[i] = -beta * a.ybar[i];
        a.vbar[i] = vb;
        a.vbar32[i] = (float)vb;
        a.vrec[i] = (float)vb;
    }
    cluster_barrier<CL>();
}

// y_bar = v_bar - alpha (2 L L^T v_bar + 2 gamma v_bar).
__global__ void adj_finish_kernel(const double *__restrict__ vbar, const double *__restrict__ llv, double alpha,
                                  double gamma, double *__restrict__ ybar, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) ybar[i] = vbar[i] - alpha * (2.0 * llv[i] + 2.0 * gamma * vbar[i]);
}

static int adj_attrs() {
    static std::once_flag once;
    static int st = MV_OK;
    std::call_once(once, [] {
        bool ok = true;
        if (cudaFuncSetAttribute(adj_proj_kernel<16>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
            ok = false;
        if (!ok) st = record_cuda_error(cudaGetLastError(), "adjoint kernel attributes", __FILE__, __LINE__);
    });
    return st;
}

static cudaError_t launch_adj_proj(int CL, const AdjArgs &a, cudaStream_t s) {
    switch (CL) {
        case 1: return launch_cluster(adj_proj_kernel<1>, 1, 0, s, a);
        case 2: return launch_cluster(adj_proj_kernel<2>, 2, 0, s, a);
        case 4: return launch_cluster(adj_proj_kernel<4>, 4, 0, s, a);
        case 8: return launch_cluster(adj_proj_kernel<8>, 8, 0, s, a);
        default: return launch_cluster(adj_proj_kernel<16>, 16, 0, s, a);
    }
}

struct BPlan {
    int K, C, ncp;
    int W;                                                  // columns per piece segment of the dL GEMM operands
    size_t o_cp_state, o_cp_x, o_cp_y, o_cp_gx, o_cp_y32;   // checkpoints
    size_t o_x1, o_vy, o_zw, o_nu;                          // segment tape
    size_t o_xbar, o_ybar, o_mubar, o_vbar, o_betas, o_k0;
    size_t o_ga, o_gb;                                      // split operands of the dL update (BF16, K-major)
    size_t total;
};

static BPlan make_bplan(const Plan &p, int K, int C) {
    BPlan b{};
    b.K = K;
    b.C = C;
    b.ncp = (K + C - 1) / C;
    size_t off = p.total;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    b.o_cp_state = take(sizeof(SolveState) * (size_t)b.ncp);
    b.o_cp_x = take(8 * (size_t)p.n * b.ncp);
    b.o_cp_y = take(8 * (size_t)p.n * b.ncp);
    b.o_cp_gx = take(8 * (size_t)p.n * b.ncp);
    b.o_cp_y32 = take(4 * (size_t)p.n * b.ncp);
    b.o_x1 = take(8 * (size_t)p.n * C);
    b.o_vy = take(4 * (size_t)p.n * 2 * C);        // rows 0..C-1: v_bar_k, rows C..2C-1: y_k
    b.o_zw = take(4 * (size_t)p.T * 2 * C);        // rows 0..C-1: z_k,     rows C..2C-1: w_k
    b.o_nu = take(8 * (size_t)C);
    b.o_xbar = take(8 * (size_t)p.n);
    b.o_ybar = take(8 * (size_t)p.n);
    b.o_mubar = take(8 * (size_t)p.n);
    b.o_vbar = take(8 * (size_t)p.n);
    b.o_betas = take(8 * (size_t)K);
    b.o_k0 = take(16);
    b.W = (2 * C + kBK - 1) / kBK * kBK;
    b.o_ga = take(2 * (size_t)p.n * kSplit3 * b.W);
    b.o_gb = take(2 * (size_t)p.T * kSplit3 * b.W);
    b.total = off;
    return b;
}

// dL += -2 alpha sum_k (v_bar_k z_k^T + y_k w_k^T) over one segment as ONE
// tcgen05 GEMM: with R = 2 len stacked vectors, A = [v_bar_k; y_k]^T (n x R)
// and B = [z_k; w_k]^T (T x R) are split into three BF16 pieces each
// (split3_t_kernel) and C = d_dL accumulates alpha A' B'^T (FP32-accurate).
static int adjoint_dl_update(const BPlan &b, int n, int T, int len, const float *VY, const float *ZW, double alpha,
                             void *ws, float *d_dL, int64_t ldD, cudaStream_t s) {
    const int R = 2 * len, KW = kSplit3 * b.W;
    __nv_bfloat16 *ga = at<__nv_bfloat16>(ws, b.o_ga), *gb = at<__nv_bfloat16>(ws, b.o_gb);
    split3_t_kernel<<<dim3((n + 31) / 32, (b.W + 31) / 32), 256, 0, s>>>(VY, R, n, n, b.W, 0, ga, KW);
    split3_t_kernel<<<dim3((T + 31) / 32, (b.W + 31) / 32), 256, 0, s>>>(ZW, R, T, T, b.W, 1, gb, KW);
    CUtensorMap ta, tb;
    MV_TRY(make_map_bf16(&ta, ga, n, KW, KW, kBM));
    MV_TRY(make_map_bf16(&tb, gb, T, KW, KW, 256));
    gemm_launch<256, kEpiAccF32>(ta, tb, n, T, KW, d_dL, ldD, nullptr, 0, s, 1, nullptr, nullptr,
                                 (float)(-2.0 * alpha));
    MV_CUDA_TRY(cudaGetLastError());
    return MV_OK;
}

}  // namespace mv

extern "C" {

size_t mv_backward_workspace_size(const mv_problem *P, const mv_solve_opts *O_in) {
    if (validate_problem(P) != MV_OK || P->layout != MV_LAYOUT_NT || P->dtype != MV_F32) return 0;
    mv_solve_opts O;
    if (O_in) O = *O_in; else mv_solve_opts_default(&O);
    if (O.max_iter < 1 || O.checkpoint_every < 1) return 0;
    const Plan p = make_plan(P->dtype, P->n, P->T, P->ld, 0, true);
    return make_bplan(p, O.max_iter, O.checkpoint_every).total;
}

int mv_npga_backward(const mv_problem *P, const mv_solve_opts *O_in, const double *d_x0, const double *d_dloss_dx,
                     double *d_dmu, float *d_dL, int64_t ldD, mv_solve_info *h_info, void *d_ws, size_t ws_bytes,
                     mv_stream_t stream) {
    MV_TRY(validate_problem(P));
    MV_TRY(require_nt(P, "mv_npga_backward"));
    if (P->dtype != MV_F32) return record_message(MV_ERR_UNSUPPORTED, "mv_npga_backward: FP32 factor only");
    if (!d_dloss_dx || !d_dmu || !d_dL || !h_info || ldD < P->T) return MV_ERR_INVALID_ARG;
    mv_solve_opts O;
    if (O_in) O = *O_in; else mv_solve_opts_default(&O);
    if (O.max_iter < 1 || O.checkpoint_every < 1 || O.power_iters < 0) return MV_ERR_INVALID_ARG;
    if (O.momentum != 0 || O.backtrack != 0)
        return record_message(MV_ERR_UNSUPPORTED, "mv_npga_backward: differentiates the fixed-step FISTA loop only");
    if (O.proj_budget < 1 || O.dykstra_iters < 0) return MV_ERR_INVALID_ARG;
    O.kkt_every = 0;          // unrolled: no early stop inside the K iterations
    O.eps = 0.0;
    // one pass over L per product, which also returns z = L^T y for the dL update
    Plan p = make_plan(P->dtype, P->n, P->T, P->ld, 0, true);
    p.want_z = true;
    const BPlan b = make_bplan(p, O.max_iter, O.checkpoint_every);
    MV_TRY(check_ws(d_ws, ws_bytes, b.total));
    MV_TRY(set_kernel_attrs());
    MV_TRY(adj_attrs());
    MV_TRY((gemm_set_attrs<256, kEpiAccF32>()));
    (void)cudaGetLastError();
    cudaStream_t s = (cudaStream_t)stream;
    void *ws = d_ws;
    SolveState *st = at<SolveState>(ws, p.o_state);
    float *y32 = at<float>(ws, p.o_y32);
    const int n = p.n, T = p.T, K = b.K, C = b.C;
    {
        int zero = 0;
        MV_CUDA_TRY(cudaMemcpyToSymbolAsync(g_gemm_err, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    }

    // ---- forward to x_K, checkpointing the state before iterations 0, C, 2C, ...
    MV_CUDA_TRY(cudaMemsetAsync(at<char>(ws, p.o_tick_t), 0, 4 * (size_t)p.t_blocks, s));
    MV_CUDA_TRY(cudaMemsetAsync(at<char>(ws, p.o_tick_n), 0, 4 * (size_t)p.n_groups, s));
    MV_CUDA_TRY(cudaMemsetAsync(at<char>(ws, p.o_err), 0, 16, s));
    if (p.use_llt) MV_CUDA_TRY(cudaMemsetAsync(llt_scratch(at<char>(ws, p.o_llt), p.n).tickets, 0, llt_ticket_bytes(), s));
    setup_kernel<<<1, kStepThreads, 0, s>>>(st, P->mu, P->power_start, nullptr, y32, n);
    if (!(O.alpha > 0.0)) {
        for (int it = 0; it < O.power_iters; ++it) {
            if (p.use_llt)
                MV_TRY(launch_llt(p, P, y32, ws, nullptr, at<double>(ws, p.o_gy), at<float>(ws, p.o_g32), s));
            else
                gemv_pair(p, P, y32, ws, nullptr, at<double>(ws, p.o_gy), s, at<float>(ws, p.o_g32));
            power_norm_kernel<<<1, kStepThreads, 0, s>>>(at<float>(ws, p.o_g32), nullptr, y32, n);
        }
        if (p.use_llt)
            MV_TRY(launch_llt(p, P, y32, ws, nullptr, at<double>(ws, p.o_gy), nullptr, s, at<float>(ws, p.o_z)));
        else
            gemv_t_only(p, P, y32, ws, s);
    }
    step_size_kernel<<<1, kStepThreads, 0, s>>>(st, at<float>(ws, p.o_z), (O.alpha > 0.0) ? 0 : T, P->gamma,
                                                O.power_safety, O.alpha);
    launch_init_x(p, P, &O, d_x0, ws, s);
    auto save_cp = [&](int c) -> int {
        MV_CUDA_TRY(cudaMemcpyAsync(at<SolveState>(ws, b.o_cp_state) + c, st, sizeof(SolveState),
                                    cudaMemcpyDeviceToDevice, s));
        MV_CUDA_TRY(cudaMemcpyAsync(at<double>(ws, b.o_cp_x) + (size_t)c * n, at<double>(ws, p.o_x), 8 * (size_t)n,
                                    cudaMemcpyDeviceToDevice, s));
        MV_CUDA_TRY(cudaMemcpyAsync(at<double>(ws, b.o_cp_y) + (size_t)c * n, at<double>(ws, p.o_y), 8 * (size_t)n,
                                    cudaMemcpyDeviceToDevice, s));
        MV_CUDA_TRY(cudaMemcpyAsync(at<double>(ws, b.o_cp_gx) + (size_t)c * n, at<double>(ws, p.o_gx), 8 * (size_t)n,
                                    cudaMemcpyDeviceToDevice, s));
        MV_CUDA_TRY(cudaMemcpyAsync(at<float>(ws, b.o_cp_y32) + (size_t)c * n, y32, 4 * (size_t)n,
                                    cudaMemcpyDeviceToDevice, s));
        return MV_OK;
    };
    auto load_cp = [&](int c) -> int {
        MV_CUDA_TRY(cudaMemcpyAsync(st, at<SolveState>(ws, b.o_cp_state) + c, sizeof(SolveState),
                                    cudaMemcpyDeviceToDevice, s));
        MV_CUDA_TRY(cudaMemcpyAsync(at<double>(ws, p.o_x), at<double>(ws, b.o_cp_x) + (size_t)c * n, 8 * (size_t)n,
                                    cudaMemcpyDeviceToDevice, s));
        MV_CUDA_TRY(cudaMemcpyAsync(at<double>(ws, p.o_y), at<double>(ws, b.o_cp_y) + (size_t)c * n, 8 * (size_t)n,
                                    cudaMemcpyDeviceToDevice, s));
        MV_CUDA_TRY(cudaMemcpyAsync(at<double>(ws, p.o_gx), at<double>(ws, b.o_cp_gx) + (size_t)c * n, 8 * (size_t)n,
                                    cudaMemcpyDeviceToDevice, s));
        MV_CUDA_TRY(cudaMemcpyAsync(y32, at<float>(ws, b.o_cp_y32) + (size_t)c * n, 4 * (size_t)n,
                                    cudaMemcpyDeviceToDevice, s));
        return MV_OK;
    };
    int launches = 4;
    const int per_it = p.use_llt ? 2 : 3;
    for (int c = 0; c < b.ncp; ++c) {
        MV_TRY(save_cp(c));
        const int len = std::min(K, (c + 1) * C) - c * C;
        if (len == C && O.use_graph) {               // a full segment: one cached graph
            cudaGraphExec_t exec = nullptr;
            MV_TRY(get_chunk_graph(p, P, &O, ws, C, nullptr, &exec));
            MV_CUDA_TRY(cudaGraphLaunch(exec, s));
        } else {
            for (int j = 0; j < len; ++j) MV_TRY(launch_iteration(p, P, &O, ws, s, nullptr));
        }
        launches += per_it * len;
    }
    MV_CUDA_TRY(cudaGetLastError());
    SolveState hs{};
    MV_CUDA_TRY(cudaMemcpyAsync(&hs, st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    MV_CUDA_TRY(cudaStreamSynchronize(s));
    if (hs.status != MV_OK && hs.status != MV_ERR_NOT_CONVERGED) {
        *h_info = mv_solve_info{};
        h_info->status = hs.status;
        return hs.status;
    }
    const double alpha = hs.alpha;
    // FISTA betas, the same recurrence in FP64 as the step kernel.
    std::vector<double> beta(K);
    {
        double t = 1.0;
        for (int k = 0; k < K; ++k) {
            const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
            beta[k] = (t - 1.0) / tn;
            t = tn;
        }
    }

    // ---- reverse sweep, segment by segment
    double *xbar = at<double>(ws, b.o_xbar), *ybar = at<double>(ws, b.o_ybar), *mubar = at<double>(ws, b.o_mubar);
    double *vbar = at<double>(ws, b.o_vbar);
    float *VY = at<float>(ws, b.o_vy), *ZW = at<float>(ws, b.o_zw);
    double *X1 = at<double>(ws, b.o_x1), *NU = at<double>(ws, b.o_nu);
    MV_CUDA_TRY(cudaMemcpyAsync(xbar, d_dloss_dx, 8 * (size_t)n, cudaMemcpyDeviceToDevice, s));
    MV_CUDA_TRY(cudaMemsetAsync(ybar, 0, 8 * (size_t)n, s));
    MV_CUDA_TRY(cudaMemsetAsync(mubar, 0, 8 * (size_t)n, s));
    MV_CUDA_TRY(cudaMemset2DAsync(d_dL, 4 * (size_t)ldD, 0, 4 * (size_t)T, (size_t)n, s));
    double *betas = at<double>(ws, b.o_betas);
    int *k0d = at<int>(ws, b.o_k0);
    MV_CUDA_TRY(cudaMemcpyAsync(betas, beta.data(), 8 * (size_t)K, cudaMemcpyHostToDevice, s));
    std::vector<int> k0s(b.ncp);
    for (int seg = 0; seg < b.ncp; ++seg) k0s[seg] = seg * C;
    // recompute a segment forward from its checkpoint, recording y_k, z_k, x_{k+1}, nu_k
    auto recompute = [&](cudaStream_t cs, int len) -> int {
        for (int j = 0; j < len; ++j) {
            MV_CUDA_TRY(cudaMemcpyAsync(VY + (size_t)(len + j) * n, y32, 4 * (size_t)n, cudaMemcpyDeviceToDevice, cs));
            MV_TRY(launch_iteration(p, P, &O, ws, cs, nullptr));
            MV_CUDA_TRY(cudaMemcpyAsync(ZW + (size_t)j * T, at<float>(ws, p.o_z), 4 * (size_t)T,
                                        cudaMemcpyDeviceToDevice, cs));
            MV_CUDA_TRY(cudaMemcpyAsync(X1 + (size_t)j * n, at<double>(ws, p.o_x), 8 * (size_t)n,
                                        cudaMemcpyDeviceToDevice, cs));
            MV_CUDA_TRY(cudaMemcpyAsync(NU + j, &st->nu, 8, cudaMemcpyDeviceToDevice, cs));
        }
        return MV_OK;
    };
    // backward through the segment (iteration k0 + j, j = len - 1 .. 0)
    auto reverse = [&](cudaStream_t cs, int len) -> int {
        for (int j = len - 1; j >= 0; --j) {
            AdjArgs a;
            a.x1 = X1 + (size_t)j * n;
            a.nu_tape = NU;
            a.betas = betas;
            a.k0 = k0d;
            a.j = j;
            a.eq = P->mode == MV_RETURN_EQ ? 1 : 0;
            a.xbar = xbar;
            a.ybar = ybar;
            a.mubar = mubar;
            a.vbar = vbar;
            a.vbar32 = y32;
            a.vrec = VY + (size_t)j * n;
            a.mu = P->mu;
            a.n = n;
            MV_CUDA_TRY(launch_adj_proj(p.cl, a, cs));
            // w = L^T v_bar (z buffer) and L w
            if (p.use_llt)
                MV_TRY(launch_llt(p, P, y32, ws, nullptr, at<double>(ws, p.o_gy), nullptr, cs, at<float>(ws, p.o_z)));
            else
                gemv_pair(p, P, y32, ws, nullptr, at<double>(ws, p.o_gy), cs);
            MV_CUDA_TRY(cudaMemcpyAsync(ZW + (size_t)(len + j) * T, at<float>(ws, p.o_z), 4 * (size_t)T,
                                        cudaMemcpyDeviceToDevice, cs));
            adj_finish_kernel<<<(n + 255) / 256, 256, 0, cs>>>(vbar, at<double>(ws, p.o_gy), alpha, P->gamma, ybar, n);
        }
        return cudaGetLastError() == cudaSuccess ? MV_OK : MV_ERR_CUDA;
    };
    for (int seg = b.ncp - 1; seg >= 0; --seg) {
        const int k0 = seg * C, k1 = std::min(K, k0 + C), len = k1 - k0;
        MV_TRY(load_cp(seg));
        MV_CUDA_TRY(cudaMemcpyAsync(k0d, &k0s[seg], sizeof(int), cudaMemcpyHostToDevice, s));
        if (len == C && O.use_graph) {                // full segments replay two cached graphs
            GraphKey kr = graph_key(p, P, &O, -1000000 - C, nullptr), kb = graph_key(p, P, &O, -2000000 - C, nullptr);
            kr.ws = kb.ws = ws;
            kb.aux = alpha;                           // adj_finish bakes the step in
            cudaGraphExec_t er = nullptr, eb = nullptr;
            MV_TRY(cached_graph(kr, [&](cudaStream_t cs) { return recompute(cs, C); }, &er));
            MV_TRY(cached_graph(kb, [&](cudaStream_t cs) { return reverse(cs, C); }, &eb));
            MV_CUDA_TRY(cudaGraphLaunch(er, s));
            MV_CUDA_TRY(cudaGraphLaunch(eb, s));
        } else {
            MV_TRY(recompute(s, len));
            MV_TRY(reverse(s, len));
        }
        launches += len * (per_it + 4);
        // dL += -2 alpha (V Z^T + Y W^T) over the segment: one tcgen05 GEMM.
        MV_TRY(adjoint_dl_update(b, n, T, len, VY, ZW, alpha, ws, d_dL, ldD, s));
    }
    MV_CUDA_TRY(cudaMemcpyAsync(d_dmu, mubar, 8 * (size_t)n, cudaMemcpyDeviceToDevice, s));
    int xerr = 0, gerr = 0;
    MV_CUDA_TRY(cudaMemcpyAsync(&xerr, at<int>(ws, p.o_err), sizeof(int), cudaMemcpyDeviceToHost, s));
    MV_CUDA_TRY(cudaMemcpyFromSymbolAsync(&gerr, g_gemm_err, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    MV_CUDA_TRY(cudaStreamSynchronize(s));
    MV_CUDA_TRY(cudaGetLastError());
    if (gerr != 0) {
        *h_info = mv_solve_info{};
        h_info->status = record_message(MV_ERR_TIMEOUT, "mv_npga_backward: the dL GEMM pipeline wait timed out");
        return h_info->status;
    }
    if (xerr != 0) {
        char msg[96];
        snprintf(msg, sizeof(msg), "mv_npga_backward: a bounded wait of the fused pass timed out (code %d)", xerr);
        *h_info = mv_solve_info{};
        h_info->status = record_message(MV_ERR_TIMEOUT, msg);
        return h_info->status;
    }
    *h_info = mv_solve_info{};
    h_info->iterations = K;
    h_info->status = MV_OK;
    h_info->alpha = alpha;
    h_info->lambda_hat = hs.lambda_hat;
    h_info->kkt = hs.kkt;
    h_info->launches = launches;
    return MV_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batch of independent problems of uneven size in one launch per kernel:
// the GEMV pair runs as one grouped launch over a tile list spanning every
// problem, the projection step as one launch of one cluster per problem.
namespace mv {

struct GOne {
    SolveState *st;
    const double *mu, *r0, *x_in;
    const float *row_scale;
    float *y32;
    const float *g32, *z;
    double *x, *y;
    int n, T, mode;
    double gamma, safety, alpha_override, R;
};

__global__ void __launch_bounds__(kStepThreads) setup_grouped(const GOne *__restrict__ A) {
    const GOne a = A[blockIdx.x];
    setup_body(a.st, a.mu, a.r0, a.row_scale, a.y32, a.n);
}
__global__ void __launch_bounds__(kStepThreads) power_norm_grouped(const GOne *__restrict__ A) {
    const GOne a = A[blockIdx.x];
    power_norm_body(a.g32, a.row_scale, a.y32, a.n);
}
__global__ void __launch_bounds__(kStepThreads) step_size_grouped(const GOne *__restrict__ A) {
    const GOne a = A[blockIdx.x];
    step_size_body(a.st, a.z, a.alpha_override > 0.0 ? 0 : a.T, a.gamma, a.safety, a.alpha_override);
}
__global__ void __launch_bounds__(kStepThreads) objective_grouped(const GOne *__restrict__ A) {
    const GOne a = A[blockIdx.x];
    objective_body(a.st, a.z, a.T, a.x, a.n, a.gamma);
}
__global__ void __launch_bounds__(kStepThreads) to_y32_grouped(const GOne *__restrict__ A) {
    const GOne a = A[blockIdx.x];
    for (int i = threadIdx.x; i < a.n; i += kStepThreads)
        a.y32[i] = (float)(a.x[i] * (a.row_scale ? (double)a.row_scale[i] : 1.0));
}
template <int CL>
__global__ void __launch_bounds__(kProjNT) init_x_grouped(const GOne *__restrict__ A) {
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ ProjSmem psm;
    const GOne a = A[blockIdx.x / CL];
    init_x_body<CL>(a.st, a.mu, a.x_in, a.x, a.y, a.y32, a.row_scale, a.n, a.R, a.mode, dsm, psm);
}

template <typename Kern, typename Arg>
static cudaError_t launch_clusters(Kern kern, int CL, int count, size_t smem, cudaStream_t s, Arg arg) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(count * CL));
    cfg.blockDim = dim3(kProjNT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, arg);
}

static int batch_attrs() {
    static std::once_flag once;
    static int st = MV_OK;
    std::call_once(once, [] {
        bool ok = cluster_attrs(npga_step_grouped<1>, 1) && cluster_attrs(npga_step_grouped<2>, 2) &&
                  cluster_attrs(npga_step_grouped<4>, 4) && cluster_attrs(npga_step_grouped<8>, 8) &&
                  cluster_attrs(npga_step_grouped<16>, 16) && cluster_attrs(init_x_grouped<1>, 1) &&
                  cluster_attrs(init_x_grouped<2>, 2) && cluster_attrs(init_x_grouped<4>, 4) &&
                  cluster_attrs(init_x_grouped<8>, 8) && cluster_attrs(init_x_grouped<16>, 16);
        const int big = 96 * 1024;
        ok = ok &&
             cudaFuncSetAttribute(gemv_n_grouped<MV_F32, kRW>, cudaFuncAttributeMaxDynamicSharedMemorySize, big) ==
                 cudaSuccess &&
             cudaFuncSetAttribute(gemv_n_grouped<MV_BF16, kRW>, cudaFuncAttributeMaxDynamicSharedMemorySize, big) ==
                 cudaSuccess &&
             cudaFuncSetAttribute(gemv_n_grouped<MV_FP8_E4M3, kRW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  big) == cudaSuccess;
        if (!ok) st = record_cuda_error(cudaGetLastError(), "batch kernel attributes", __FILE__, __LINE__);
    });
    return st;
}

// Tiles of the grouped GEMVs: rows per split of gemv_t, bytes of L per row
// per split of gemv_n.  The solve times every candidate on the batch itself
// the first time it sees a batch shape and keeps the fastest (the choice is
// cached per shape signature; MV_BATCH_AUTOTUNE=0 keeps the default).
struct BatchTiles {
    int t_rows, n_bytes;
};
constexpr BatchTiles kBatchDefault = {512, 16384};
constexpr BatchTiles kBatchCandidates[] = {{256, 8192}, {256, 16384}, {256, 32768}, {512, 8192}, {512, 16384},
                                           {512, 32768}, {1024, 8192}, {1024, 16384}, {1024, 32768}};

struct BatchLayout {
    std::vector<Plan> plans;
    std::vector<size_t> base;       // workspace offset of each problem's plan
    size_t o_gp, o_gp_all, o_sa, o_one, o_tt, o_tn, o_zero;
    int nt_tiles, nn_tiles, cl, max_ncols, max_n;
    size_t total;
};

static int batch_layout(const mv_problem *probs, int64_t count, BatchLayout *Lo, BatchTiles tiles = kBatchDefault) {
    Lo->plans.clear();
    Lo->base.clear();
    int64_t ntt = 0, nnt = 0;
    int max_n = 1, max_ncols = 0;
    for (int64_t i = 0; i < count; ++i) {
        MV_TRY(validate_problem(probs + i));
        MV_TRY(require_nt(probs + i, "batch solve"));
        if (probs[i].dtype != probs[0].dtype) return record_message(MV_ERR_INVALID_ARG, "batch: mixed dtypes");
        Plan p = make_plan(probs[i].dtype, probs[i].n, probs[i].T, probs[i].ld, tiles.t_rows, false, false,
                           tiles.n_bytes);
        ntt += (int64_t)p.t_blocks * p.t_splits;
        nnt += (int64_t)p.n_groups * p.n_splits;
        max_n = std::max(max_n, p.n);
        max_ncols = std::max(max_ncols, p.n_cols);
        Lo->plans.push_back(p);
    }
    if (ntt >= (1LL << 31) || nnt >= (1LL << 31))
        return record_message(MV_ERR_UNSUPPORTED, "batch: the tile list exceeds 2^31 entries");
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    Lo->o_gp = take(sizeof(GemvProb) * (size_t)count);
    Lo->o_gp_all = take(sizeof(GemvProb) * (size_t)count);
    Lo->o_sa = take(sizeof(StepArgs) * (size_t)count);
    Lo->o_one = take(sizeof(GOne) * (size_t)count);
    Lo->o_tt = take(sizeof(int4) * (size_t)ntt);
    Lo->o_tn = take(sizeof(int4) * (size_t)nnt);
    Lo->o_zero = take(sizeof(int));
    for (int64_t i = 0; i < count; ++i) Lo->base.push_back(take(Lo->plans[i].total));
    Lo->nt_tiles = (int)ntt;
    Lo->nn_tiles = (int)nnt;
    Lo->cl = proj_cluster_size(max_n);
    Lo->max_ncols = max_ncols;
    Lo->max_n = max_n;
    Lo->total = off;
    return MV_OK;
}

template <int DT>
static void batch_gemv(const BatchLayout &Lo, void *ws, bool all, bool with_n, cudaStream_t s) {
    const GemvProb *gp = at<GemvProb>(ws, all ? Lo.o_gp_all : Lo.o_gp);
    gemv_t_grouped<DT><<<Lo.nt_tiles, kGemvThreads, 0, s>>>(gp, at<int4>(ws, Lo.o_tt));
    if (with_n)
        gemv_n_grouped<DT, kRW><<<Lo.nn_tiles, kGemvThreads, (size_t)Lo.max_ncols * 4, s>>>(gp, at<int4>(ws, Lo.o_tn));
}

static void batch_gemv_any(int dt, const BatchLayout &Lo, void *ws, bool all, bool with_n, cudaStream_t s) {
    if (dt == MV_F32) batch_gemv<MV_F32>(Lo, ws, all, with_n, s);
    else if (dt == MV_BF16) batch_gemv<MV_BF16>(Lo, ws, all, with_n, s);
    else batch_gemv<MV_FP8_E4M3>(Lo, ws, all, with_n, s);
}

static cudaError_t batch_step(const BatchLayout &Lo, void *ws, int count, cudaStream_t s) {
    const size_t smem = proj_elem_bytes((Lo.max_n + Lo.cl - 1) / Lo.cl);
    const StepArgs *sa = at<StepArgs>(ws, Lo.o_sa);
    switch (Lo.cl) {
        case 1: return launch_clusters(npga_step_grouped<1>, 1, count, smem, s, sa);
        case 2: return launch_clusters(npga_step_grouped<2>, 2, count, smem, s, sa);
        case 4: return launch_clusters(npga_step_grouped<4>, 4, count, smem, s, sa);
        case 8: return launch_clusters(npga_step_grouped<8>, 8, count, smem, s, sa);
        default: return launch_clusters(npga_step_grouped<16>, 16, count, smem, s, sa);
    }
}

// Writes every problem's GEMV, step and set-up descriptors and the tile
// lists of layout Lo into the workspace (blocking: the host copies are freed).
static int batch_setup(const BatchLayout &Lo, const mv_problem *probs, int64_t count, const mv_solve_opts &O, void *ws,
                       cudaStream_t s) {
    const int cnt = (int)count;
    std::vector<GemvProb> gp(cnt), gpa(cnt);
    std::vector<StepArgs> sa(cnt);
    std::vector<GOne> one(cnt);
    std::vector<int4> tt, tn;
    tt.reserve(Lo.nt_tiles);
    tn.reserve(Lo.nn_tiles);
    const int *zero = at<int>(ws, Lo.o_zero);
    for (int i = 0; i < cnt; ++i) {
        const Plan &p = Lo.plans[i];
        char *w = reinterpret_cast<char *>(ws) + Lo.base[i];
        const mv_problem &P = probs[i];
        const float *rs = P.dtype == MV_FP8_E4M3 ? P.row_scale : nullptr;
        SolveState *st = at<SolveState>(w, p.o_state);
        GemvProb g;
        g.L = P.L;
        g.ld = P.ld;
        g.n = p.n;
        g.T = p.T;
        g.y32 = at<float>(w, p.o_y32);
        g.zpart = at<float>(w, p.o_zpart);
        g.zstride = p.zstride;
        g.z = at<float>(w, p.o_z);
        g.tick_t = at<unsigned>(w, p.o_tick_t);
        g.t_rows = p.t_rows;
        g.t_splits = p.t_splits;
        g.gpart = at<float>(w, p.o_gpart);
        g.gy = at<double>(w, p.o_gy);
        g.g32 = at<float>(w, p.o_g32);
        g.tick_n = at<unsigned>(w, p.o_tick_n);
        g.n_cols = p.n_cols;
        g.n_splits = p.n_splits;
        g.row_scale = rs;
        g.done = &st->done;
        gp[i] = g;
        g.done = zero;
        gpa[i] = g;
        StepArgs a;
        a.st = st;
        a.gy = at<double>(w, p.o_gy);
        a.x = at<double>(w, p.o_x);
        a.y = at<double>(w, p.o_y);
        a.gx = at<double>(w, p.o_gx);
        a.y32 = at<float>(w, p.o_y32);
        a.mu = P.mu;
        a.row_scale = rs;
        a.n = p.n;
        a.mode = P.mode;
        a.kkt_every = O.kkt_every;
        a.max_iter = O.max_iter;
        a.R = P.R_target;
        a.gamma = P.gamma;
        a.eps = O.eps;
        sa[i] = a;
        GOne o;
        o.st = st;
        o.mu = P.mu;
        o.r0 = P.power_start;
        o.x_in = nullptr;
        o.row_scale = rs;
        o.y32 = at<float>(w, p.o_y32);
        o.g32 = at<float>(w, p.o_g32);
        o.z = at<float>(w, p.o_z);
        o.x = at<double>(w, p.o_x);
        o.y = at<double>(w, p.o_y);
        o.n = p.n;
        o.T = p.T;
        o.mode = P.mode;
        o.gamma = P.gamma;
        o.safety = O.power_safety;
        o.alpha_override = O.alpha > 0.0 ? O.alpha : 0.0;
        o.R = P.R_target;
        one[i] = o;
        for (int b = 0; b < p.t_blocks; ++b)
            for (int sp = 0; sp < p.t_splits; ++sp) tt.push_back(make_int4(i, b, sp, 0));
        for (int gq = 0; gq < p.n_groups; ++gq)
            for (int sp = 0; sp < p.n_splits; ++sp) tn.push_back(make_int4(i, gq, sp, 0));
        MV_CUDA_TRY(cudaMemsetAsync(w + p.o_tick_t, 0, 4 * (size_t)p.t_blocks, s));
        MV_CUDA_TRY(cudaMemsetAsync(w + p.o_tick_n, 0, 4 * (size_t)p.n_groups, s));
    }
    MV_CUDA_TRY(cudaMemsetAsync(at<int>(ws, Lo.o_zero), 0, sizeof(int), s));
    MV_CUDA_TRY(cudaMemcpyAsync(at<GemvProb>(ws, Lo.o_gp), gp.data(), sizeof(GemvProb) * cnt, cudaMemcpyHostToDevice, s));
    MV_CUDA_TRY(cudaMemcpyAsync(at<GemvProb>(ws, Lo.o_gp_all), gpa.data(), sizeof(GemvProb) * cnt,
                                cudaMemcpyHostToDevice, s));
    MV_CUDA_TRY(cudaMemcpyAsync(at<StepArgs>(ws, Lo.o_sa), sa.data(), sizeof(StepArgs) * cnt, cudaMemcpyHostToDevice, s));
    MV_CUDA_TRY(cudaMemcpyAsync(at<GOne>(ws, Lo.o_one), one.data(), sizeof(GOne) * cnt, cudaMemcpyHostToDevice, s));
    MV_CUDA_TRY(cudaMemcpyAsync(at<int4>(ws, Lo.o_tt), tt.data(), sizeof(int4) * tt.size(), cudaMemcpyHostToDevice, s));
    MV_CUDA_TRY(cudaMemcpyAsync(at<int4>(ws, Lo.o_tn), tn.data(), sizeof(int4) * tn.size(), cudaMemcpyHostToDevice, s));
    MV_CUDA_TRY(cudaStreamSynchronize(s));   // host descriptor buffers may now be released
    return MV_OK;
}

// Times the grouped GEMV pair of every tile candidate on this batch (one
// warm pass, then two timed) and returns the fastest; cached per batch shape.
static uint64_t batch_key(const mv_problem *probs, int64_t count) {
    uint64_t key = 1469598103934665603ull;                // FNV-1a over the batch shape
    auto mix = [&](uint64_t v) { key = (key ^ v) * 1099511628211ull; };
    mix((uint64_t)probs[0].dtype);
    mix((uint64_t)count);
    for (int64_t i = 0; i < count; ++i) {
        mix((uint64_t)probs[i].n);
        mix((uint64_t)probs[i].T);
        mix((uint64_t)probs[i].ld);
    }
    return key;
}
static std::mutex g_tiles_mu;
static std::unordered_map<uint64_t, BatchTiles> g_tiles;

// The tiles a batch of this shape runs with: MV_OK and the tuned choice, or
// MV_ERR_NOT_CONVERGED and the defaults if it has not been tuned yet.
static int batch_tune_lookup(const mv_problem *probs, int64_t count, BatchTiles *out) {
    std::lock_guard<std::mutex> lock(g_tiles_mu);
    auto it = g_tiles.find(batch_key(probs, count));
    if (it == g_tiles.end()) {
        *out = kBatchDefault;
        return MV_ERR_NOT_CONVERGED;
    }
    *out = it->second;
    return MV_OK;
}

static int batch_tune(const mv_problem *probs, int64_t count, const mv_solve_opts &O, void *ws, size_t ws_bytes,
                      cudaStream_t s, BatchTiles *out) {
    *out = kBatchDefault;
    if (const char *env = getenv("MV_BATCH_AUTOTUNE"))
        if (atoi(env) == 0) return MV_OK;
    if (batch_tune_lookup(probs, count, out) == MV_OK) return MV_OK;
    const uint64_t key = batch_key(probs, count);
    cudaEvent_t e0, e1;
    MV_CUDA_TRY(cudaEventCreate(&e0));
    MV_CUDA_TRY(cudaEventCreate(&e1));
    float best = INFINITY;
    BatchTiles best_t = kBatchDefault;
    int st = MV_OK;
    for (const BatchTiles &c : kBatchCandidates) {
        BatchLayout Lo;
        st = batch_layout(probs, count, &Lo, c);
        if (st != MV_OK) break;
        if (Lo.total > ws_bytes) continue;
        st = batch_setup(Lo, probs, count, O, ws, s);
        if (st != MV_OK) break;
        setup_grouped<<<(int)count, kStepThreads, 0, s>>>(at<GOne>(ws, Lo.o_one));
        batch_gemv_any(probs[0].dtype, Lo, ws, true, true, s);
        cudaEventRecord(e0, s);
        for (int r = 0; r < 2; ++r) batch_gemv_any(probs[0].dtype, Lo, ws, true, true, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = record_cuda_error(cudaGetLastError(), "batch tile tuning", __FILE__, __LINE__);
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_t = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    MV_TRY(st);
    *out = best_t;
    std::lock_guard<std::mutex> lock(g_tiles_mu);
    g_tiles[key] = best_t;
    return MV_OK;
}

}  // namespace mv

extern "C" {

size_t mv_batch_workspace_size(const mv_problem *probs, int64_t count) {
    if (probs == nullptr || count < 1 || count > 65535) return 0;
    size_t total = 0;                              // room for every tile candidate of the tuning
    for (const BatchTiles &c : kBatchCandidates) {
        BatchLayout Lo;
        if (batch_layout(probs, count, &Lo, c) != MV_OK) return 0;
        total = std::max(total, Lo.total);
    }
    return total;
}

int mv_batch_tiles(const mv_problem *probs, int64_t count, int32_t *h_t_rows, int32_t *h_n_split_bytes) {
    if (probs == nullptr || h_t_rows == nullptr || h_n_split_bytes == nullptr || count < 1 || count > 65535)
        return MV_ERR_INVALID_ARG;
    BatchTiles t = kBatchDefault;
    const int st = batch_tune_lookup(probs, count, &t);
    *h_t_rows = t.t_rows;
    *h_n_split_bytes = t.n_bytes;
    return st;
}

int mv_npga_solve_batch(const mv_problem *probs, int64_t count, const mv_solve_opts *O_in, double *const *h_x_dev,
                        mv_solve_info *h_infos, void *d_ws, size_t ws_bytes, mv_stream_t stream) {
    if (probs == nullptr || h_x_dev == nullptr || h_infos == nullptr || count < 1 || count > 65535)
        return MV_ERR_INVALID_ARG;
    mv_solve_opts O;
    if (O_in) O = *O_in; else mv_solve_opts_default(&O);
    if (O.max_iter < 0 || O.kkt_every < 0 || O.power_iters < 0 || !(O.eps >= 0.0)) return MV_ERR_INVALID_ARG;
    if (O.power_iters == 0 && !(O.alpha > 0.0)) return MV_ERR_INVALID_ARG;
    if (O.momentum != 0 || O.backtrack != 0)
        return record_message(MV_ERR_UNSUPPORTED, "batch solve: fixed step and FISTA momentum only");
    BatchLayout Lo;
    MV_TRY(batch_layout(probs, count, &Lo));
    MV_TRY(check_ws(d_ws, ws_bytes, Lo.total));
    MV_TRY(set_kernel_attrs());
    MV_TRY(batch_attrs());
    (void)cudaGetLastError();
    cudaStream_t s = (cudaStream_t)stream;
    void *ws = d_ws;
    BatchTiles tiles;
    MV_TRY(batch_tune(probs, count, O, ws, ws_bytes, s, &tiles));
    MV_TRY(batch_layout(probs, count, &Lo, tiles));
    MV_TRY(check_ws(d_ws, ws_bytes, Lo.total));
    const int cnt = (int)count, dt = probs[0].dtype;
    MV_TRY(batch_setup(Lo, probs, count, O, ws, s));

    const GOne *d_one = at<GOne>(ws, Lo.o_one);
    int launches = 0;
    setup_grouped<<<cnt, kStepThreads, 0, s>>>(d_one);
    if (!(O.alpha > 0.0)) {
        for (int it = 0; it < O.power_iters; ++it) {
            batch_gemv_any(dt, Lo, ws, true, true, s);
            power_norm_grouped<<<cnt, kStepThreads, 0, s>>>(d_one);
            launches += 3;
        }
        if (O.power_iters > 0) {
            batch_gemv_any(dt, Lo, ws, true, false, s);
            ++launches;
        }
    }
    step_size_grouped<<<cnt, kStepThreads, 0, s>>>(d_one);
    {
        const size_t smem = proj_elem_bytes((Lo.max_n + Lo.cl - 1) / Lo.cl);
        cudaError_t e;
        switch (Lo.cl) {
            case 1: e = launch_clusters(init_x_grouped<1>, 1, cnt, smem, s, d_one); break;
            case 2: e = launch_clusters(init_x_grouped<2>, 2, cnt, smem, s, d_one); break;
            case 4: e = launch_clusters(init_x_grouped<4>, 4, cnt, smem, s, d_one); break;
            case 8: e = launch_clusters(init_x_grouped<8>, 8, cnt, smem, s, d_one); break;
            default: e = launch_clusters(init_x_grouped<16>, 16, cnt, smem, s, d_one); break;
        }
        MV_CUDA_TRY(e);
    }
    launches += 3;
    MV_CUDA_TRY(cudaGetLastError());

    const int chunk = O.kkt_every > 0 ? O.kkt_every : 8;
    cudaGraphExec_t exec = nullptr;
    if (O.use_graph) {
        cudaStream_t cs;
        MV_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            for (int c = 0; c < chunk; ++c) {
                batch_gemv_any(dt, Lo, ws, false, true, cs);
                batch_step(Lo, ws, cnt, cs);
            }
            if (cudaStreamEndCapture(cs, &graph) == cudaSuccess) {
                if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) exec = nullptr;
                cudaGraphDestroy(graph);
            }
        }
        cudaStreamDestroy(cs);
        (void)cudaGetLastError();
    }
    std::vector<SolveState> hs(cnt);
    const int64_t max_chunks = ((int64_t)O.max_iter + 1 + chunk - 1) / chunk + 1;
    for (int64_t c = 0; c < max_chunks; ++c) {
        if (exec) {
            MV_CUDA_TRY(cudaGraphLaunch(exec, s));
        } else {
            for (int i = 0; i < chunk; ++i) {
                batch_gemv_any(dt, Lo, ws, false, true, s);
                MV_CUDA_TRY(batch_step(Lo, ws, cnt, s));
            }
        }
        launches += 3 * chunk;
        for (int i = 0; i < cnt; ++i)
            MV_CUDA_TRY(cudaMemcpyAsync(&hs[i], reinterpret_cast<char *>(ws) + Lo.base[i] + Lo.plans[i].o_state,
                                        sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        MV_CUDA_TRY(cudaStreamSynchronize(s));
        bool all = true;
        for (int i = 0; i < cnt; ++i) all = all && hs[i].done;
        if (all) break;
    }
    if (exec) cudaGraphExecDestroy(exec);
    // objectives: z = L^T x for every problem, then ||z||^2 + gamma ||x||^2
    to_y32_grouped<<<cnt, kStepThreads, 0, s>>>(d_one);
    batch_gemv_any(dt, Lo, ws, true, false, s);
    objective_grouped<<<cnt, kStepThreads, 0, s>>>(d_one);
    launches += 3;
    MV_CUDA_TRY(cudaGetLastError());
    for (int i = 0; i < cnt; ++i) {
        MV_CUDA_TRY(cudaMemcpyAsync(h_x_dev[i], reinterpret_cast<char *>(ws) + Lo.base[i] + Lo.plans[i].o_x,
                                    8 * (size_t)Lo.plans[i].n, cudaMemcpyDeviceToDevice, s));
        MV_CUDA_TRY(cudaMemcpyAsync(&hs[i], reinterpret_cast<char *>(ws) + Lo.base[i] + Lo.plans[i].o_state,
                                    sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    }
    MV_CUDA_TRY(cudaStreamSynchronize(s));
    int worst = MV_OK;
    for (int i = 0; i < cnt; ++i) {
        mv_solve_info &I = h_infos[i];
        I = mv_solve_info{};
        I.iterations = hs[i].k;
        I.status = hs[i].done ? hs[i].status : MV_ERR_NOT_CONVERGED;
        I.converged = hs[i].converged;
        I.proj_failures = hs[i].proj_fail;
        I.proj_steps = hs[i].proj_steps;
        I.kkt = hs[i].kkt;
        I.objective = hs[i].objective;
        I.alpha = hs[i].alpha;
        I.lambda_hat = hs[i].lambda_hat;
        I.nu = hs[i].nu;
        I.launches = launches;
        if (I.status != MV_OK && worst == MV_OK) worst = I.status;
    }
    return worst;
}

int mv_npga_solve_refined(const mv_problem *P_lo, const mv_problem *P_hi, const mv_solve_opts *O_in, double eps_lo,
                          double *d_x_inout, mv_solve_info *h_info, void *d_ws, size_t ws_bytes, mv_stream_t stream) {
    MV_TRY(validate_problem(P_lo));
    MV_TRY(validate_problem(P_hi));
    if (h_info == nullptr || d_x_inout == nullptr || !(eps_lo >= 0.0)) return MV_ERR_INVALID_ARG;
    if (P_hi->dtype != MV_F32 || P_lo->n != P_hi->n || P_lo->T != P_hi->T || P_lo->gamma != P_hi->gamma ||
        P_lo->mu != P_hi->mu || P_lo->R_target != P_hi->R_target || P_lo->mode != P_hi->mode)
        return MV_ERR_INVALID_ARG;
    mv_solve_opts O;
    if (O_in) O = *O_in; else mv_solve_opts_default(&O);
    mv_solve_opts O1 = O;
    O1.eps = eps_lo;
    mv_solve_info i1{};
    int st = mv_npga_solve(P_lo, &O1, d_x_inout, &i1, d_ws, ws_bytes, stream);
    if (st != MV_OK && st != MV_ERR_NOT_CONVERGED) {
        *h_info = i1;
        return st;
    }
    mv_solve_opts O2 = O;
    O2.warm_start = 1;
    O2.alpha = i1.alpha / (1.0 + 1e-2);
    mv_solve_info i2{};
    st = mv_npga_solve(P_hi, &O2, d_x_inout, &i2, d_ws, ws_bytes, stream);
    *h_info = i2;
    h_info->iterations = i1.iterations + i2.iterations;
    h_info->refine_iterations = i2.iterations;
    h_info->lambda_hat = i1.lambda_hat;
    h_info->proj_failures = i1.proj_failures + i2.proj_failures;
    h_info->proj_steps = i1.proj_steps + i2.proj_steps;
    h_info->launches = i1.launches + i2.launches;
    h_info->timed_pairs = i1.timed_pairs + i2.timed_pairs;
    h_info->t_gemv_t_ms = i1.t_gemv_t_ms + i2.t_gemv_t_ms;
    h_info->t_gemv_n_ms = i1.t_gemv_n_ms + i2.t_gemv_n_ms;
    h_info->t_step_ms = i1.t_step_ms + i2.t_step_ms;
    return st;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free gradient: mv_gradient with its scratch in a fixed device
// array rather than a caller workspace, for callers that may not allocate
// device memory (they only receive input and output buffers from a host
// framework that owns the memory pool, or cannot pay cudaMalloc's implicit
// synchronisation in a latency-bound loop).
namespace mv {

static __device__ __align__(256) unsigned char g_noalloc_scratch[MV_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[128];   // device address of the array, per device ordinal

// The host-side name of the array is only a stand-in, so its device address
// is looked up with the device current.  A call outside stream capture looks
// it up every time (cheap once the module is loaded), so the address stays
// right after a device reset, which reloads the module at a new address.
// Inside a capture no look-up is made and the device's last address is used.
static int noalloc_scratch(cudaStream_t s, void **out) {
    int dev = 0;
    MV_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) return record_message(MV_ERR_UNSUPPORTED, "mv_gradient_noalloc: device ordinal >= 128");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    MV_CUDA_TRY(cudaStreamIsCapturing(s, &cap));
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        MV_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_addr[dev] = p;
    } else if (g_noalloc_addr[dev] == nullptr) {
        return record_message(MV_ERR_UNSUPPORTED,
                              "mv_gradient_noalloc: the first call on a device must come before stream capture");
    }
    *out = g_noalloc_addr[dev];
    return MV_OK;
}

// The scratch this call needs: the plan of the two-pass GEMV path (its row
// splits follow the device's SM count, so the figure is per device).
static int noalloc_plan(const mv_problem *P, Plan *out) {
    MV_TRY(validate_problem(P));
    if (is_sigma(P)) return record_message(MV_ERR_UNSUPPORTED, "mv_gradient_noalloc: explicit Sigma is not supported");
    *out = make_plan(P->dtype, P->n, P->T, P->ld, 0, false, is_tn(P));
    return MV_OK;
}

}  // namespace mv

extern "C" size_t mv_gradient_noalloc_scratch_size(const mv_problem *P) {
    Plan p{};
    return noalloc_plan(P, &p) == MV_OK ? p.total : 0;
}

extern "C" int mv_gradient_noalloc(const mv_problem *P, const double *d_y, float *d_z, double *d_g,
                                   mv_stream_t stream) {
    Plan p{};
    MV_TRY(noalloc_plan(P, &p));
    if (d_y == nullptr || d_g == nullptr) return MV_ERR_INVALID_ARG;
    if (p.total > MV_NOALLOC_SCRATCH_BYTES) {
        char msg[200];
        snprintf(msg, sizeof(msg),
                 "mv_gradient_noalloc: this problem needs %zu bytes of scratch; the fixed array holds %zu",
                 p.total, (size_t)MV_NOALLOC_SCRATCH_BYTES);
        return record_message(MV_ERR_UNSUPPORTED, msg);
    }
    cudaStream_t s = (cudaStream_t)stream;
    void *ws = nullptr;
    MV_TRY(noalloc_scratch(s, &ws));
    MV_TRY(set_kernel_attrs());
    (void)cudaGetLastError();
    float *y32 = at<float>(ws, p.o_y32);
    double *lz = at<double>(ws, p.o_gy);
    // The array keeps the previous call's contents: the gemv tickets must start at zero.
    MV_CUDA_TRY(cudaMemsetAsync(at<char>(ws, p.o_tick_t), 0, 4 * (size_t)p.t_blocks, s));
    MV_CUDA_TRY(cudaMemsetAsync(at<char>(ws, p.o_tick_n), 0, 4 * (size_t)p.n_groups, s));
    const float *rs = P->dtype == MV_FP8_E4M3 ? P->row_scale : nullptr;
    to_y32_kernel<<<(p.n + 255) / 256, 256, 0, s>>>(d_y, rs, y32, p.n);
    gemv_pair(p, P, y32, ws, nullptr, lz, s);
    grad_finish_kernel<<<(p.n + 255) / 256, 256, 0, s>>>(lz, d_y, P->gamma, d_g, p.n);
    if (d_z) MV_CUDA_TRY(cudaMemcpyAsync(d_z, at<float>(ws, p.o_z), 4 * (size_t)p.T, cudaMemcpyDeviceToDevice, s));
    MV_CUDA_TRY(cudaGetLastError());
    return MV_OK;
}
