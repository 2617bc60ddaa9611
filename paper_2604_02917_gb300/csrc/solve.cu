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
#include <cfloat>

#include "solve_internal.cuh"

namespace mv {

int sm_count() {
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


// The fused pass pays a cluster exchange per 128-byte column block, so it is
// used where a block holds many rows and there are many blocks.
// gemv_t (column sums) and gemv_n (row dots) run over the stored matrix:
// L (n x T) for MV_LAYOUT_NT, where z = L^T y is gemv_t and g = L z is
// gemv_n; L^T (T x n) for MV_LAYOUT_TN, where the two swap roles.
Plan make_plan(int dt, int64_t n, int64_t T, int64_t ld, int grouped_rows, bool fused, bool tn, int n_bytes) {
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
    p.o_lan = take(8 * kLanczosDoubles);
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
    p.o_lan = take(8 * kLanczosDoubles);
    p.o_err = take(16);
    p.total = off;
    return p;
}


// ------------------------------------------------------------------ kernels
// This block's slice of the Dykstra scratch (4 arrays of nl doubles).
__device__ __forceinline__ double *dyk_slice(double *base, int rank, int nl) {
    return base ? base + (size_t)rank * 4 * nl : nullptr;
}

// With q0 != nullptr the FP64 start vector of the Lanczos recurrence is also
// written there and its record `lan` cleared.
__device__ __forceinline__ void setup_body(SolveState *st, const double *__restrict__ mu, const double *__restrict__ r0,
             const float *__restrict__ row_scale, float *__restrict__ y32, int n,
             float *__restrict__ q0 = nullptr, double *__restrict__ lan = nullptr) {
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
        if (q0) q0[i] = (float)(r * inv);
    }
    if (lan && threadIdx.x < 2) lan[threadIdx.x] = 0.0;
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
             const float *__restrict__ row_scale, float *__restrict__ y32, int n, float *__restrict__ q0 = nullptr,
             double *__restrict__ lan = nullptr) {
    setup_body(st, mu, r0, row_scale, y32, n, q0, lan);
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
    umma::launch_dependents();     // the next fused pass may start streaming L
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

// One step of the Lanczos recurrence on A = L L^T, for the largest singular
// value of L_eff that the fixed step of Sec. 3.1 may use.  w = A q_j arrives
// as the FP32 copy of the product of y32 = q_j:
//   alpha_j = q_j^T w,  r = w - alpha_j q_j - beta_j q_{j-1},
//   beta_{j+1} = ||r||,  q_{j+1} = r / beta_{j+1},
// q_{j+1} overwriting q_{j-1} and going out as the next product input.
// Vectors and per-thread sums in FP32 (FP64 is scarce on this part and the
// products carry FP32 rounding anyway), alpha and beta combined and kept in
// FP64.  The recurrence stops (and later steps return at once) when
// beta_{j+1} is negligible against alpha_j + beta_j: K_{j+1} is then
// invariant under A and the Ritz values are eigenvalues.  No
// reorthogonalisation: a lost orthogonality only repeats converged Ritz
// values.  One block of kLanczosThreads; the loops are unrolled so that
// each thread keeps several loads in flight (the vectors sit in L2).
constexpr int kLanczosThreads = 1024;

__global__ void __launch_bounds__(kLanczosThreads)
lanczos_kernel(const float *__restrict__ w, const float *__restrict__ qj, float *__restrict__ qprev,
               double *__restrict__ lan, const float *__restrict__ row_scale, float *__restrict__ y32, int n, int j) {
    umma::launch_dependents();     // the next fused pass may start streaming L
    __shared__ double red[kLanczosThreads / kWarp + 1];
    if (lan[1] != 0.0) return;     // the same value in every thread: written below, after the barriers
    const double b = j > 0 ? lan[2 + kMaxLanczos + j - 1] : 0.0;
    const float bf = (float)b;
    float pa = 0.f;
#pragma unroll 4
    for (int i = threadIdx.x; i < n; i += kLanczosThreads) pa = fmaf(qj[i], w[i], pa);
    double v[1] = {(double)pa};
    block_sum<1, kLanczosThreads>(v, red);
    const double a = v[0];
    const float af = (float)a;
    float ps = 0.f;
#pragma unroll 4
    for (int i = threadIdx.x; i < n; i += kLanczosThreads) {
        float r = fmaf(-af, qj[i], w[i]);
        if (j > 0) r = fmaf(-bf, qprev[i], r);
        ps = fmaf(r, r, ps);
    }
    double ss[1] = {(double)ps};
    block_sum<1, kLanczosThreads>(ss, red);
    const double bn = sqrt(ss[0]);
    const bool stop = !(bn > 1e-12 * (fabs(a) + b));
    if (!stop) {
        const float inv = (float)(1.0 / bn);
#pragma unroll 4
        for (int i = threadIdx.x; i < n; i += kLanczosThreads) {
            float r = fmaf(-af, qj[i], w[i]);
            if (j > 0) r = fmaf(-bf, qprev[i], r);
            const float q = r * inv;
            qprev[i] = q;
            y32[i] = row_scale ? q * row_scale[i] : q;
        }
    }
    if (threadIdx.x == 0) {
        lan[2 + j] = a;
        lan[2 + kMaxLanczos + j] = bn;
        lan[0] = (double)(j + 1);
        if (stop) lan[1] = 1.0;
    }
}

// Number of eigenvalues below x of the symmetric tridiagonal matrix with
// diagonal a[0..k) and squared off-diagonal b2[i] (coupling i and i + 1):
// the negative pivots of the LDL^T factorisation of T - x I (Sturm count).
__device__ __forceinline__ int sturm_count(const float *a, const float *b2, int k, float x, float pivmin) {
    int c = 0;
    float d = 1.f;
    for (int i = 0; i < k; ++i) {
        d = (a[i] - x) - (i > 0 ? b2[i - 1] / d : 0.f);
        if (fabsf(d) < pivmin) d = -pivmin;
        c += d < 0.f;
    }
    return c;
}

// lambda_hat = the largest eigenvalue of the Lanczos tridiagonal matrix
// (diagonal alpha_0..alpha_{k-1}, off-diagonal beta_1..beta_{k-1}) by
// multisection on one warp: the matrix is scaled by its Gershgorin bound s
// (FP64) so that every entry lies in [-1, 1], and each round the bracket
// [lo, hi] is cut at 32 points, one FP32 Sturm count per lane, and narrowed
// to the piece where the count reaches k, down to FP32 resolution: the
// estimate carries a relative error of order k * 2^-24, far inside the
// step's safety factor.  FP32 because FP64 division is a long-latency
// sequence on this part: the same multisection in FP64 (12 rounds) measured
// 154 us per launch at k = 25.
constexpr int kLanczosEigRounds = 6;       // 33^6 > 2^30: past FP32 resolution

__global__ void __launch_bounds__(kWarp)
lanczos_step_size_kernel(SolveState *st, const double *__restrict__ lan, double gamma, double safety,
                         double alpha_override) {
    __shared__ float a[kMaxLanczos], b2[kMaxLanczos];
    const int lane = threadIdx.x;
    const int k = min(kMaxLanczos, (int)lan[0]);
    bool bad = false;
    double lo = INFINITY, hi = -INFINITY;
    for (int i = lane; i < k; i += kWarp) {
        const double ai = lan[2 + i];
        const double bl = i > 0 ? fabs(lan[2 + kMaxLanczos + i - 1]) : 0.0;
        const double br = i + 1 < k ? fabs(lan[2 + kMaxLanczos + i]) : 0.0;
        bad = bad || !isfinite(ai) || !isfinite(bl) || !isfinite(br);
        lo = fmin(lo, ai - bl - br);
        hi = fmax(hi, ai + bl + br);
    }
    bad = __any_sync(0xffffffffu, bad);
    lo = warp_min(lo);
    hi = warp_max(hi);
    const double sc = fmax(fabs(lo), fabs(hi));
    double lam = 0.0;
    if (bad || !isfinite(sc)) {
        lam = NAN;
    } else if (k == 1) {
        lam = lan[2];              // the 1 x 1 matrix: its entry, exactly
    } else if (k > 1 && sc > 0.0) {
        const double inv = 1.0 / sc;
        for (int i = lane; i < k; i += kWarp) {
            a[i] = (float)(lan[2 + i] * inv);
            const double bs = lan[2 + kMaxLanczos + i] * inv;
            b2[i] = (float)(bs * bs);
        }
        __syncwarp();
        float flo = (float)(lo * inv) - 0x1p-20f, fhi = (float)(hi * inv) + 0x1p-20f;
        for (int round = 0; round < kLanczosEigRounds && fhi - flo > 0.f; ++round) {
            const float h = (fhi - flo) / (float)(kWarp + 1);
            const float x = flo + h * (float)(lane + 1);
            // the lanes whose point has at most k - 1 eigenvalues below it form a prefix
            const unsigned below = __ballot_sync(0xffffffffu, sturm_count(a, b2, k, x, FLT_MIN) <= k - 1);
            const int t = below ? 31 - __clz((int)below) : -1;
            const float nlo = t >= 0 ? flo + h * (float)(t + 1) : flo;
            const float nhi = t + 1 < kWarp ? flo + h * (float)(t + 2) : fhi;
            flo = nlo;
            fhi = nhi;
        }
        lam = sc * (0.5 * ((double)flo + (double)fhi));
    }
    if (lane == 0) set_step(st, lam, gamma, safety, alpha_override);
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
    const double nu0 = st->nu, tau0 = st->tau;
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
        // warm start from this iteration's multipliers: x^k - alpha grad f(x^k)
        // lies next to the point x^k was projected from (y^k -> x^k as the
        // iterates settle), so its support usually matches and the search
        // stops after the verifying reduction
        // (measured the same as the previous test's multipliers: 37.6 against 37.8 us per step)
        const ProjOut o = P.solve(a.R, a.mode, mn, mx, nu0, tau0, a.budget);
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
    umma::launch_dependents();     // the next fused pass may start streaming L
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
    umma::launch_dependents();
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
int validate_problem(const mv_problem *P) {
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


// The plan of a single-problem call: explicit Sigma, or a factor in either layout.
static Plan plan_for(const mv_problem *P, bool fused) {
    if (is_sigma(P)) return make_plan_sigma(P->n, P->ld);
    return make_plan(P->dtype, P->n, P->T, P->ld, 0, fused, is_tn(P));
}

// The calls that read L only through the NT-layout kernels.
int require_nt(const mv_problem *P, const char *what) {
    if (P->layout == MV_LAYOUT_NT) return MV_OK;
    char msg[128];
    snprintf(msg, sizeof(msg), "%s: the factor must be stored n x T (MV_LAYOUT_NT)", what);
    return record_message(MV_ERR_UNSUPPORTED, msg);
}

int check_ws(void *ws, size_t ws_bytes, size_t need) {
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

// The solve loop and the power graph launch the fused pass as a
// programmatic dependent of the step / normalisation kernel before it.
constexpr bool kFusedPdl = true;

// g = L L^T y (row-scaled) in one pass over L; capturable (no synchronisation).
int launch_llt(const Plan &p, const mv_problem *P, const float *y32, void *ws, const int *done, double *g_out,
               float *g32, cudaStream_t s, float *z, bool pdl) {
    LltScratch sc = llt_scratch(at<char>(ws, p.o_llt), p.n);
    sc.err = at<int>(ws, p.o_err);             // read back by the solve
    return llt_launch(p.lp, p.dt, P->L, p.n, p.T, p.ld, y32, P->dtype == MV_FP8_E4M3 ? P->row_scale : nullptr, sc,
                      done, g_out, g32, s, z, pdl);
}

// Kernel attributes are set once per process, before any stream capture.
int set_kernel_attrs() {
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

void gemv_pair(const Plan &p, const mv_problem *P, const float *y32, void *ws, const int *done, double *g_out,
               cudaStream_t s, float *g32) {
    launch_z(p, P, y32, ws, done, s);
    launch_g(p, P, at<float>(ws, p.o_z), ws, done, g_out, g32, s);
}

void gemv_t_only(const Plan &p, const mv_problem *P, const float *y32, void *ws, cudaStream_t s) {
    launch_z(p, P, y32, ws, nullptr, s);
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

void launch_init_x(const Plan &p, const mv_problem *P, const mv_solve_opts *O, const double *x_in, void *ws,
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
int launch_iteration(const Plan &p, const mv_problem *P, const mv_solve_opts *O, void *ws,
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
            MV_TRY(launch_llt(p, P, y32, ws, done, gy, nullptr, s, p.want_z ? at<float>(ws, p.o_z) : nullptr,
                              kFusedPdl && ev == nullptr));   // timed runs keep launches apart
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

static std::mutex g_graph_mu;
static std::unordered_map<GraphKey, cudaGraphExec_t, GraphKeyHash> g_graphs;

int cached_graph(const GraphKey &key, const std::function<int(cudaStream_t)> &enqueue, cudaGraphExec_t *out) {
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

GraphKey graph_key(const Plan &p, const mv_problem *P, const mv_solve_opts *O, int chunk, const void *ev) {
    return GraphKey{P->L, P->mu, P->row_scale, nullptr, P->n, P->T, P->ld, P->dtype, P->mode, O->kkt_every,
                    O->max_iter, chunk, p.sig ? 2 : (p.use_llt ? (p.want_z ? 3 : 1) : 0), P->R_target, P->gamma, O->eps, ev,
                    O->momentum, O->backtrack, O->proj_budget, O->dykstra_iters, O->bt_rho, O->m_f};
}

int get_chunk_graph(const Plan &p, const mv_problem *P, const mv_solve_opts *O, void *ws, int chunk,
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
            // after the previous power normalisation (the first launch has no
            // kernel before it in the captured graph)
            MV_TRY(launch_llt(p, P, y32, ws, nullptr, at<double>(ws, p.o_gy), at<float>(ws, p.o_g32), s, nullptr,
                              kFusedPdl));
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

// The Lanczos alternative: `steps` products L L^T q_j, each followed by one
// step of the recurrence (FP32 q_j alternates between the x and y buffers,
// free until x^0 is set); capturable.  Adds the launches to *count.
static int launch_lanczos(const Plan &p, const mv_problem *P, int steps, void *ws, cudaStream_t s, int *count) {
    const float *rs = P->dtype == MV_FP8_E4M3 ? P->row_scale : nullptr;
    float *y32 = at<float>(ws, p.o_y32);
    double *wd = at<double>(ws, p.o_gy);
    float *w = at<float>(ws, p.o_g32);
    float *q[2] = {at<float>(ws, p.o_x), at<float>(ws, p.o_y)};
    for (int j = 0; j < steps; ++j) {
        if (p.sig) {
            MV_TRY(launch_symv(p, P, y32, ws, nullptr, wd, w, s));
            *count += 2;
        } else if (p.use_llt) {
            MV_TRY(launch_llt(p, P, y32, ws, nullptr, wd, w, s, nullptr, kFusedPdl));
            *count += 2;
        } else {
            gemv_pair(p, P, y32, ws, nullptr, wd, s, w);
            *count += 3;
        }
        lanczos_kernel<<<1, kLanczosThreads, 0, s>>>(w, q[j & 1], q[(j + 1) & 1], at<double>(ws, p.o_lan), rs, y32,
                                                  p.n, j);
    }
    return cudaGetLastError() == cudaSuccess ? MV_OK : MV_ERR_CUDA;
}

static int get_power_graph(const Plan &p, const mv_problem *P, const mv_solve_opts *O, void *ws,
                           cudaGraphExec_t *out) {
    const bool lz = O->lanczos == 1;
    GraphKey key = graph_key(p, P, O, (lz ? -(1 << 20) : -1) - O->power_iters, nullptr);
    key.ws = ws;
    int dummy = 0;
    return cached_graph(key, [&](cudaStream_t cs) {
        return lz ? launch_lanczos(p, P, O->power_iters, ws, cs, &dummy)
                  : launch_power(p, P, O->power_iters, ws, cs, &dummy);
    }, out);
}

void launch_setup(SolveState *st, const double *mu, const double *r0, const float *rs, float *y32, int n,
                  cudaStream_t s, float *q0, double *lan) {
    setup_kernel<<<1, kStepThreads, 0, s>>>(st, mu, r0, rs, y32, n, q0, lan);
}
void launch_lanczos_step(const float *w, const float *qj, float *qprev, double *lan, const float *rs, float *y32,
                         int n, int j, cudaStream_t s) {
    lanczos_kernel<<<1, kLanczosThreads, 0, s>>>(w, qj, qprev, lan, rs, y32, n, j);
}
void launch_lanczos_step_size(SolveState *st, const double *lan, double gamma, double safety, double alpha,
                              cudaStream_t s) {
    lanczos_step_size_kernel<<<1, kWarp, 0, s>>>(st, lan, gamma, safety, alpha);
}
void launch_power_norm(const float *g32, const float *rs, float *y32, int n, cudaStream_t s) {
    power_norm_kernel<<<1, kStepThreads, 0, s>>>(g32, rs, y32, n);
}
void launch_step_size(SolveState *st, const float *z, int T, double gamma, double safety, double alpha,
                      cudaStream_t s) {
    step_size_kernel<<<1, kStepThreads, 0, s>>>(st, z, T, gamma, safety, alpha);
}
void launch_to_y32(const double *x, const float *rs, float *y32, int n, cudaStream_t s) {
    to_y32_kernel<<<(n + 255) / 256, 256, 0, s>>>(x, rs, y32, n);
}
void launch_grad_finish(const double *lz, const double *y, double gamma, double *g, int n, cudaStream_t s) {
    grad_finish_kernel<<<(n + 255) / 256, 256, 0, s>>>(lz, y, gamma, g, n);
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
    o->lanczos = 0;
    o->reserved_opts = 0;
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
    if (O.lanczos != 0 && O.lanczos != 1) return MV_ERR_INVALID_ARG;
    const bool lanczos = O.lanczos == 1 && !(O.alpha > 0.0);
    if (lanczos && (O.power_iters < 1 || O.power_iters > kMaxLanczos))
        return record_message(MV_ERR_INVALID_ARG, "Lanczos step size: power_iters must be in 1..512");
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
    setup_kernel<<<1, kStepThreads, 0, s>>>(st, P->mu, P->power_start, rs, y32, p.n,
                                            lanczos ? at<float>(d_ws, p.o_x) : nullptr,
                                            lanczos ? at<double>(d_ws, p.o_lan) : nullptr);
    // Power method (or Lanczos) for ||L_eff||_2^2, skipped when the step is
    // given: one cached graph of all its launches, or host-issued when graphs
    // are off.
    int launches = 4;
    if (!(O.alpha > 0.0)) {
        if (O.use_graph && !O.timing) {
            cudaGraphExec_t pexec = nullptr;
            MV_TRY(get_power_graph(p, P, &O, d_ws, &pexec));
            MV_CUDA_TRY(cudaGraphLaunch(pexec, s));
            int cnt = 0;
            for (int it = 0; it < O.power_iters; ++it) cnt += (p.sig || p.use_llt) ? 2 : 3;
            launches += cnt + (lanczos ? 0 : 1);
        } else if (lanczos) {
            MV_TRY(launch_lanczos(p, P, O.power_iters, d_ws, s, &launches));
        } else {
            MV_TRY(launch_power(p, P, O.power_iters, d_ws, s, &launches));
        }
    }
    if (lanczos)
        lanczos_step_size_kernel<<<1, kWarp, 0, s>>>(st, at<double>(d_ws, p.o_lan), P->gamma, O.power_safety, O.alpha);
    else if (p.sig)
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

// Problems stored transposed (MV_LAYOUT_TN) take the fused single pass,
// grouped: one launch per cluster size over a list of (problem, cluster)
// pairs; problems stored n x T take the grouped GEMV pair.  Both can share
// a batch.
constexpr int kGroupSizes = 4;                       // cluster sizes 1, 2, 4, 8
struct BatchLayout {
    std::vector<Plan> plans;
    std::vector<size_t> base;       // workspace offset of each problem's plan
    std::vector<LltGroupPlan> gpl;  // grouped-pass geometry (TN problems)
    std::vector<size_t> o_lsc;      // grouped-pass scratch of each TN problem
    size_t o_gp, o_gp_all, o_sa, o_one, o_tt, o_tn, o_zero;
    size_t o_lgrp, o_lgrp_all, o_lcl, o_lerr;
    int nt_tiles, nn_tiles, cl, max_ncols, max_n;
    int n_tn, n_lcl;
    int lstart[kGroupSizes], lcount[kGroupSizes];
    size_t lsmem[kGroupSizes];
    size_t total;
    // a second stream (and fork/join events) on which one of two or more
    // grouped fused launches runs beside the others; null: one stream
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

static int group_index(int C) { return C == 1 ? 0 : C == 2 ? 1 : C == 4 ? 2 : 3; }

// Cluster size of the batch's step launch, which holds one cluster per
// problem: the smallest one whose blocks take at most kBatchStepElems
// elements, so that the launch stays near one wave (a lone problem prefers
// more, smaller blocks: proj_cluster_size).
constexpr int kBatchStepElems = 1536;
static int batch_cluster_size(int max_n) {
    int c = 1;
    while (c < kProjMaxCL && (max_n + c - 1) / c > kBatchStepElems) c *= 2;
    return c;
}

static int batch_layout(const mv_problem *probs, int64_t count, BatchLayout *Lo, BatchTiles tiles = kBatchDefault) {
    Lo->plans.clear();
    Lo->base.clear();
    Lo->gpl.assign((size_t)count, LltGroupPlan{});
    Lo->o_lsc.assign((size_t)count, 0);
    int64_t ntt = 0, nnt = 0, ncl = 0;
    int max_n = 1, max_ncols = 0, n_tn = 0;
    for (int g = 0; g < kGroupSizes; ++g) {
        Lo->lstart[g] = Lo->lcount[g] = 0;
        Lo->lsmem[g] = 0;
    }
    for (int64_t i = 0; i < count; ++i) {
        MV_TRY(validate_problem(probs + i));
        if (is_sigma(probs + i)) return record_message(MV_ERR_UNSUPPORTED, "batch solve: factor layouts only");
        if (probs[i].dtype != probs[0].dtype) return record_message(MV_ERR_INVALID_ARG, "batch: mixed dtypes");
        const bool tn = is_tn(probs + i);
        Plan p = make_plan(probs[i].dtype, probs[i].n, probs[i].T, probs[i].ld, tiles.t_rows, false, tn,
                           tiles.n_bytes);
        if (tn) {
            LltGroupPlan gp{};
            if (!llt_group_plan(probs[i].dtype, probs[i].n, probs[i].T, &gp))
                return record_message(MV_ERR_UNSUPPORTED, "batch: no cluster shape of the fused pass fits this n");
            Lo->gpl[(size_t)i] = gp;
            const int gi = group_index(gp.C);
            Lo->lcount[gi] += gp.G;
            Lo->lsmem[gi] = std::max(Lo->lsmem[gi], gp.smem);
            ncl += gp.G;
            ++n_tn;
        } else {
            ntt += (int64_t)p.t_blocks * p.t_splits;
            nnt += (int64_t)p.n_groups * p.n_splits;
            max_ncols = std::max(max_ncols, p.n_cols);
        }
        max_n = std::max(max_n, p.n);
        Lo->plans.push_back(p);
    }
    for (int g = 1; g < kGroupSizes; ++g) Lo->lstart[g] = Lo->lstart[g - 1] + Lo->lcount[g - 1];
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
    Lo->o_lgrp = take(llt_group_bytes() * (size_t)count);
    Lo->o_lgrp_all = take(llt_group_bytes() * (size_t)count);
    Lo->o_lcl = take(sizeof(int2) * (size_t)std::max<int64_t>(ncl, 1));
    Lo->o_lerr = take(16);
    for (int64_t i = 0; i < count; ++i) {
        Lo->base.push_back(take(Lo->plans[i].total));
        if (is_tn(probs + i)) Lo->o_lsc[(size_t)i] = take(llt_group_scratch_bytes(probs[i].n, Lo->gpl[(size_t)i].G));
    }
    Lo->nt_tiles = (int)ntt;
    Lo->nn_tiles = (int)nnt;
    Lo->n_tn = n_tn;
    Lo->n_lcl = (int)ncl;
    Lo->cl = batch_cluster_size(max_n);
    Lo->max_ncols = max_ncols;
    Lo->max_n = max_n;
    Lo->total = off;
    return MV_OK;
}

template <int DT>
static void batch_gemv(const BatchLayout &Lo, void *ws, bool all, bool with_n, cudaStream_t s) {
    const GemvProb *gp = at<GemvProb>(ws, all ? Lo.o_gp_all : Lo.o_gp);
    if (Lo.nt_tiles > 0) gemv_t_grouped<DT><<<Lo.nt_tiles, kGemvThreads, 0, s>>>(gp, at<int4>(ws, Lo.o_tt));
    if (with_n && Lo.nn_tiles > 0)
        gemv_n_grouped<DT, kRW><<<Lo.nn_tiles, kGemvThreads, (size_t)Lo.max_ncols * 4, s>>>(gp, at<int4>(ws, Lo.o_tn));
}

// One product for every problem: the grouped GEMV pair over the n x T
// problems (z only when !with_n) and, unless gemv_only, the grouped fused
// pass over the transposed ones (which always forms both z and g).  all:
// every problem, converged or not (the power method and the objectives);
// else converged problems return at once.
static int batch_gemv_any(int dt, const BatchLayout &Lo, void *ws, bool all, bool with_n, cudaStream_t s,
                          bool gemv_only = false) {
    if (dt == MV_F32) batch_gemv<MV_F32>(Lo, ws, all, with_n, s);
    else if (dt == MV_BF16) batch_gemv<MV_BF16>(Lo, ws, all, with_n, s);
    else batch_gemv<MV_FP8_E4M3>(Lo, ws, all, with_n, s);
    if (gemv_only || Lo.n_tn == 0) return MV_OK;
    const void *groups = at<char>(ws, all ? Lo.o_lgrp_all : Lo.o_lgrp);
    const int2 *cl = at<int2>(ws, Lo.o_lcl);
    int ng = 0;
    for (int g = 0; g < kGroupSizes; ++g) ng += Lo.lcount[g] > 0 ? 1 : 0;
    // With two or more cluster sizes the first launch runs on the side
    // stream beside the others, so their last waves overlap.
    const bool fork = ng >= 2 && Lo.side != nullptr;
    if (fork) {
        MV_CUDA_TRY(cudaEventRecord(Lo.fork, s));
        MV_CUDA_TRY(cudaStreamWaitEvent(Lo.side, Lo.fork, 0));
    }
    bool first = true;
    for (int g = 0; g < kGroupSizes; ++g)
        if (Lo.lcount[g] > 0) {
            // ordinary launches: early launch measured slower here (the
            // waiting clusters hold SMs the multi-wave step grid needs)
            const cudaStream_t gs = (fork && first) ? Lo.side : s;
            first = false;
            const cudaError_t e =
                llt_launch_grouped(dt, 1 << g, Lo.lcount[g], Lo.lsmem[g], groups, cl + Lo.lstart[g], gs, false);
            if (e != cudaSuccess) return record_cuda_error(e, "grouped fused pass launch", __FILE__, __LINE__);
        }
    if (fork) {
        MV_CUDA_TRY(cudaEventRecord(Lo.join, Lo.side));
        MV_CUDA_TRY(cudaStreamWaitEvent(s, Lo.join, 0));
    }
    return MV_OK;
}

// The side stream and events of a batch solve, released on every return.
struct BatchSide {
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    int create() {
        MV_CUDA_TRY(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
        MV_CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        MV_CUDA_TRY(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
        return MV_OK;
    }
    ~BatchSide() {
        if (join) cudaEventDestroy(join);
        if (fork) cudaEventDestroy(fork);
        if (side) cudaStreamDestroy(side);
    }
};

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
    const size_t gbytes = llt_group_bytes();
    std::vector<unsigned char> lg(Lo.n_tn > 0 ? gbytes * (size_t)cnt : 0), lga(lg.size());
    std::vector<int> tn_order[kGroupSizes];
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
        if (is_tn(&P)) {
            const LltGroupPlan &q = Lo.gpl[(size_t)i];
            char *sc = reinterpret_cast<char *>(ws) + Lo.o_lsc[(size_t)i];
            int *err = at<int>(ws, Lo.o_lerr);
            MV_TRY(llt_group_write(lg.data() + (size_t)i * gbytes, q, P.dtype, P.L, p.n, p.T, P.ld, g.y32, rs, sc, err,
                                   &st->done, g.gy, g.g32, nullptr));
            MV_TRY(llt_group_write(lga.data() + (size_t)i * gbytes, q, P.dtype, P.L, p.n, p.T, P.ld, g.y32, rs, sc, err,
                                   nullptr, g.gy, g.g32, g.z));
            MV_CUDA_TRY(cudaMemsetAsync(sc + llt_group_ticket_offset(p.n, q.G), 0, llt_ticket_bytes(), s));
            tn_order[group_index(q.C)].push_back(i);
            continue;
        }
        for (int b = 0; b < p.t_blocks; ++b)
            for (int sp = 0; sp < p.t_splits; ++sp) tt.push_back(make_int4(i, b, sp, 0));
        for (int gq = 0; gq < p.n_groups; ++gq)
            for (int sp = 0; sp < p.n_splits; ++sp) tn.push_back(make_int4(i, gq, sp, 0));
        MV_CUDA_TRY(cudaMemsetAsync(w + p.o_tick_t, 0, 4 * (size_t)p.t_blocks, s));
        MV_CUDA_TRY(cudaMemsetAsync(w + p.o_tick_n, 0, 4 * (size_t)p.n_groups, s));
    }
    // The grouped pass's cluster list: per cluster size, the problems whose
    // clusters take longest first (the short ones fill the last wave), each
    // problem's clusters adjacent (neighbouring row blocks of its L^T).
    std::vector<int2> lcl;
    lcl.reserve((size_t)Lo.n_lcl);
    for (int gi = 0; gi < kGroupSizes; ++gi) {
        std::vector<int> &ord = tn_order[gi];
        std::stable_sort(ord.begin(), ord.end(),
                         [&](int a, int b) { return Lo.gpl[(size_t)a].est_us > Lo.gpl[(size_t)b].est_us; });
        for (int i : ord)
            for (int c = 0; c < Lo.gpl[(size_t)i].G; ++c) lcl.push_back(make_int2(i, c));
    }
    if ((int)lcl.size() != Lo.n_lcl) return record_message(MV_ERR_UNSUPPORTED, "batch: cluster list size");
    if (Lo.n_tn > 0) {
        MV_CUDA_TRY(cudaMemcpyAsync(at<char>(ws, Lo.o_lgrp), lg.data(), lg.size(), cudaMemcpyHostToDevice, s));
        MV_CUDA_TRY(cudaMemcpyAsync(at<char>(ws, Lo.o_lgrp_all), lga.data(), lga.size(), cudaMemcpyHostToDevice, s));
        MV_CUDA_TRY(cudaMemcpyAsync(at<int2>(ws, Lo.o_lcl), lcl.data(), sizeof(int2) * lcl.size(),
                                    cudaMemcpyHostToDevice, s));
    }
    MV_CUDA_TRY(cudaMemsetAsync(at<char>(ws, Lo.o_lerr), 0, 16, s));
    MV_CUDA_TRY(cudaMemsetAsync(at<int>(ws, Lo.o_zero), 0, sizeof(int), s));
    MV_CUDA_TRY(cudaMemcpyAsync(at<GemvProb>(ws, Lo.o_gp), gp.data(), sizeof(GemvProb) * cnt, cudaMemcpyHostToDevice, s));
    MV_CUDA_TRY(cudaMemcpyAsync(at<GemvProb>(ws, Lo.o_gp_all), gpa.data(), sizeof(GemvProb) * cnt,
                                cudaMemcpyHostToDevice, s));
    MV_CUDA_TRY(cudaMemcpyAsync(at<StepArgs>(ws, Lo.o_sa), sa.data(), sizeof(StepArgs) * cnt, cudaMemcpyHostToDevice, s));
    MV_CUDA_TRY(cudaMemcpyAsync(at<GOne>(ws, Lo.o_one), one.data(), sizeof(GOne) * cnt, cudaMemcpyHostToDevice, s));
    if (!tt.empty())
        MV_CUDA_TRY(cudaMemcpyAsync(at<int4>(ws, Lo.o_tt), tt.data(), sizeof(int4) * tt.size(), cudaMemcpyHostToDevice, s));
    if (!tn.empty())
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
        mix((uint64_t)probs[i].layout);
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
        if (Lo.nt_tiles == 0) break;                     // every problem takes the fused pass: nothing to tune
        st = batch_setup(Lo, probs, count, O, ws, s);
        if (st != MV_OK) break;
        setup_grouped<<<(int)count, kStepThreads, 0, s>>>(at<GOne>(ws, Lo.o_one));
        batch_gemv_any(probs[0].dtype, Lo, ws, true, true, s, true);
        cudaEventRecord(e0, s);
        for (int r = 0; r < 2; ++r) batch_gemv_any(probs[0].dtype, Lo, ws, true, true, s, true);
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
    if (O.lanczos != 0) return record_message(MV_ERR_UNSUPPORTED, "batched solve: power-method step only");
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
    BatchSide side;
    if (Lo.n_tn > 0) {
        MV_TRY(side.create());
        Lo.side = side.side;
        Lo.fork = side.fork;
        Lo.join = side.join;
    }

    const GOne *d_one = at<GOne>(ws, Lo.o_one);
    int launches = 0;
    setup_grouped<<<cnt, kStepThreads, 0, s>>>(d_one);
    // kernels per product: the GEMV pair (or z alone) over the n x T
    // problems, one grouped fused launch per cluster size over the others
    int fused_launches = 0;
    for (int g = 0; g < kGroupSizes; ++g) fused_launches += Lo.lcount[g] > 0 ? 1 : 0;
    const int per_pair = (Lo.nt_tiles > 0 ? 1 : 0) + (Lo.nn_tiles > 0 ? 1 : 0) + fused_launches;
    const int per_z = (Lo.nt_tiles > 0 ? 1 : 0) + fused_launches;
    if (!(O.alpha > 0.0)) {
        for (int it = 0; it < O.power_iters; ++it) {
            MV_TRY(batch_gemv_any(dt, Lo, ws, true, true, s));
            power_norm_grouped<<<cnt, kStepThreads, 0, s>>>(d_one);
            launches += per_pair + 1;
        }
        if (O.power_iters > 0) {
            MV_TRY(batch_gemv_any(dt, Lo, ws, true, false, s));
            launches += per_z;
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
            int cst = MV_OK;
            for (int c = 0; c < chunk && cst == MV_OK; ++c) {
                cst = batch_gemv_any(dt, Lo, ws, false, true, cs);
                if (cst == MV_OK && batch_step(Lo, ws, cnt, cs) != cudaSuccess) cst = MV_ERR_CUDA;
            }
            if (cudaStreamEndCapture(cs, &graph) == cudaSuccess) {
                if (cst != MV_OK || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) exec = nullptr;
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
                MV_TRY(batch_gemv_any(dt, Lo, ws, false, true, s));
                MV_CUDA_TRY(batch_step(Lo, ws, cnt, s));
            }
        }
        launches += (per_pair + 1) * chunk;
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
    MV_TRY(batch_gemv_any(dt, Lo, ws, true, false, s));
    objective_grouped<<<cnt, kStepThreads, 0, s>>>(d_one);
    launches += per_z + 2;
    MV_CUDA_TRY(cudaGetLastError());
    int lerr = 0;
    MV_CUDA_TRY(cudaMemcpyAsync(&lerr, at<int>(ws, Lo.o_lerr), sizeof(int), cudaMemcpyDeviceToHost, s));
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
        if (lerr != 0 && Lo.gpl[(size_t)i].G > 0) I.status = MV_ERR_TIMEOUT;
        if (I.status != MV_OK && worst == MV_OK) worst = I.status;
    }
    if (lerr != 0) {
        char msg[96];
        snprintf(msg, sizeof(msg), "grouped single-pass product: a bounded wait timed out (code %d)", lerr);
        return record_message(MV_ERR_TIMEOUT, msg);
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

