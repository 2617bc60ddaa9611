// Adjoint of the unrolled NPGA solve (mv_npga_backward).
#include "solve_internal.cuh"

using namespace mv;

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
    if (O.lanczos != 0) return record_message(MV_ERR_UNSUPPORTED, "mv_npga_backward: power-method step only");
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
    launch_setup(st, P->mu, P->power_start, nullptr, y32, n, s);
    if (!(O.alpha > 0.0)) {
        for (int it = 0; it < O.power_iters; ++it) {
            if (p.use_llt)
                MV_TRY(launch_llt(p, P, y32, ws, nullptr, at<double>(ws, p.o_gy), at<float>(ws, p.o_g32), s));
            else
                gemv_pair(p, P, y32, ws, nullptr, at<double>(ws, p.o_gy), s, at<float>(ws, p.o_g32));
            launch_power_norm(at<float>(ws, p.o_g32), nullptr, y32, n, s);
        }
        if (p.use_llt)
            MV_TRY(launch_llt(p, P, y32, ws, nullptr, at<double>(ws, p.o_gy), nullptr, s, at<float>(ws, p.o_z)));
        else
            gemv_t_only(p, P, y32, ws, s);
    }
    launch_step_size(st, at<float>(ws, p.o_z), (O.alpha > 0.0) ? 0 : T, P->gamma, O.power_safety, O.alpha, s);
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

