// Declarations shared by the solve's translation units: solve.cu (the
// single-problem loop, the batch, the refined solve), frontier.cu (many
// targets on one factor), adjoint.cu (the reverse sweep) and noalloc.cu
// (the allocation-free gradient).
#pragma once

#include <stdlib.h>

#include <functional>
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
constexpr int kMaxLanczos = 512;           // Lanczos steps of the step-size estimate
// Lanczos record (FP64): [0] steps taken, [1] 1 once stopped, alpha_j at
// [2 + j], beta_{j+1} at [2 + kMaxLanczos + j].
constexpr size_t kLanczosDoubles = 2 + 2 * (size_t)kMaxLanczos;

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
    size_t o_lan;                          // Lanczos record (kLanczosDoubles)
    int64_t zstride;                       // row pitch (floats) of the gemv_t partials
    size_t total;
};

static constexpr int kRW = 4;   // rows per warp in gemv_n

template <typename T_>
inline T_ *at(void *ws, size_t off) {
    return reinterpret_cast<T_ *>(reinterpret_cast<char *>(ws) + off);
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
// ---- defined in solve.cu
int sm_count();
// gemv_t (column sums) and gemv_n (row dots) run over the stored matrix:
// L (n x T) for MV_LAYOUT_NT, where z = L^T y is gemv_t and g = L z is
// gemv_n; L^T (T x n) for MV_LAYOUT_TN, where the two swap roles.
Plan make_plan(int dt, int64_t n, int64_t T, int64_t ld, int grouped_rows = 0, bool fused = false, bool tn = false,
               int n_bytes = 16384);
int validate_problem(const mv_problem *P);
inline bool is_tn(const mv_problem *P) { return P->layout == MV_LAYOUT_TN; }
inline bool is_sigma(const mv_problem *P) { return P->layout == MV_LAYOUT_SIGMA; }
int require_nt(const mv_problem *P, const char *what);
int check_ws(void *ws, size_t ws_bytes, size_t need);
int set_kernel_attrs();
// g = L L^T y (row-scaled) in one pass over L; capturable (no synchronisation).
// pdl: launched as a programmatic dependent of the previous kernel (which
// must not write L; see llt_launch).
int launch_llt(const Plan &p, const mv_problem *P, const float *y32, void *ws, const int *done, double *g_out,
               float *g32, cudaStream_t s, float *z = nullptr, bool pdl = false);
void gemv_pair(const Plan &p, const mv_problem *P, const float *y32, void *ws, const int *done, double *g_out,
               cudaStream_t s, float *g32 = nullptr);
void gemv_t_only(const Plan &p, const mv_problem *P, const float *y32, void *ws, cudaStream_t s);
void launch_init_x(const Plan &p, const mv_problem *P, const mv_solve_opts *O, const double *x_in, void *ws,
                   cudaStream_t s);
int launch_iteration(const Plan &p, const mv_problem *P, const mv_solve_opts *O, void *ws, cudaStream_t s,
                     const cudaEvent_t *ev);
GraphKey graph_key(const Plan &p, const mv_problem *P, const mv_solve_opts *O, int chunk, const void *ev);
// The cached executable graph of `key`, capturing `enqueue(stream)` into it on first use.
int cached_graph(const GraphKey &key, const std::function<int(cudaStream_t)> &enqueue, cudaGraphExec_t *out);
int get_chunk_graph(const Plan &p, const mv_problem *P, const mv_solve_opts *O, void *ws, int chunk,
                    const cudaEvent_t *ev, cudaGraphExec_t *out);
// Kernel launches of solve.cu's set-up, power-method, Lanczos and step-size
// kernels (q0 / lan: the Lanczos start vector and record, or nullptr).
void launch_setup(SolveState *st, const double *mu, const double *r0, const float *rs, float *y32, int n,
                  cudaStream_t s, float *q0 = nullptr, double *lan = nullptr);
void launch_lanczos_step(const float *w, const float *qj, float *qprev, double *lan, const float *rs, float *y32,
                         int n, int j, cudaStream_t s);
void launch_lanczos_step_size(SolveState *st, const double *lan, double gamma, double safety, double alpha,
                              cudaStream_t s);
void launch_power_norm(const float *g32, const float *rs, float *y32, int n, cudaStream_t s);
void launch_step_size(SolveState *st, const float *z, int T, double gamma, double safety, double alpha,
                      cudaStream_t s);
void launch_to_y32(const double *x, const float *rs, float *y32, int n, cudaStream_t s);
void launch_grad_finish(const double *lz, const double *y, double gamma, double *g, int n, cudaStream_t s);

// Kernel attributes of a cluster kernel (dynamic shared memory, size > 8).
template <typename Kern>
inline bool cluster_attrs(Kern k, int CL) {
    const int smem = (int)proj_elem_bytes(kProjMaxLocal);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return false;
    if (CL > 8 && cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        return false;
    return true;
}

template <typename Kern, typename... Args>
inline cudaError_t launch_cluster(Kern kern, int CL, size_t smem, cudaStream_t s, Args... args) {
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

}  // namespace mv
