// mv_project: batched exact projection onto F (Sec. 3.1), one block per problem.
#include "project.cuh"

namespace mv {

constexpr int kProjThreads = 512;
constexpr int kProjSmemMax = 12800;   // n up to this stages v and mu in shared memory

__global__ void __launch_bounds__(kProjThreads)
project_batch_kernel(const double *__restrict__ v, const double *__restrict__ mu, const double *__restrict__ Rt,
                     int n, int mode, double *__restrict__ x, mv_proj_info *__restrict__ info, int use_smem) {
    extern __shared__ double sm[];
    __shared__ double red[(kProjThreads / kWarp + 1) * 5];
    const int b = blockIdx.x;
    const double *vb = v + (int64_t)b * n;
    double *xb = x + (int64_t)b * n;
    const double *V = vb, *MU = mu;
    if (use_smem) {
        for (int i = threadIdx.x; i < n; i += kProjThreads) {
            sm[i] = vb[i];
            sm[n + i] = mu[i];
        }
        V = sm;
        MU = sm + n;
    }
    double mn = INFINITY, mx = -INFINITY;
    for (int i = threadIdx.x; i < n; i += kProjThreads) {
        const double m = mu[i];
        mn = fmin(mn, m);
        mx = fmax(mx, m);
    }
    block_minmax<kProjThreads>(mn, mx, red);
    __syncthreads();
    const double R = Rt[b];
    Projector<kProjThreads> P{V, MU, n, red, 0};
    const ProjOut o = P.solve(R, mode, mn, mx, 0.0, -INFINITY, 100);
    const bool bad = (o.status == MV_ERR_INFEASIBLE || o.status == MV_ERR_NUMERIC);
    double acc[2] = {0.0, 0.0};
    for (int i = threadIdx.x; i < n; i += kProjThreads) {
        const double xi = bad ? NAN : fmax(fma(o.nu, MU[i], V[i]) - o.tau, 0.0);
        xb[i] = xi;
        acc[0] = fma(MU[i], xi, acc[0]);
        acc[1] += (xi > 0.0) ? 1.0 : 0.0;
    }
    block_sum<2, kProjThreads>(acc, red);
    if (threadIdx.x == 0) {
        mv_proj_info r;
        r.nu = o.nu;
        r.tau = o.tau;
        r.residual = bad ? NAN : acc[0] - R;
        r.support = (int32_t)acc[1];
        r.status = o.status;
        r.steps = o.steps;
        r.active = (o.nu != 0.0) ? 1 : 0;
        info[b] = r;
    }
}

}  // namespace mv

using namespace mv;

extern "C" int mv_project(const double *d_v, const double *d_mu, const double *d_R_target, int64_t n, int64_t batch,
                          int mode, double *d_x, mv_proj_info *d_info, mv_stream_t stream) {
    if (d_v == nullptr || d_mu == nullptr || d_R_target == nullptr || d_x == nullptr || d_info == nullptr)
        return MV_ERR_INVALID_ARG;
    if (n < 1 || n > 65536 || batch < 1 || batch > (1LL << 31) - 1) return MV_ERR_INVALID_ARG;
    if (mode != MV_RETURN_GE && mode != MV_RETURN_EQ) return MV_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int use_smem = n <= kProjSmemMax ? 1 : 0;
    const size_t smem = use_smem ? (size_t)16 * n : 0;
    static bool attr_set = false;
    if (!attr_set) {
        MV_CUDA_TRY(cudaFuncSetAttribute(project_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         16 * kProjSmemMax));
        attr_set = true;
    }
    project_batch_kernel<<<(unsigned)batch, kProjThreads, smem, s>>>(d_v, d_mu, d_R_target, (int)n, mode, d_x, d_info,
                                                                    use_smem);
    MV_CUDA_TRY(cudaGetLastError());
    return MV_OK;
}
