// mv_project: batched exact projection onto F (Sec. 3.1); one thread-block
// cluster per problem (see project.cuh for the search and its arithmetic).
#include "project.cuh"

namespace mv {

template <int CL>
__global__ void __launch_bounds__(kProjNT)
project_batch_kernel(const double *__restrict__ v, const double *__restrict__ mu, const double *__restrict__ Rt,
                     int n, int mode, double *__restrict__ x, mv_proj_info *__restrict__ info) {
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ ProjSmem psm;
    const int b = blockIdx.x / CL;
    const int rank = cluster_rank<CL>();
    const int nl = (n + CL - 1) / CL;
    const int r0 = min(n, rank * nl);
    const int r1 = min(n, r0 + nl);
    ProjElems el = carve_elems(dsm, nl);
    el.n = r1 - r0;
    proj_smem_init(&psm);
    const double *vb = v + (int64_t)b * n;
    double mn = INFINITY, mx = -INFINITY;
    for (int i = threadIdx.x; i < el.n; i += kProjNT) {
        const double m = mu[r0 + i];
        el.v[i] = vb[r0 + i];
        el.mu[i] = m;
        mn = fmin(mn, m);
        mx = fmax(mx, m);
    }
    __syncthreads();
    ClusterProj<CL> P{&psm, el};
    P.reduce_minmax(mn, mx);
    P.prepare();
    const double R = Rt[b];
    const ProjOut o = P.solve(R, mode, mn, mx, 0.0, -INFINITY, 100);
    const bool bad = (o.status == MV_ERR_INFEASIBLE || o.status == MV_ERR_NUMERIC);
    double *xb = x + (int64_t)b * n;
    double acc = 0.0, cnt = 0.0;
    for (int i = threadIdx.x; i < el.n; i += kProjNT) {
        const double xi = bad ? NAN : fmax(fma(o.nu, el.mu[i], el.v[i]) - o.tau, 0.0);
        xb[r0 + i] = xi;
        acc = fma(el.mu[i], xi, acc);
        cnt += (xi > 0.0) ? 1.0 : 0.0;
    }
    const double phi = P.reduce_double(acc);
    const double sup = P.reduce_double(cnt);
    if (rank == 0 && threadIdx.x == 0) {
        mv_proj_info r;
        r.nu = o.nu;
        r.tau = o.tau;
        r.residual = bad ? NAN : phi - R;
        r.support = (int32_t)sup;
        r.status = o.status;
        r.steps = o.steps;
        r.active = (o.nu != 0.0) ? 1 : 0;
        info[b] = r;
    }
    cluster_barrier<CL>();   // no block leaves while a peer may still address its shared memory
}

template <int CL>
static int launch_project(const double *v, const double *mu, const double *Rt, int n, int64_t batch, int mode,
                          double *x, mv_proj_info *info, cudaStream_t s) {
    const int nl = (n + CL - 1) / CL;
    const size_t smem = proj_elem_bytes(nl);
    auto kern = project_batch_kernel<CL>;
    MV_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (CL > 8) MV_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(batch * CL));
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
    MV_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, v, mu, Rt, n, mode, x, info));
    return MV_OK;
}

}  // namespace mv

using namespace mv;

extern "C" int mv_project(const double *d_v, const double *d_mu, const double *d_R_target, int64_t n, int64_t batch,
                          int mode, double *d_x, mv_proj_info *d_info, mv_stream_t stream) {
    if (d_v == nullptr || d_mu == nullptr || d_R_target == nullptr || d_x == nullptr || d_info == nullptr)
        return MV_ERR_INVALID_ARG;
    if (n < 1 || n > kProjMaxN || batch < 1 || batch > 65535) return MV_ERR_INVALID_ARG;
    if (mode != MV_RETURN_GE && mode != MV_RETURN_EQ) return MV_ERR_INVALID_ARG;
    (void)cudaGetLastError();
    cudaStream_t s = (cudaStream_t)stream;
    switch (proj_cluster_size(n)) {
        case 1: return launch_project<1>(d_v, d_mu, d_R_target, (int)n, batch, mode, d_x, d_info, s);
        case 2: return launch_project<2>(d_v, d_mu, d_R_target, (int)n, batch, mode, d_x, d_info, s);
        case 4: return launch_project<4>(d_v, d_mu, d_R_target, (int)n, batch, mode, d_x, d_info, s);
        case 8: return launch_project<8>(d_v, d_mu, d_R_target, (int)n, batch, mode, d_x, d_info, s);
        default: return launch_project<16>(d_v, d_mu, d_R_target, (int)n, batch, mode, d_x, d_info, s);
    }
}
