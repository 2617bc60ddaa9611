// Allocation-free gradient (mv_gradient_noalloc).
#include "solve_internal.cuh"

using namespace mv;

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
    launch_to_y32(d_y, rs, y32, p.n, s);
    gemv_pair(p, P, y32, ws, nullptr, lz, s);
    launch_grad_finish(lz, d_y, P->gamma, d_g, p.n, s);
    if (d_z) MV_CUDA_TRY(cudaMemcpyAsync(d_z, at<float>(ws, p.o_z), 4 * (size_t)p.T, cudaMemcpyDeviceToDevice, s));
    MV_CUDA_TRY(cudaGetLastError());
    return MV_OK;
}
