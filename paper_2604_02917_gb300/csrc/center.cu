// mv_center_factor: mu = R 1/T, L = (R - mu 1^T)/sqrt(T-1), tr(Sigma) = ||L||_F^2 (Sec. 2.1).
//
// One block per asset row.  Pass 1 sums the row in FP64 for mu_i; pass 2
// accumulates sum_t ((R_it - mu_i) c)^2 in FP64 (and max |.| for the FP8
// row scale); pass 3 writes L in the storage type, zero-filling columns
// T..ldL-1.  For the transposed layout (L^T, T x n) pass 3 is replaced by a
// tiled transpose that reads R again along periods.  Passes 2 and 3 re-read a row the block has just streamed, so
// they mostly hit L2.  Per-row sums of squares are added in a second,
// single-block kernel in fixed order, so tr(Sigma) is deterministic.
#include <stdio.h>
#include <string.h>

#include "mv_internal.cuh"

namespace mv {

static thread_local char g_last_error[512] = "";

int record_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
    const char *base = strrchr(file, '/');
    snprintf(g_last_error, sizeof(g_last_error), "%s (%s) at %s:%d: %s", cudaGetErrorName(e), cudaGetErrorString(e),
             base ? base + 1 : file, line, what);
    return MV_ERR_CUDA;
}

int record_message(int status, const char *msg) {
    snprintf(g_last_error, sizeof(g_last_error), "%s", msg);
    return status;
}

constexpr int kCenterThreads = 512;

template <int DT>
__device__ __forceinline__ void store_elem(void *L, int64_t idx, double val, float inv_scale) {
    if constexpr (DT == MV_F32) {
        reinterpret_cast<float *>(L)[idx] = (float)val;
    } else if constexpr (DT == MV_BF16) {
        reinterpret_cast<__nv_bfloat16 *>(L)[idx] = __double2bfloat16(val);
    } else {
        const float q = (float)val * inv_scale;
        reinterpret_cast<__nv_fp8_storage_t *>(L)[idx] = __nv_cvt_float_to_fp8(q, __NV_SATFINITE, __NV_E4M3);
    }
}

// One block per asset row.  Pass 1: mu_i = sum_t R_it / T in FP64, and the
// FP32 range of the row; the FP8 scale max_t |d_it| / 448 follows exactly
// from it, because d = ((double)x - mu) c is monotone in x.  Pass 2 (WRITE):
// d_it in FP64, stored in the storage type, and sum_t d_it^2 for the trace;
// the re-read of the row mostly hits L2.  With WRITE = false (transposed
// layout) pass 2 is done by transpose_center_kernel.
template <int DT, bool WRITE>
__global__ void __launch_bounds__(kCenterThreads)
center_kernel(const float *__restrict__ R, int64_t ldR, int T, void *__restrict__ L, int64_t ldL,
              float *__restrict__ row_scale, double *__restrict__ mu, double *__restrict__ rowsq) {
    __shared__ double red[(kCenterThreads / kWarp + 1) * 2];
    const int64_t i = blockIdx.x;
    const float *r = R + i * ldR;
    double s[1] = {0.0};
    float xmin = INFINITY, xmax = -INFINITY;
    for (int t = threadIdx.x; t < T; t += kCenterThreads) {
        const float x = r[t];
        s[0] += (double)x;
        if constexpr (DT == MV_FP8_E4M3) {
            xmin = fminf(xmin, x);
            xmax = fmaxf(xmax, x);
        }
    }
    block_sum<1, kCenterThreads>(s, red);
    const double mean = s[0] / (double)T;
    const double c = 1.0 / sqrt((double)(T - 1));
    float inv_scale = 1.f;
    if constexpr (DT == MV_FP8_E4M3) {
        double mn = (double)xmin, mx = (double)xmax;
        __syncthreads();
        block_minmax<kCenterThreads>(mn, mx, red);
        const double amax = fmax((mx - mean) * c, (mean - mn) * c);
        const float scale = amax > 0.0 ? (float)(amax / 448.0) : 1.f;
        inv_scale = 1.f / scale;
        if (threadIdx.x == 0) row_scale[i] = scale;
    }
    if constexpr (WRITE) {
        double q[1] = {0.0};
        for (int64_t t = threadIdx.x; t < ldL; t += kCenterThreads) {
            const double d = t < T ? ((double)r[t] - mean) * c : 0.0;
            q[0] = fma(d, d, q[0]);
            store_elem<DT>(L, i * ldL + t, d, inv_scale);
        }
        __syncthreads();
        block_sum<1, kCenterThreads>(q, red);
        if (threadIdx.x == 0) rowsq[i] = q[0];
    }
    if (threadIdx.x == 0) mu[i] = mean;
}

// L^T (T x ldM, row t = period t) from R (n x T).  A block owns 32 assets and
// one of kSlices period slices, walking it in 32 x 32 tiles through shared
// memory: read along periods, written along assets; columns n..ldM-1 are
// written as zeros.  Values as center_kernel's; each block leaves
// sum_t d_it^2 of its slice in sqpart[slice][i] (added in fixed order by
// trace_kernel).
constexpr int kTile = 32;
constexpr int kSlices = 8;
template <int DT>
__global__ void __launch_bounds__(kTile * 8)
transpose_center_kernel(const float *__restrict__ R, int64_t ldR, int64_t n, int T, void *__restrict__ M, int64_t ldM,
                        const float *__restrict__ row_scale, const double *__restrict__ mu,
                        double *__restrict__ sqpart) {
    __shared__ double tile[kTile][kTile + 1];
    const int64_t i0 = (int64_t)blockIdx.y * kTile;        // assets
    const int slice = blockIdx.x;
    const int per = ((T + kSlices - 1) / kSlices + kTile - 1) / kTile * kTile;
    const int tb = slice * per, te = min(T, tb + per);
    const double c = 1.0 / sqrt((double)(T - 1));
    const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
    double mloc[4];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int64_t i = i0 + ty + 8 * j;
        mloc[j] = i < n ? mu[i] : 0.0;
    }
    float inv = 1.f;
    if (DT == MV_FP8_E4M3 && i0 + tx < n) inv = 1.f / row_scale[i0 + tx];
    for (int t0 = tb; t0 < te; t0 += kTile) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = ty + 8 * j;
            const int64_t i = i0 + k, t = t0 + tx;
            const double d = (i < n && t < te) ? ((double)R[i * ldR + t] - mloc[j]) * c : 0.0;
            acc[j] = fma(d, d, acc[j]);
            tile[k][tx] = d;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = ty + 8 * j;
            const int64_t t = t0 + k, i = i0 + tx;
            if (t < te && i < ldM) store_elem<DT>(M, t * ldM + i, tile[tx][k], i < n ? inv : 1.f);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        double v = warp_sum(acc[j]);
        const int64_t i = i0 + ty + 8 * j;
        if (tx == 0 && i < n) sqpart[(int64_t)slice * n + i] = v;
    }
}

// trace(Sigma) = sum_i rowsq_i, each rowsq_i the sum of its `parts` slice
// partials (parts = 1 for the n x T layout), in a fixed order.
__global__ void __launch_bounds__(kCenterThreads)
trace_kernel(const double *__restrict__ rowsq, int64_t n, int parts, double *__restrict__ trace) {
    __shared__ double red[(kCenterThreads / kWarp + 1) * 1];
    double s[1] = {0.0};
    for (int64_t i = threadIdx.x; i < n; i += kCenterThreads) {
        double r = 0.0;
        for (int k = 0; k < parts; ++k) r += rowsq[(int64_t)k * n + i];
        s[0] += r;
    }
    block_sum<1, kCenterThreads>(s, red);
    if (threadIdx.x == 0) *trace = s[0];
}

}  // namespace mv

using namespace mv;

extern "C" {

size_t mv_center_workspace_size(int64_t n, int64_t T) {
    (void)T;
    return n > 0 ? align_up((size_t)n * 8 * kSlices, 256) : 0;
}

int mv_center_factor(const float *d_R, int64_t n, int64_t T, int64_t ldR, int out_dtype, int layout, void *d_L,
                     int64_t ldL, float *d_row_scale, double *d_mu, double *d_trace, void *d_ws, size_t ws_bytes,
                     mv_stream_t stream) {
    if (d_R == nullptr || d_L == nullptr || d_mu == nullptr || d_trace == nullptr) return MV_ERR_INVALID_ARG;
    if (layout != MV_LAYOUT_NT && layout != MV_LAYOUT_TN) return MV_ERR_INVALID_ARG;
    const bool tn = layout == MV_LAYOUT_TN;
    if (n < 1 || T < 2 || ldR < T || ldL < (tn ? n : T) || n > (1LL << 31) - 1 || T > (1LL << 31) - 1)
        return MV_ERR_INVALID_ARG;
    const int es = dtype_size(out_dtype);
    if (es == 0) return MV_ERR_INVALID_ARG;
    if (out_dtype == MV_FP8_E4M3 && d_row_scale == nullptr) return MV_ERR_INVALID_ARG;
    const size_t need = mv_center_workspace_size(n, T);
    if (d_ws == nullptr || ws_bytes < need || ((uintptr_t)d_ws) % 256 != 0) return MV_ERR_WORKSPACE;
    (void)cudaGetLastError();
    cudaStream_t s = (cudaStream_t)stream;
    double *rowsq = reinterpret_cast<double *>(d_ws);
    const dim3 tgrid((unsigned)kSlices, (unsigned)((ldL + kTile - 1) / kTile));
    if (tn && tgrid.y > 65535u) return MV_ERR_UNSUPPORTED;
    switch (out_dtype) {
        case MV_F32:
            if (tn) {
                center_kernel<MV_F32, false><<<(unsigned)n, kCenterThreads, 0, s>>>(d_R, ldR, (int)T, nullptr, 0,
                                                                                    nullptr, d_mu, rowsq);
                transpose_center_kernel<MV_F32><<<tgrid, kTile * 8, 0, s>>>(d_R, ldR, n, (int)T, d_L, ldL, nullptr,
                                                                            d_mu, rowsq);
            } else {
                center_kernel<MV_F32, true><<<(unsigned)n, kCenterThreads, 0, s>>>(d_R, ldR, (int)T, d_L, ldL, nullptr,
                                                                                   d_mu, rowsq);
            }
            break;
        case MV_BF16:
            if (tn) {
                center_kernel<MV_BF16, false><<<(unsigned)n, kCenterThreads, 0, s>>>(d_R, ldR, (int)T, nullptr, 0,
                                                                                     nullptr, d_mu, rowsq);
                transpose_center_kernel<MV_BF16><<<tgrid, kTile * 8, 0, s>>>(d_R, ldR, n, (int)T, d_L, ldL, nullptr,
                                                                            d_mu, rowsq);
            } else {
                center_kernel<MV_BF16, true><<<(unsigned)n, kCenterThreads, 0, s>>>(d_R, ldR, (int)T, d_L, ldL,
                                                                                    nullptr, d_mu, rowsq);
            }
            break;
        default:
            if (tn) {
                center_kernel<MV_FP8_E4M3, false><<<(unsigned)n, kCenterThreads, 0, s>>>(d_R, ldR, (int)T, nullptr, 0,
                                                                                         d_row_scale, d_mu, rowsq);
                transpose_center_kernel<MV_FP8_E4M3><<<tgrid, kTile * 8, 0, s>>>(d_R, ldR, n, (int)T, d_L, ldL,
                                                                                 d_row_scale, d_mu, rowsq);
            } else {
                center_kernel<MV_FP8_E4M3, true><<<(unsigned)n, kCenterThreads, 0, s>>>(d_R, ldR, (int)T, d_L, ldL,
                                                                                        d_row_scale, d_mu, rowsq);
            }
            break;
    }
    trace_kernel<<<1, kCenterThreads, 0, s>>>(rowsq, n, tn ? kSlices : 1, d_trace);
    MV_CUDA_TRY(cudaGetLastError());
    return MV_OK;
}

const char *mv_status_string(int status) {
    switch (status) {
        case MV_OK: return "MV_OK";
        case MV_ERR_INVALID_ARG: return "MV_ERR_INVALID_ARG: bad pointer, size, alignment or option";
        case MV_ERR_INFEASIBLE: return "MV_ERR_INFEASIBLE: the feasible set F is empty";
        case MV_ERR_NOT_CONVERGED: return "MV_ERR_NOT_CONVERGED: iteration budget reached";
        case MV_ERR_TIMEOUT: return "MV_ERR_TIMEOUT: a bounded device wait gave up";
        case MV_ERR_NUMERIC: return "MV_ERR_NUMERIC: NaN or Inf encountered";
        case MV_ERR_CUDA: return "MV_ERR_CUDA: a CUDA runtime call failed";
        case MV_ERR_UNSUPPORTED: return "MV_ERR_UNSUPPORTED: not implemented for these arguments";
        case MV_ERR_WORKSPACE: return "MV_ERR_WORKSPACE: workspace missing, too small or misaligned";
        default: return "unknown mv_status";
    }
}

const char *mv_version(void) { return "mv 0.1 sm_103a"; }

const char *mv_last_error(void) { return g_last_error; }

}  // extern "C"
