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
              float *__restrict__ row_scale, double *__restrict__ mu, double *__restrict__ rowsq, int64_t i_base) {
    __shared__ double red[(kCenterThreads / kWarp + 1) * 2];
    const int64_t i = i_base + blockIdx.x;                 // asset; R holds rows i_base ..
    const float *r = R + (int64_t)blockIdx.x * ldR;
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
// trace_kernel).  The slice count is chosen per call to fill the GPU.
constexpr int kTile = 32;
constexpr int kMaxSlices = 64;                  // period slices per asset tile (grid fill), at most
template <int DT>
__global__ void __launch_bounds__(kTile * 8)
transpose_center_kernel(const float *__restrict__ R, int64_t ldR, int64_t n, int T, void *__restrict__ M, int64_t ldM,
                        const float *__restrict__ row_scale, const double *__restrict__ mu,
                        double *__restrict__ sqpart, int64_t i_base, int slices) {
    __shared__ double tile[kTile][kTile + 1];
    const int64_t i0 = i_base + (int64_t)blockIdx.y * kTile;   // assets; R holds rows i_base ..
    const int slice = blockIdx.x;
    const int per = ((T + slices - 1) / slices + kTile - 1) / kTile * kTile;
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
            const double d = (i < n && t < te) ? ((double)R[(i - i_base) * ldR + t] - mloc[j]) * c : 0.0;
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

// Centering of the asset rows [i0, i1) of R, whose row i0 is at R_rows.
// The last chunk of the transposed layout also zero-fills columns n..ldL-1.
// Period slices of the transposed write: about 8 blocks per SM over the
// asset tiles of a chunk of `rows` assets.
static int center_slices(int64_t rows, int64_t T) {
    const int64_t tiles = (rows + kTile - 1) / kTile;
    int64_t sl = (8 * 152 + tiles - 1) / tiles;
    const int64_t max_by_T = (T + kTile - 1) / kTile;
    sl = sl < 1 ? 1 : (sl > kMaxSlices ? kMaxSlices : sl);
    return (int)(sl < max_by_T ? sl : max_by_T);
}

static void center_chunk(const float *R_rows, int64_t ldR, int64_t n, int64_t T, int out_dtype, bool tn, void *d_L,
                         int64_t ldL, float *d_row_scale, double *d_mu, double *rowsq, int64_t i0, int64_t i1,
                         int slices, cudaStream_t s) {
    const unsigned rows = (unsigned)(i1 - i0);
    const int64_t wend = (tn && i1 == n) ? ldL : i1;          // transposed: columns written by this chunk
    const dim3 tgrid((unsigned)slices, (unsigned)((wend - i0 + kTile - 1) / kTile));
#define MV_CENTER_CASE(DT, RS)                                                                                   \
    if (tn) {                                                                                                    \
        center_kernel<DT, false><<<rows, kCenterThreads, 0, s>>>(R_rows, ldR, (int)T, nullptr, 0, RS, d_mu,      \
                                                                 rowsq, i0);                                     \
        transpose_center_kernel<DT><<<tgrid, kTile * 8, 0, s>>>(R_rows, ldR, n, (int)T, d_L, ldL, RS, d_mu,      \
                                                                rowsq, i0, slices);                              \
    } else {                                                                                                     \
        center_kernel<DT, true><<<rows, kCenterThreads, 0, s>>>(R_rows, ldR, (int)T, d_L, ldL, RS, d_mu, rowsq,  \
                                                                i0);                                             \
    }
    switch (out_dtype) {
        case MV_F32: MV_CENTER_CASE(MV_F32, nullptr) break;
        case MV_BF16: MV_CENTER_CASE(MV_BF16, nullptr) break;
        default: MV_CENTER_CASE(MV_FP8_E4M3, d_row_scale) break;
    }
#undef MV_CENTER_CASE
}

static int center_args(const void *R, int64_t n, int64_t T, int64_t ldR, int out_dtype, int layout, void *d_L,
                       int64_t ldL, float *d_row_scale, double *d_mu, double *d_trace) {
    if (R == nullptr || d_L == nullptr || d_mu == nullptr || d_trace == nullptr) return MV_ERR_INVALID_ARG;
    if (layout != MV_LAYOUT_NT && layout != MV_LAYOUT_TN) return MV_ERR_INVALID_ARG;
    const bool tn = layout == MV_LAYOUT_TN;
    if (n < 1 || T < 2 || ldR < T || ldL < (tn ? n : T) || n > (1LL << 31) - 1 || T > (1LL << 31) - 1)
        return MV_ERR_INVALID_ARG;
    if (dtype_size(out_dtype) == 0) return MV_ERR_INVALID_ARG;
    if (out_dtype == MV_FP8_E4M3 && d_row_scale == nullptr) return MV_ERR_INVALID_ARG;
    if (tn && (ldL + kTile - 1) / kTile > 65535)
        return record_message(MV_ERR_UNSUPPORTED, "mv_center_factor: the transposed output needs ldL <= 65535 * 32");
    return MV_OK;
}

// Chunked host-to-device pipeline of mv_center_factor_host.
constexpr int64_t kHostChunkBytes = 64ll << 20;

static int64_t host_chunk_rows(int64_t n, int64_t T) {
    int64_t m = kHostChunkBytes / (T * 4);
    m = m / kTile * kTile;
    if (m < kTile) m = kTile;
    return m < n ? m : n;
}

}  // namespace mv

using namespace mv;

extern "C" {

size_t mv_center_workspace_size(int64_t n, int64_t T) {
    (void)T;
    return n > 0 ? align_up((size_t)n * 8 * kMaxSlices, 256) : 0;
}

int mv_center_factor(const float *d_R, int64_t n, int64_t T, int64_t ldR, int out_dtype, int layout, void *d_L,
                     int64_t ldL, float *d_row_scale, double *d_mu, double *d_trace, void *d_ws, size_t ws_bytes,
                     mv_stream_t stream) {
    MV_TRY(center_args(d_R, n, T, ldR, out_dtype, layout, d_L, ldL, d_row_scale, d_mu, d_trace));
    const size_t need = mv_center_workspace_size(n, T);
    if (d_ws == nullptr || ws_bytes < need || ((uintptr_t)d_ws) % 256 != 0) return MV_ERR_WORKSPACE;
    (void)cudaGetLastError();
    cudaStream_t s = (cudaStream_t)stream;
    const bool tn = layout == MV_LAYOUT_TN;
    double *rowsq = reinterpret_cast<double *>(d_ws);
    const int slices = center_slices(n, T);
    center_chunk(d_R, ldR, n, T, out_dtype, tn, d_L, ldL, d_row_scale, d_mu, rowsq, 0, n, slices, s);
    trace_kernel<<<1, kCenterThreads, 0, s>>>(rowsq, n, tn ? slices : 1, d_trace);
    MV_CUDA_TRY(cudaGetLastError());
    return MV_OK;
}

size_t mv_center_host_workspace_size(int64_t n, int64_t T) {
    if (n < 1 || T < 2) return 0;
    const int64_t m = host_chunk_rows(n, T);
    return mv_center_workspace_size(n, T) + 2 * align_up((size_t)m * (size_t)T * 4, 256);
}

int mv_center_factor_host(const float *h_R, int64_t n, int64_t T, int64_t ldR, int out_dtype, int layout, void *d_L,
                          int64_t ldL, float *d_row_scale, double *d_mu, double *d_trace, void *d_ws, size_t ws_bytes,
                          mv_stream_t stream) {
    MV_TRY(center_args(h_R, n, T, ldR, out_dtype, layout, d_L, ldL, d_row_scale, d_mu, d_trace));
    const size_t need = mv_center_host_workspace_size(n, T);
    if (d_ws == nullptr || ws_bytes < need || ((uintptr_t)d_ws) % 256 != 0) return MV_ERR_WORKSPACE;
    (void)cudaGetLastError();
    cudaStream_t s = (cudaStream_t)stream;
    const bool tn = layout == MV_LAYOUT_TN;
    const int64_t m = host_chunk_rows(n, T);
    const int slices = center_slices(m, T);
    char *ws = reinterpret_cast<char *>(d_ws);
    double *rowsq = reinterpret_cast<double *>(ws);
    const size_t o_stage = mv_center_workspace_size(n, T), stage_bytes = align_up((size_t)m * (size_t)T * 4, 256);
    float *stage[2] = {reinterpret_cast<float *>(ws + o_stage), reinterpret_cast<float *>(ws + o_stage + stage_bytes)};
    // The copies run on a stream of their own, one chunk ahead of the kernels.
    cudaStream_t cs;
    MV_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaEvent_t copied[2], used[2], start;
    for (int b = 0; b < 2; ++b) {
        MV_CUDA_TRY(cudaEventCreateWithFlags(&copied[b], cudaEventDisableTiming));
        MV_CUDA_TRY(cudaEventCreateWithFlags(&used[b], cudaEventDisableTiming));
    }
    MV_CUDA_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    MV_CUDA_TRY(cudaEventRecord(start, s));
    MV_CUDA_TRY(cudaStreamWaitEvent(cs, start, 0));            // the copies follow earlier work on `stream`
    int st = MV_OK;
    int k = 0;
    for (int64_t i0 = 0; i0 < n && st == MV_OK; i0 += m, ++k) {
        const int64_t i1 = i0 + m < n ? i0 + m : n;
        const int b = k & 1;
        if (k >= 2 && cudaStreamWaitEvent(cs, used[b], 0) != cudaSuccess) st = MV_ERR_CUDA;
        if (st == MV_OK &&
            cudaMemcpy2DAsync(stage[b], (size_t)T * 4, h_R + i0 * ldR, (size_t)ldR * 4, (size_t)T * 4,
                              (size_t)(i1 - i0), cudaMemcpyHostToDevice, cs) != cudaSuccess)
            st = record_cuda_error(cudaGetLastError(), "cudaMemcpy2DAsync (host R chunk)", __FILE__, __LINE__);
        if (st == MV_OK && cudaEventRecord(copied[b], cs) != cudaSuccess) st = MV_ERR_CUDA;
        if (st == MV_OK && cudaStreamWaitEvent(s, copied[b], 0) != cudaSuccess) st = MV_ERR_CUDA;
        if (st == MV_OK) {
            center_chunk(stage[b], T, n, T, out_dtype, tn, d_L, ldL, d_row_scale, d_mu, rowsq, i0, i1, slices, s);
            if (cudaEventRecord(used[b], s) != cudaSuccess) st = MV_ERR_CUDA;
        }
    }
    if (st == MV_OK) trace_kernel<<<1, kCenterThreads, 0, s>>>(rowsq, n, tn ? slices : 1, d_trace);
    // `stream` waits for every copy before the events and the copy stream go away.
    cudaEvent_t fin;
    if (cudaEventCreateWithFlags(&fin, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(fin, cs);
        cudaStreamWaitEvent(s, fin, 0);
        cudaEventDestroy(fin);
    }
    for (int b = 0; b < 2; ++b) {
        cudaEventDestroy(copied[b]);
        cudaEventDestroy(used[b]);
    }
    cudaEventDestroy(start);
    cudaStreamDestroy(cs);
    MV_TRY(st);
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
