// The two bandwidth-bound half-products of the NPGA gradient
// (Sec. 2.7, Eq. npga-unified-grad):  z = L^T y  and  g = L z.
//
// L is n x T, row-major (one asset per row), stored as FP32, BF16 or FP8
// e4m3 with one scale per row; every element is streamed from HBM once per
// half-product with 16-byte read-once loads, and accumulation is FP32.
//
// gemv_t (z = L^T y): a block owns a strip of 256*VEC consecutive columns
// and a split of rows.  Each thread keeps VEC column accumulators in
// registers and walks down its rows with 8 loads in flight; the row weights
// y_i of the split sit in shared memory.  Partial sums of every split are
// written to a [splits x T] buffer and the last block to finish a strip
// (atomic ticket after a fence -- no spinning) adds them in fixed split
// order, so the result is deterministic.
//
// gemv_n (g = L z): a block owns 8 warps x RW rows and a column split whose
// slice of z is staged in shared memory.  A warp reads RW rows at once,
// lanes covering consecutive 16-byte vectors (512 contiguous bytes per
// instruction), then reduces with shuffles.  The last block of a row group
// adds the column-split partials in fixed order, in FP64, and applies the
// FP8 row scale.
//
// FP8 row scales s_i are folded in: gemv_t consumes y'_i = s_i y_i (the
// producer of y writes it scaled) and gemv_n multiplies its row sum by s_i.
#pragma once

#include "mv_internal.cuh"

namespace mv {

constexpr int kGemvThreads = 256;
constexpr int kGemvUnroll = 8;
constexpr int kMaxRowsPerSplit = 2048;

// One block of z = L^T y: column strip `strip`, row split `split` of `nsplits`.
// The result, multiplied by cscale[col] if cscale is non-NULL, goes to z
// (FP32, may be NULL) and, when z64 is non-NULL, also to z64 in FP64: the
// transposed layout uses this kernel for g = L z with the FP8 asset scales.
template <int DT>
__device__ __forceinline__ void gemv_t_body(const void *__restrict__ L, int64_t ld, int n, int T,
                                            const float *__restrict__ y32, float *__restrict__ zpart, int64_t zstride,
                                            float *__restrict__ z, unsigned *__restrict__ tickets, int rows_per_split,
                                            int strip, int split, int nsplits, double *__restrict__ z64 = nullptr,
                                            const float *__restrict__ cscale = nullptr) {
    using S = Store<DT>;
    constexpr int VEC = S::VEC;
    constexpr int ES = (int)sizeof(typename S::elem);
    __shared__ float s_y[kMaxRowsPerSplit];
    __shared__ bool s_last;

    const int r0 = split * rows_per_split;
    const int rows = min(n - r0, rows_per_split);
    for (int i = threadIdx.x; i < rows; i += kGemvThreads) s_y[i] = y32[r0 + i];
    __syncthreads();

    const int64_t col = ((int64_t)strip * kGemvThreads + threadIdx.x) * VEC;
    float acc[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[e] = 0.f;

    if (col + VEC <= T) {
        const char *p = reinterpret_cast<const char *>(L) + ((int64_t)r0 * ld + col) * ES;
        const int64_t stride = ld * ES;
        int i = 0;
        for (; i + kGemvUnroll <= rows; i += kGemvUnroll) {
            uint4 u[kGemvUnroll];
#pragma unroll
            for (int j = 0; j < kGemvUnroll; ++j) u[j] = ld_stream16(p + (int64_t)(i + j) * stride);
#pragma unroll
            for (int j = 0; j < kGemvUnroll; ++j) {
                float f[VEC];
                S::unpack(u[j], f);
                const float yy = s_y[i + j];
#pragma unroll
                for (int e = 0; e < VEC; ++e) acc[e] = fmaf(f[e], yy, acc[e]);
            }
        }
        for (; i < rows; ++i) {
            float f[VEC];
            S::unpack(ld_stream16(p + (int64_t)i * stride), f);
            const float yy = s_y[i];
#pragma unroll
            for (int e = 0; e < VEC; ++e) acc[e] = fmaf(f[e], yy, acc[e]);
        }
    } else if (col < T) {                       // ragged tail of the last strip
        const int ne = (int)(T - col);
        for (int i = 0; i < rows; ++i) {
            const float yy = s_y[i];
            const int64_t base = (int64_t)(r0 + i) * ld + col;
#pragma unroll
            for (int e = 0; e < VEC; ++e)
                if (e < ne) acc[e] = fmaf(S::load1(L, base + e), yy, acc[e]);
        }
    }

    // Partial sums of this split; rows of zpart are 64-byte aligned (zstride).
    float *zp = zpart + (int64_t)split * zstride;
    const bool full = (col + VEC <= T);
    if (full) {
#pragma unroll
        for (int e = 0; e < VEC; e += 4)
            *reinterpret_cast<float4 *>(zp + col + e) = make_float4(acc[e], acc[e + 1], acc[e + 2], acc[e + 3]);
    } else if (col < T) {
#pragma unroll
        for (int e = 0; e < VEC; ++e)
            if (col + e < T) zp[col + e] = acc[e];
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned ticket = atomicAdd(&tickets[strip], 1u);
        s_last = (ticket == (unsigned)nsplits - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // Last block of the strip: add the splits in fixed order, 4 splits of
    // 16-byte loads in flight at a time.
    const int splits = nsplits;
    if (full) {
        float sacc[VEC];
#pragma unroll
        for (int e = 0; e < VEC; ++e) sacc[e] = 0.f;
        int sp = 0;
        for (; sp + 4 <= splits; sp += 4) {
            float4 q[4][VEC / 4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int e4 = 0; e4 < VEC / 4; ++e4)
                    q[u][e4] = __ldcg(reinterpret_cast<const float4 *>(zpart + (int64_t)(sp + u) * zstride + col) + e4);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int e4 = 0; e4 < VEC / 4; ++e4) {
                    sacc[4 * e4 + 0] += q[u][e4].x;
                    sacc[4 * e4 + 1] += q[u][e4].y;
                    sacc[4 * e4 + 2] += q[u][e4].z;
                    sacc[4 * e4 + 3] += q[u][e4].w;
                }
        }
        for (; sp < splits; ++sp) {
#pragma unroll
            for (int e4 = 0; e4 < VEC / 4; ++e4) {
                const float4 q = __ldcg(reinterpret_cast<const float4 *>(zpart + (int64_t)sp * zstride + col) + e4);
                sacc[4 * e4 + 0] += q.x;
                sacc[4 * e4 + 1] += q.y;
                sacc[4 * e4 + 2] += q.z;
                sacc[4 * e4 + 3] += q.w;
            }
        }
        if (z != nullptr) {
            float o[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) o[e] = cscale != nullptr ? sacc[e] * cscale[col + e] : sacc[e];
#pragma unroll
            for (int e = 0; e < VEC; e += 4)
                *reinterpret_cast<float4 *>(z + col + e) = make_float4(o[e], o[e + 1], o[e + 2], o[e + 3]);
        }
        if (z64 != nullptr) {
#pragma unroll
            for (int e = 0; e < VEC; ++e)
                z64[col + e] = (double)sacc[e] * (cscale != nullptr ? (double)cscale[col + e] : 1.0);
        }
    } else if (col < T) {
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            if (col + e < T) {
                float sm = 0.f;
                for (int sp = 0; sp < splits; ++sp) sm += __ldcg(zpart + (int64_t)sp * zstride + col + e);
                if (z != nullptr) z[col + e] = cscale != nullptr ? sm * cscale[col + e] : sm;
                if (z64 != nullptr) z64[col + e] = (double)sm * (cscale != nullptr ? (double)cscale[col + e] : 1.0);
            }
        }
    }
    if (threadIdx.x == 0) tickets[strip] = 0u;   // ready for the next launch
}

template <int DT>
__global__ void __launch_bounds__(kGemvThreads)
gemv_t_kernel(const void *__restrict__ L, int64_t ld, int n, int T, const float *__restrict__ y32,
              float *__restrict__ zpart, int64_t zstride, float *__restrict__ z, unsigned *__restrict__ tickets,
              int rows_per_split, const volatile int *done, double *__restrict__ z64 = nullptr,
              const float *__restrict__ cscale = nullptr) {
    if (done != nullptr && *done) return;
    gemv_t_body<DT>(L, ld, n, T, y32, zpart, zstride, z, tickets, rows_per_split, blockIdx.x, blockIdx.y, gridDim.y,
                    z64, cscale);
}

// One block of g = L z: row group `grp`, column split `split` of `nsplits`.
template <int DT, int RW>
__device__ __forceinline__ void gemv_n_body(const void *__restrict__ L, int64_t ld, int n, int T,
                                            const float *__restrict__ z, const float *__restrict__ row_scale,
                                            float *__restrict__ gpart, double *__restrict__ g, float *__restrict__ g32,
                                            unsigned *__restrict__ tickets, int cols_per_split, int grp, int split,
                                            int nsplits) {
    using S = Store<DT>;
    constexpr int VEC = S::VEC;
    constexpr int ES = (int)sizeof(typename S::elem);
    constexpr int ROWS = (kGemvThreads / kWarp) * RW;
    extern __shared__ float s_z[];
    __shared__ bool s_last;

    const int c0 = split * cols_per_split;
    const int ncol = min(T - c0, cols_per_split);
    for (int c = threadIdx.x; c < ncol; c += kGemvThreads) s_z[c] = z[c0 + c];
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rbase = grp * ROWS + warp * RW;
    float acc[RW];
    const char *rp[RW];
#pragma unroll
    for (int j = 0; j < RW; ++j) {
        acc[j] = 0.f;
        const int r = min(rbase + j, n - 1);      // clamp: rows past n are computed and dropped
        rp[j] = reinterpret_cast<const char *>(L) + ((int64_t)r * ld + c0) * ES;
    }
    const int nfull = ncol / VEC * VEC;
#pragma unroll 2
    for (int c = lane * VEC; c < nfull; c += kWarp * VEC) {
        float zz[VEC];
#pragma unroll
        for (int e = 0; e < VEC; e += 4) {
            const float4 q = *reinterpret_cast<const float4 *>(s_z + c + e);
            zz[e] = q.x;
            zz[e + 1] = q.y;
            zz[e + 2] = q.z;
            zz[e + 3] = q.w;
        }
        uint4 u[RW];
#pragma unroll
        for (int j = 0; j < RW; ++j) u[j] = ld_stream16(rp[j] + (int64_t)c * ES);
#pragma unroll
        for (int j = 0; j < RW; ++j) {
            float f[VEC];
            S::unpack(u[j], f);
#pragma unroll
            for (int e = 0; e < VEC; ++e) acc[j] = fmaf(f[e], zz[e], acc[j]);
        }
    }
    for (int c = nfull + lane; c < ncol; c += kWarp) {      // ragged tail
#pragma unroll
        for (int j = 0; j < RW; ++j) {
            const int r = min(rbase + j, n - 1);
            acc[j] = fmaf(S::load1(L, (int64_t)r * ld + c0 + c), s_z[c], acc[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < RW; ++j) acc[j] = warp_sumf(acc[j]);
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < RW; ++j)
            if (rbase + j < n) gpart[(int64_t)split * n + rbase + j] = acc[j];
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned ticket = atomicAdd(&tickets[grp], 1u);
        s_last = (ticket == (unsigned)nsplits - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int splits = nsplits;
    for (int r = grp * ROWS + threadIdx.x; r < min(n, (grp + 1) * ROWS); r += kGemvThreads) {
        double s = 0.0;
        for (int sp = 0; sp < splits; ++sp) s += (double)__ldcg(gpart + (int64_t)sp * n + r);
        if (row_scale != nullptr) s *= (double)row_scale[r];
        g[r] = s;
        if (g32 != nullptr) g32[r] = (float)s;
    }
    if (threadIdx.x == 0) tickets[grp] = 0u;
}

template <int DT, int RW>
__global__ void __launch_bounds__(kGemvThreads)
gemv_n_kernel(const void *__restrict__ L, int64_t ld, int n, int T, const float *__restrict__ z,
              const float *__restrict__ row_scale, float *__restrict__ gpart, double *__restrict__ g,
              float *__restrict__ g32, unsigned *__restrict__ tickets, int cols_per_split, const volatile int *done) {
    if (done != nullptr && *done) return;
    gemv_n_body<DT, RW>(L, ld, n, T, z, row_scale, gpart, g, g32, tickets, cols_per_split, blockIdx.x, blockIdx.y,
                        gridDim.y);
}

// ---------------------------------------------------------------- grouped form
// Many independent problems in one launch: block b runs tile tiles[b] =
// (problem, strip or row group, split) of the problem's own grid, skipping
// problems whose `done` flag is set.
struct GemvProb {
    const void *L;
    int64_t ld;
    int n, T;
    const float *y32;
    float *zpart;
    int64_t zstride;
    float *z;
    unsigned *tick_t;
    int t_rows, t_splits;
    float *gpart;
    double *gy;
    float *g32;
    unsigned *tick_n;
    int n_cols, n_splits;
    const float *row_scale;
    const int *done;
};

template <int DT>
__global__ void __launch_bounds__(kGemvThreads)
gemv_t_grouped(const GemvProb *__restrict__ probs, const int4 *__restrict__ tiles) {
    const int4 t = tiles[blockIdx.x];
    const GemvProb &p = probs[t.x];
    if (*(const volatile int *)p.done) return;
    gemv_t_body<DT>(p.L, p.ld, p.n, p.T, p.y32, p.zpart, p.zstride, p.z, p.tick_t, p.t_rows, t.y, t.z, p.t_splits);
}

template <int DT, int RW>
__global__ void __launch_bounds__(kGemvThreads)
gemv_n_grouped(const GemvProb *__restrict__ probs, const int4 *__restrict__ tiles) {
    const int4 t = tiles[blockIdx.x];
    const GemvProb &p = probs[t.x];
    if (*(const volatile int *)p.done) return;
    gemv_n_body<DT, RW>(p.L, p.ld, p.n, p.T, p.z, p.row_scale, p.gpart, p.gy, p.g32, p.tick_n, p.n_cols, t.y, t.z,
                        p.n_splits);
}

}  // namespace mv
