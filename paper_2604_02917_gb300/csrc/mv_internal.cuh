// Internal helpers shared by the libmv translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <math.h>

#include "../../include/mv.h"

namespace mv {

constexpr int kWarp = 32;

// Records the failing call for mv_last_error() and returns MV_ERR_CUDA.
int record_cuda_error(cudaError_t e, const char *what, const char *file, int line);
// Records a message for mv_last_error() and returns `status`.
int record_message(int status, const char *msg);

#define MV_CUDA_TRY(expr)                                                     \
    do {                                                                      \
        cudaError_t _e = (expr);                                              \
        if (_e != cudaSuccess) return record_cuda_error(_e, #expr, __FILE__, __LINE__); \
    } while (0)

#define MV_TRY(expr)                                           \
    do {                                                       \
        int _s = (expr);                                       \
        if (_s != MV_OK) return _s;                            \
    } while (0)

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------- storage
// 16-byte read-once load: L is streamed from HBM exactly once per pass, so
// it bypasses L1 allocation.
__device__ __forceinline__ uint4 ld_stream16(const void *p) {
    uint4 r;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(p));
    return r;
}

template <int DT> struct Store;

template <> struct Store<MV_F32> {
    using elem = float;
    static constexpr int VEC = 4;  // elements per 16-byte vector
    __device__ __forceinline__ static void unpack(const uint4 &u, float *f) {
        f[0] = __uint_as_float(u.x);
        f[1] = __uint_as_float(u.y);
        f[2] = __uint_as_float(u.z);
        f[3] = __uint_as_float(u.w);
    }
    __device__ __forceinline__ static float load1(const void *base, int64_t idx) {
        return __ldg(reinterpret_cast<const float *>(base) + idx);
    }
};

template <> struct Store<MV_BF16> {
    using elem = __nv_bfloat16;
    static constexpr int VEC = 8;
    __device__ __forceinline__ static void two(uint32_t w, float *f) {
        f[0] = __uint_as_float(w << 16);
        f[1] = __uint_as_float(w & 0xffff0000u);
    }
    __device__ __forceinline__ static void unpack(const uint4 &u, float *f) {
        two(u.x, f + 0);
        two(u.y, f + 2);
        two(u.z, f + 4);
        two(u.w, f + 6);
    }
    __device__ __forceinline__ static float load1(const void *base, int64_t idx) {
        unsigned short b = __ldg(reinterpret_cast<const unsigned short *>(base) + idx);
        return __uint_as_float(((uint32_t)b) << 16);
    }
};

template <> struct Store<MV_FP8_E4M3> {
    using elem = __nv_fp8_e4m3;
    static constexpr int VEC = 16;
    __device__ __forceinline__ static void four(uint32_t w, float *f) {
        __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w & 0xffffu), __NV_E4M3);
        __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w >> 16), __NV_E4M3);
        float2 a = __half22float2(*reinterpret_cast<__half2 *>(&lo));
        float2 b = __half22float2(*reinterpret_cast<__half2 *>(&hi));
        f[0] = a.x;
        f[1] = a.y;
        f[2] = b.x;
        f[3] = b.y;
    }
    __device__ __forceinline__ static void unpack(const uint4 &u, float *f) {
        four(u.x, f + 0);
        four(u.y, f + 4);
        four(u.z, f + 8);
        four(u.w, f + 12);
    }
    __device__ __forceinline__ static float load1(const void *base, int64_t idx) {
        unsigned char b = __ldg(reinterpret_cast<const unsigned char *>(base) + idx);
        __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)b, __NV_E4M3);
        return __half2float(*reinterpret_cast<__half *>(&h));
    }
};

inline int dtype_size(int dt) { return dt == MV_F32 ? 4 : (dt == MV_BF16 ? 2 : (dt == MV_FP8_E4M3 ? 1 : 0)); }

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum of NV doubles held by every thread; all threads get the
// totals.  `red` needs (NT/32 + 1) * NV doubles of shared memory.  Two
// barriers; the result slot is disjoint from the partial slots, so
// back-to-back calls need no extra barrier.
template <int NV, int NT>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *red) {
    constexpr int NW = NT / kWarp;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) red[warp * NV + k] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = lane < NW ? red[lane * NV + k] : 0.0;
            s = warp_sum(s);
            if (lane == 0) red[NW * NV + k] = s;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = red[NW * NV + k];
}

template <int NT>
__device__ __forceinline__ void block_minmax(double &mn, double &mx, double *red) {
    constexpr int NW = NT / kWarp;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    mn = warp_min(mn);
    mx = warp_max(mx);
    if (lane == 0) {
        red[warp * 2 + 0] = mn;
        red[warp * 2 + 1] = mx;
    }
    __syncthreads();
    if (warp == 0) {
        double a = lane < NW ? red[lane * 2 + 0] : INFINITY;
        double b = lane < NW ? red[lane * 2 + 1] : -INFINITY;
        a = warp_min(a);
        b = warp_max(b);
        if (lane == 0) {
            red[NW * 2 + 0] = a;
            red[NW * 2 + 1] = b;
        }
    }
    __syncthreads();
    mn = red[NW * 2 + 0];
    mx = red[NW * 2 + 1];
}

}  // namespace mv
