// Counter-based random draws of the sketch stage (Sec. 2.3): the Gaussian
// JL matrix Phi (entries N(0, 1/s)) and the CountSketch hash and signs, made
// on the device from a 64-bit seed.
//
// Generator: Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11) -- a 128-bit
// counter and a 64-bit key; each round forms the 64-bit products of counter
// words 0 and 2 with 0xD2511F53 and 0xCD9E8D57 and mixes their halves with
// words 1 and 3 and the key, and the key advances by the Weyl constants
// 0x9E3779B9 and 0xBB67AE85 between rounds.
//
// Draw definitions (key = (seed mod 2^32, seed div 2^32)):
//  * Phi^T entry (j, t): block at counter (t div 4, j, 0, 0).  Words w_0..w_3
//    give u = ((w_a >> 8) + 1) 2^-24 in (0, 1] (a = 0, 2) and
//    v = (w_b >> 8) 2^-24 in [0, 1) (b = 1, 3), exact in FP32; the
//    Box--Muller transform r = sqrt(-2 ln u), (r cos 2 pi v, r sin 2 pi v) of
//    (u_0, v_1) and (u_2, v_3) gives four standard normals, taken by
//    t mod 4 = 0..3; the entry is that normal times 1/sqrt(s), rounded to
//    BF16 (to nearest, ties to even) from its exact value.  The transform is
//    evaluated in FP32 (logf, sqrtf, sincospif and three roundings: within
//    8 FP32 ulps of the exact value); when that FP32 value lies within 16 ulps of a BF16
//    rounding midpoint (about 1 entry in 2000) it is evaluated again in FP64,
//    so the rounded entry is the correctly rounded one in either case.
//  * CountSketch period t: block at counter (t, 0, 1, 0);
//    h(t) = (w_0 s) >> 32 (multiply-shift) and s_t = 1 - 2 (w_1 & 1).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace mv {

struct Philox4 {
    uint32_t w[4];
};

__host__ __device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                          uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    Philox4 o;
    o.w[0] = c0;
    o.w[1] = c1;
    o.w[2] = c2;
    o.w[3] = c3;
    return o;
}

// One entry: (u, v) -> BF16(r(u) cs(2 pi v) / sqrt(s)) with cs = cos (which
// = 0) or sin (which = 1).
__device__ __forceinline__ __nv_bfloat16 bm_entry(float u, float v, int which, float scale32, double scale64) {
    float sn, cs;
    sincospif(2.0f * v, &sn, &cs);
    const float y = sqrtf(-2.0f * logf(u)) * (which ? sn : cs) * scale32;
    const uint32_t low = __float_as_uint(y) & 0xFFFFu;
    const int d = (int)low - 0x8000;
    if (d > 16 || d < -16) return __float2bfloat16_rn(y);
    double s64, c64;
    sincospi(2.0 * (double)v, &s64, &c64);
    return __double2bfloat16(sqrt(-2.0 * log((double)u)) * (which ? s64 : c64) * scale64);
}

// Phi^T (s x T BF16, row pitch ld): one thread per Philox block (four
// periods of one sketch column).  Columns T..ld-1 are written as zeros.
static __global__ void __launch_bounds__(256) gaussian_sketch_kernel(uint32_t k0, uint32_t k1, int s, int T, int64_t ld,
                                                                     float scale32, double scale64,
                                                                     __nv_bfloat16 *__restrict__ out) {
    const int Q = (int)((ld + 3) / 4);                   // blocks per row, padding included
    const int64_t total = (int64_t)s * Q;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(idx / Q), q = (int)(idx - (int64_t)j * Q);
        const int t0 = 4 * q;
        __nv_bfloat16 z[4];
        if (t0 < T) {
            const Philox4 b = philox4x32_10((uint32_t)q, (uint32_t)j, 0u, 0u, k0, k1);
            const float u0 = (float)((b.w[0] >> 8) + 1u) * 5.9604644775390625e-8f;   // 2^-24
            const float v1 = (float)(b.w[1] >> 8) * 5.9604644775390625e-8f;
            const float u2 = (float)((b.w[2] >> 8) + 1u) * 5.9604644775390625e-8f;
            const float v3 = (float)(b.w[3] >> 8) * 5.9604644775390625e-8f;
            z[0] = bm_entry(u0, v1, 0, scale32, scale64);
            z[1] = bm_entry(u0, v1, 1, scale32, scale64);
            z[2] = bm_entry(u2, v3, 0, scale32, scale64);
            z[3] = bm_entry(u2, v3, 1, scale32, scale64);
        }
        __nv_bfloat16 *row = out + (int64_t)j * ld;
        const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
        if (t0 + 4 <= ld) {
            uint2 v;
            __nv_bfloat16 e[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) e[a] = (t0 + a < T) ? z[a] : zero;
            v.x = (uint32_t)__bfloat16_as_ushort(e[0]) | ((uint32_t)__bfloat16_as_ushort(e[1]) << 16);
            v.y = (uint32_t)__bfloat16_as_ushort(e[2]) | ((uint32_t)__bfloat16_as_ushort(e[3]) << 16);
            *reinterpret_cast<uint2 *>(row + t0) = v;
        } else {
            for (int a = 0; a < 4 && t0 + a < ld; ++a) row[t0 + a] = (t0 + a < T) ? z[a] : zero;
        }
    }
}

static __global__ void __launch_bounds__(256) countsketch_draw_kernel(uint32_t k0, uint32_t k1, int T, uint32_t s,
                                                               int32_t *__restrict__ h, int8_t *__restrict__ sign) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        const Philox4 b = philox4x32_10((uint32_t)t, 0u, 1u, 0u, k0, k1);
        h[t] = (int32_t)(((uint64_t)b.w[0] * s) >> 32);
        sign[t] = (int8_t)(1 - 2 * (int)(b.w[1] & 1u));
    }
}

}  // namespace mv
