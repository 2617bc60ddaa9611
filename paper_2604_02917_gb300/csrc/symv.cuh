// g = Sigma y for a symmetric n x n FP32 Sigma (explicit-covariance NPGA:
// the gradient of Sec. 3 with Sigma in place of L_eff L_eff^T).
//
// Only the tiles on and above the diagonal are read, once each: Sigma is cut
// into 128 x 128 tiles (I, J), I <= J, one CTA per tile.  An off-diagonal
// tile gives two products from the same registers,
//     rows of block I:    Sigma_IJ   y_J
//     rows of block J:    Sigma_IJ^T y_I   (= Sigma_JI y_I by symmetry),
// and a diagonal tile gives Sigma_II y_I.  Block row b thus receives exactly
// nb partial vectors, one per tile it meets; tile (I, J) stores its two into
// slot J of block I and slot I of block J.  The CTA that brings a block
// row's ticket to nb sums its nb slots (two halves in slot order, FP32 with a
// compensation term, added in FP64; fixed order: the result does not depend
// on CTA timing) and resets the ticket.
//
// Per CTA: 8 warps x 16 rows, a lane owns 4 consecutive columns (one 16-byte
// load per row, 512 contiguous bytes per warp-row); a thread issues its 16
// loads back to back before using any of them.  Column sums over a
// warp's 16 rows stay in registers and are added across warps through
// shared memory; the 16 row dot products of a warp are reduced across lanes
// by halving exchanges (8 + 4 + 2 + 1 + 1 shuffles for 16 rows).
#pragma once

#include "mv_internal.cuh"

namespace mv {

constexpr int kSymTile = 128;
constexpr int kSymThreads = 256;
constexpr int kSymRowsPerWarp = kSymTile / (kSymThreads / kWarp);   // 16

struct SymvArgs {
    const float *S;          // n x n, leading dim ld (multiple of 4), 16-byte aligned
    int64_t ld;
    int n, nb;               // nb = ceil(n / 128) tile rows
    const float *y;          // n FP32
    float *part;             // nb slots x (nb * 128) FP32 partials
    unsigned *tickets;       // nb counters, zero between launches
    double *out64;           // n FP64: Sigma y
    float *out32;            // optional n FP32 copy
    const int *done;         // optional: return at once when set
    int *err;                // error word of the caller (no wait here can time out)
};

__host__ __device__ inline int64_t symv_tiles(int nb) { return (int64_t)nb * (nb + 1) / 2; }
inline size_t symv_part_bytes(int n) {
    const int64_t nb = (n + kSymTile - 1) / kSymTile;
    return (size_t)nb * (size_t)(nb * kSymTile) * 4;
}

// L2 policy for Sigma: evict last, so the triangle stays resident from one
// iteration to the next.
__device__ __forceinline__ uint64_t l2_evict_last() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ float4 symv_ld(const float *p, uint64_t pol) {
    float4 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p), "l"(pol));
    return v;
}

// Sum the nb slots of block row b and publish: the 256 threads take the
// 128 rows twice, the first half of the slots and the second, each half in
// slot order in FP32 with a compensation term (the partials are FP32; FP64
// arithmetic is scarce on this part); the two halves are added in FP64.
// Fixed order: the result does not depend on CTA timing.  Called by the
// whole block (block-uniform condition); uses red[2][kSymTile] of shared
// memory.
__device__ __forceinline__ void symv_finish_block(const SymvArgs &a, int b, float (*red)[kSymTile]) {
    static_assert(kSymThreads == 2 * kSymTile, "two threads per row");
    const int stride = a.nb * kSymTile;
    const int i = threadIdx.x & (kSymTile - 1), h = threadIdx.x / kSymTile;
    const int r = b * kSymTile + i;
    const int jh = (a.nb + 1) / 2, j0 = h * jh, j1 = min(a.nb, j0 + jh);
    float s = 0.f, c = 0.f;
    if (r < a.n) {
#pragma unroll 8
        for (int j = j0; j < j1; ++j) {
            const float y = __ldcg(a.part + (int64_t)j * stride + r) - c;
            const float t = s + y;
            c = (t - s) - y;
            s = t;
        }
    }
    if (h == 1) {
        red[0][i] = s;
        red[1][i] = c;
    }
    __syncthreads();
    if (h == 0 && r < a.n) {
        const double v = ((double)s - (double)c) + ((double)red[0][i] - (double)red[1][i]);
        a.out64[r] = v;
        if (a.out32) a.out32[r] = (float)v;
    }
    __syncthreads();                  // red is reused by a second finish
}

static __global__ void __launch_bounds__(kSymThreads) symv_kernel(SymvArgs a) {
    if (a.done && *(volatile const int *)a.done) return;
    __shared__ float yI[kSymTile], yJ[kSymTile];
    __shared__ float colred[kSymThreads / kWarp][kSymTile];
    __shared__ int s_last[2];
    // tile -> (I, J), I <= J, row-major over the upper triangle
    int t = blockIdx.x, I = 0;
    while (t >= a.nb - I) {
        t -= a.nb - I;
        ++I;
    }
    const int J = I + t;
    const int r0 = I * kSymTile, c0 = J * kSymTile;
    for (int i = threadIdx.x; i < kSymTile; i += kSymThreads) {
        yI[i] = r0 + i < a.n ? a.y[r0 + i] : 0.f;
        yJ[i] = c0 + i < a.n ? a.y[c0 + i] : 0.f;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rw = warp * kSymRowsPerWarp;
    const int col = c0 + 4 * lane;
    // All 16 loads are issued before any use: addresses are clamped into the
    // matrix (row n-1, the last 4-column group), and what the clamp brings in
    // is cancelled below (zero y entries for rows, masks for columns).
    const uint64_t pol = l2_evict_last();
    const int cl = min(col, (a.n - 1) & ~3);
    float4 v[kSymRowsPerWarp];
#pragma unroll
    for (int j = 0; j < kSymRowsPerWarp; ++j) {
        const int r = min(r0 + rw + j, a.n - 1);
        v[j] = symv_ld(a.S + (int64_t)r * a.ld + cl, pol);
    }
    if (col + 3 >= a.n) {          // the last column block only: columns past n are not Sigma's
#pragma unroll
        for (int j = 0; j < kSymRowsPerWarp; ++j) {
            v[j].x = col + 0 < a.n ? v[j].x : 0.f;
            v[j].y = col + 1 < a.n ? v[j].y : 0.f;
            v[j].z = col + 2 < a.n ? v[j].z : 0.f;
            v[j].w = col + 3 < a.n ? v[j].w : 0.f;
        }
    }
    const float4 yj = *reinterpret_cast<const float4 *>(&yJ[4 * lane]);
    float cx = 0.f, cy = 0.f, cz = 0.f, cw = 0.f;
    float rp[kSymRowsPerWarp];
#pragma unroll
    for (int j = 0; j < kSymRowsPerWarp; ++j) {
        const float yi = yI[rw + j];          // 0 for rows past n
        cx = fmaf(v[j].x, yi, cx);
        cy = fmaf(v[j].y, yi, cy);
        cz = fmaf(v[j].z, yi, cz);
        cw = fmaf(v[j].w, yi, cw);
        rp[j] = fmaf(v[j].w, yj.w, fmaf(v[j].z, yj.z, fmaf(v[j].y, yj.y, v[j].x * yj.x)));
    }
    // Row sums across the 32 lanes: halving exchanges leave row
    // rw + (lane >> 1) in lanes 2i and 2i+1.
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const bool up = lane & 16;
        const float send = up ? rp[k] : rp[k + 8];
        const float keep = up ? rp[k + 8] : rp[k];
        rp[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const bool up = lane & 8;
        const float send = up ? rp[k] : rp[k + 4];
        const float keep = up ? rp[k + 4] : rp[k];
        rp[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const bool up = lane & 4;
        const float send = up ? rp[k] : rp[k + 2];
        const float keep = up ? rp[k + 2] : rp[k];
        rp[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    {
        const bool up = lane & 2;
        const float send = up ? rp[0] : rp[1];
        const float keep = up ? rp[1] : rp[0];
        rp[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    rp[0] += __shfl_xor_sync(0xffffffffu, rp[0], 1);
    const int stride = a.nb * kSymTile;
    // row index held: bits 4..1 of the lane, most significant first
    const int rr = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
    if ((lane & 1) == 0 && r0 + rw + rr < a.n) a.part[(int64_t)J * stride + r0 + rw + rr] = rp[0];
    if (I != J) {
        *reinterpret_cast<float4 *>(&colred[warp][4 * lane]) = make_float4(cx, cy, cz, cw);
        __syncthreads();
        for (int c = threadIdx.x; c < kSymTile; c += kSymThreads) {
            float s = 0.f;
#pragma unroll
            for (int w = 0; w < kSymThreads / kWarp; ++w) s += colred[w][c];
            if (c0 + c < a.n) a.part[(int64_t)I * stride + c0 + c] = s;
        }
    }
    // tickets: the last of the nb contributors of a block row reduces it
    // (the block barrier, then one thread's device fence, publishes every
    // thread's partials before the ticket)
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last[0] = atomicAdd(&a.tickets[I], 1u) == (unsigned)(a.nb - 1);
        s_last[1] = (I != J) && atomicAdd(&a.tickets[J], 1u) == (unsigned)(a.nb - 1);
    }
    __syncthreads();
    if (s_last[0]) {
        __threadfence();
        symv_finish_block(a, I, colred);
        if (threadIdx.x == 0) a.tickets[I] = 0u;
    }
    if (s_last[1]) {
        __threadfence();
        symv_finish_block(a, J, colred);
        if (threadIdx.x == 0) a.tickets[J] = 0u;
    }
}

// Enqueue Sigma y (capturable): one CTA per upper tile.
inline int symv_launch(const SymvArgs &a, cudaStream_t s) {
    symv_kernel<<<(unsigned)symv_tiles(a.nb), kSymThreads, 0, s>>>(a);
    return MV_OK;
}

}  // namespace mv
