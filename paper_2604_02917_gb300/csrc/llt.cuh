// Fused Gram product  g = L (L^T y)  in ONE pass over L (Sec. 2.7: the
// NPGA gradient 2 L L^T y + 2 gamma y and the power method's L L^T u both
// need only this product, never z = L^T y itself).
//
// Column blocking.  L (n x T, row-major) is cut into column blocks of W
// columns, W * sizeof(elem) = RB bytes (32 by default: one DRAM sector per row).  A
// thread-block cluster of C CTAs (C = 2, a TPC pair, for n up to about 6000;
// 4 or 8 beyond) owns one column block at a time: CTA rank r holds rows
// [r*rpc, (r+1)*rpc) of the block in shared memory (TMA 2-D loads with the
// RB-byte swizzle, zero fill past n and T).  Per block:
//   A. each of 16 consumer warps forms the partial column sums of one
//      16-byte chunk over a share of the CTA's rows, all-reduces them over
//      the warp and pushes them into every CTA of the cluster with st.async
//      (distributed shared memory; completion counted in bytes on an mbarrier
//      of the receiver) -- no block barrier;
//   B. every CTA adds the partials of each column in a fixed order (the
//      same bits on all CTAs), giving z_b = L[:, b]^T y, and accumulates
//      g[rows_r] += L[rows_r, b] z_b  (one thread per row, compensated sums
//      in registers) from the block still in shared memory.
// So every element of L is read from HBM once per product instead of once
// per half-product.  Clusters are persistent and take column blocks
// round-robin; their per-row partial sums of g go to a [clusters x n]
// buffer, added in a fixed two-level order in FP64 by the last CTAs to
// finish (atomic tickets after a fence, no spinning).
//
// Roles: one producer warp keeps a 2-stage ring of row blocks in flight
// (full/empty mbarriers); a stage is ~87 KB per CTA at n = 5440 FP32, about
// 2 us of this SM's share of HBM bandwidth, against well under 1 us of
// compute and exchange per block, so the loads stay back to back.  Two
// exchange slots suffice: a CTA pushes block j+2 only after it received
// block j+1 from every peer warp, which each peer pushed after it had
// consumed block j.  One block barrier per column block (after the receive).
//
// Every mbarrier wait is bounded in time; on timeout the thread records an
// error code and carries on with short waits, so no peer is left waiting.
#pragma once

#include <cooperative_groups.h>

#include "gemm.cuh"
#include "llt_api.h"

namespace mv {

constexpr int kLltConsumerWarps = 16;
constexpr int kLltConsumers = kLltConsumerWarps * 32;
constexpr int kLltThreads = kLltConsumers + 32; // + one producer warp
constexpr int kLltSlots = 2;
constexpr int kLltStages = 2;
constexpr int kLltRowsPerThread = 8;            // rows of phase B per consumer thread (max)
constexpr uint64_t kLltWaitNs = 2000000000ull;
constexpr uint64_t kLltBailNs = 1000000ull;     // after a timeout: 1 ms per wait

struct LltArgs {
    const float *y32;          // n: gemv input (FP8: pre-multiplied by the row scale)
    const float *row_scale;    // n or null (FP8)
    float *gpart;              // [G x n] per-cluster partials
    double *gq;                // [groups x n] group sums
    double *g;                 // n: L L^T y (row-scaled)
    float *g32;                // n or null
    float *z;                  // T or null: z = L^T y, the slices the exchange forms anyway
    unsigned *tick1;           // [C x kLltMaxGroups], zero between launches
    unsigned *tick2;           // [C], zero between launches
    int *err;                  // error word (0 = fine)
    const int *done;           // early-exit flag or null
    int n, T;
    int rpc, box_rows, nbox, nb, G;
    int early;                 // launched as a programmatic dependent: the loads of L (which
                               // no predecessor writes) go out before the grid-dependency wait
};

namespace llt {

__device__ __forceinline__ uint32_t mapa(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
// Asynchronous 16-byte store into another CTA's shared memory; the bytes
// are counted on that CTA's mbarrier.
__device__ __forceinline__ void st_async_v4(uint32_t raddr, float4 v, uint32_t rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                     raddr),
                 "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(rbar)
                 : "memory");
}
__device__ __forceinline__ void st_async_f32(uint32_t raddr, float v, uint32_t rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];" ::"r"(raddr), "f"(v),
                 "r"(rbar)
                 : "memory");
}
__device__ __forceinline__ void st_async_v2(uint32_t raddr, float a, float b, uint32_t rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(raddr),
                 "f"(a), "f"(b), "r"(rbar)
                 : "memory");
}
__device__ __forceinline__ bool try_wait_cluster(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool wait_cluster(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
    if (try_wait_cluster(bar, parity)) return true;
    const uint64_t t0 = umma::globaltimer();
    while (true) {
        if (try_wait_cluster(bar, parity)) return true;
        if (umma::globaltimer() - t0 > limit_ns) return false;
    }
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Named barrier over the consumer warps only (the producer never joins it).
__device__ __forceinline__ void bar_consumers() {
    asm volatile("bar.sync 1, %0;" ::"n"(kLltConsumers) : "memory");
}
// Byte offset of 16-byte chunk c of row r of RB-byte rows under the RB-byte
// TMA swizzle: the chunk lands at c ^ ((r / (128 / RB)) mod (RB / 16)).
template <int RB>
__device__ __forceinline__ int swz(int r, int c) {
    return r * RB + ((c ^ ((r / (128 / RB)) & (RB / 16 - 1))) << 4);
}

}  // namespace llt

// Fixed-order two-level reduction of the per-cluster partials of the rows
// [row0, row0 + a.rpc) of this rank: the last CTA of each group of kLltFan
// clusters adds the group's partials (FP64), the last group adds the group
// sums, applies the FP8 scale and writes g.  Every thread of the CTA calls it.
__device__ __forceinline__ void llt_final_reduce(const LltArgs &a, int cid, int rank, int row0) {
    __shared__ int s_flag;
    const int tid = threadIdx.x;
    const int ngrp = (a.G + kLltFan - 1) / kLltFan, mygrp = cid / kLltFan;
    const int c0 = mygrp * kLltFan, c1 = min(a.G, c0 + kLltFan);
    // Four rows per thread with every load of a level issued at once (the
    // levels are L2-latency bound); the sums keep the same order either way.
    const bool vec = (a.n % 4 == 0) && (row0 % 4 == 0) && (a.rpc % 4 == 0);
    __threadfence();
    __syncthreads();
    if (tid == 0) s_flag = atomicAdd(&a.tick1[rank * kLltMaxGroups + mygrp], 1u) == (unsigned)(c1 - c0 - 1);
    __syncthreads();
    if (!s_flag) return;
    __threadfence();
    if (vec) {
        for (int i = 4 * tid; i < a.rpc; i += 4 * kLltThreads) {
            const int r = row0 + i;
            if (r >= a.n) break;
            float4 v[kLltFan];
#pragma unroll
            for (int c = 0; c < kLltFan; ++c)
                v[c] = c0 + c < c1 ? __ldcg(reinterpret_cast<const float4 *>(a.gpart + (size_t)(c0 + c) * a.n + r))
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
#pragma unroll
            for (int c = 0; c < kLltFan; ++c) {
                if (c0 + c < c1) {
                    s0 += (double)v[c].x;
                    s1 += (double)v[c].y;
                    s2 += (double)v[c].z;
                    s3 += (double)v[c].w;
                }
            }
            double2 *q = reinterpret_cast<double2 *>(a.gq + (size_t)mygrp * a.n + r);
            q[0] = make_double2(s0, s1);
            q[1] = make_double2(s2, s3);
        }
    } else {
        for (int i = tid; i < a.rpc; i += kLltThreads) {
            const int r = row0 + i;
            if (r >= a.n) break;
            double s = 0.0;
#pragma unroll 8
            for (int c = c0; c < c1; ++c) s += (double)__ldcg(a.gpart + (size_t)c * a.n + r);
            a.gq[(size_t)mygrp * a.n + r] = s;
        }
    }
    if (tid == 0) a.tick1[rank * kLltMaxGroups + mygrp] = 0u;
    __threadfence();
    __syncthreads();
    if (tid == 0) s_flag = atomicAdd(&a.tick2[rank], 1u) == (unsigned)(ngrp - 1);
    __syncthreads();
    if (!s_flag) return;
    __threadfence();
    if (vec) {
        for (int i = 4 * tid; i < a.rpc; i += 4 * kLltThreads) {
            const int r = row0 + i;
            if (r >= a.n) break;
            double t[4] = {0.0, 0.0, 0.0, 0.0};
            for (int k0 = 0; k0 < ngrp; k0 += 4) {            // four groups' loads in flight at a time
                double2 v[8];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const double2 *q = reinterpret_cast<const double2 *>(a.gq + (size_t)(k0 + k) * a.n + r);
                    v[2 * k] = k0 + k < ngrp ? __ldcg(q) : make_double2(0.0, 0.0);
                    v[2 * k + 1] = k0 + k < ngrp ? __ldcg(q + 1) : make_double2(0.0, 0.0);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (k0 + k < ngrp) {
                        t[0] += v[2 * k].x;
                        t[1] += v[2 * k].y;
                        t[2] += v[2 * k + 1].x;
                        t[3] += v[2 * k + 1].y;
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                double g = t[e];
                if (a.row_scale != nullptr) g *= (double)a.row_scale[r + e];
                a.g[r + e] = g;
                if (a.g32 != nullptr) a.g32[r + e] = (float)g;
            }
        }
    } else {
        for (int i = tid; i < a.rpc; i += kLltThreads) {
            const int r = row0 + i;
            if (r >= a.n) break;
            double s = 0.0;
#pragma unroll 8
            for (int k = 0; k < ngrp; ++k) s += __ldcg(a.gq + (size_t)k * a.n + r);
            if (a.row_scale != nullptr) s *= (double)a.row_scale[r];
            a.g[r] = s;
            if (a.g32 != nullptr) a.g32[r] = (float)s;
        }
    }
    if (tid == 0) a.tick2[rank] = 0u;
}

// Shared-memory layout (bytes) for a given geometry.
struct LltSmem {
    size_t stage, o_slots, o_y, o_zc, o_bars, total;
};
__host__ __device__ inline LltSmem llt_smem_layout(int rpc, int RB, int W, int C) {
    LltSmem m{};
    m.stage = (size_t)rpc * RB;
    size_t off = m.stage * kLltStages;
    m.o_slots = off;
    off += (size_t)kLltSlots * C * (kLltConsumerWarps / (RB / 16)) * W * 4;
    m.o_y = off;
    off += (size_t)rpc * 4;
    m.o_zc = off;
    off += (size_t)2 * W * 4;
    off = (off + 15) / 16 * 16;
    m.o_bars = off;
    off += 8 * (size_t)(2 * kLltStages + kLltSlots);
    m.total = off + 1024;                // slack for aligning the dynamic base to 1024 bytes
    return m;
}

template <int DT, int C, int RB>
__global__ void __launch_bounds__(kLltThreads, 1)
llt_kernel(const __grid_constant__ CUtensorMap tmL, const LltArgs a) {
    using S = Store<DT>;
    constexpr int EPC = S::VEC;                        // elements per 16-byte chunk
    constexpr int NCH = RB / 16;                       // 16-byte chunks per row
    constexpr int W = RB / (int)sizeof(typename S::elem);
    constexpr int NG = kLltConsumerWarps / NCH;        // row groups of phase A
    constexpr int V4 = EPC / 4;                        // float4 pieces of one chunk's partials
    constexpr int RPT = kLltRowsPerThread;
    namespace cg = cooperative_groups;
    if (a.done != nullptr && *(const volatile int *)a.done) return;

    extern __shared__ uint8_t smem_raw[];
    // aligned up to 1024 bytes by pointer arithmetic on the shared array (an
    // integer round trip would hide from the compiler that it is shared memory)
    uint8_t *sm = smem_raw + ((1024u - (uint32_t)(reinterpret_cast<uintptr_t>(smem_raw) & 1023u)) & 1023u);
    const LltSmem L = llt_smem_layout(a.rpc, RB, W, C);
    float *slots = reinterpret_cast<float *>(sm + L.o_slots);       // [2][C][NG][W]
    float *s_y = reinterpret_cast<float *>(sm + L.o_y);
    float *s_zc = reinterpret_cast<float *>(sm + L.o_zc);           // [2][W]
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L.o_bars);
    const uint32_t full0 = umma::smem_u32(bars), empty0 = umma::smem_u32(bars + kLltStages);
    const uint32_t xchg0 = umma::smem_u32(bars + 2 * kLltStages);
    const uint32_t slots_u32 = umma::smem_u32(slots);

    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int cid = blockIdx.x / C;
    const int row0 = rank * a.rpc;
    const int nj = (a.nb - cid + a.G - 1) / a.G;       // column blocks of this cluster (>= 1)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t xbytes = (uint32_t)(C * NG * W * 4);
    const uint32_t stage_tx = (uint32_t)(a.nbox * a.box_rows * RB);

    if (tid == 0) {
        for (int s = 0; s < kLltStages; ++s) {
            umma::mbar_init(full0 + 8 * s, 1);
            umma::mbar_init(empty0 + 8 * s, kLltConsumerWarps);
        }
        for (int q = 0; q < kLltSlots; ++q) umma::mbar_init(xchg0 + 8 * q, 1);
        umma::mbar_fence_init();
        for (int q = 0; q < kLltSlots && q < nj; ++q) umma::mbar_arrive_expect_tx(xchg0 + 8 * q, xbytes);
    }
    __syncthreads();
    // The first stages' loads go out before the cluster barrier: they touch
    // only this CTA's shared memory and barriers.
    auto issue = [&](int j) {
        const int s = j % kLltStages;
        const int b = cid + j * a.G;
        const uint32_t dst = umma::smem_u32(sm + (size_t)s * L.stage);
        umma::mbar_arrive_expect_tx(full0 + 8 * s, stage_tx);
        for (int i = 0; i < a.nbox; ++i)
            umma::tma_load_2d(dst + (uint32_t)(i * a.box_rows * RB), &tmL, b * W, row0 + i * a.box_rows,
                              full0 + 8 * s);
    };
    if (warp == kLltConsumerWarps && lane == 0) {
        umma::prefetch_tensormap(&tmL);
        for (int j = 0; j < kLltStages && j < nj; ++j) issue(j);
    }
    for (int i = tid; i < a.rpc; i += kLltThreads) {
        const int r = row0 + i;
        s_y[i] = r < a.n ? a.y32[r] : 0.f;
    }
    cluster.sync();                                     // peers' barriers exist before any push

    float gs[RPT], gc[RPT];                            // consumers: compensated g of rows tid + 512 k
#pragma unroll
    for (int k = 0; k < RPT; ++k) gs[k] = gc[k] = 0.f;

    if (warp == kLltConsumerWarps) {
        // ---------------- producer: column block j of this cluster -> stage j % 2
        if (lane == 0) {
            bool bail = false;
            for (int j = kLltStages; j < nj; ++j) {
                const int s = j % kLltStages;
                if (!umma::mbar_wait(empty0 + 8 * s, (uint32_t)(j / kLltStages - 1) & 1u,
                                     bail ? kLltBailNs : kLltWaitNs)) {
                    atomicExch(a.err, 3);
                    bail = true;
                }
                issue(j);
            }
            // Drain: every stage's last load has landed before the CTA may exit.
            for (int j = nj - kLltStages < 0 ? 0 : nj - kLltStages; j < nj; ++j)
                if (!umma::mbar_wait(full0 + 8 * (j % kLltStages), (uint32_t)(j / kLltStages) & 1u, kLltWaitNs))
                    atomicExch(a.err, 4);
        }
        __syncwarp();
    } else {
        // ---------------- consumers
        bool bail = false;
        const int ch = warp % NCH, grp = warp / NCH;
        for (int j = 0; j < nj; ++j) {
            const int s = j % kLltStages, q = j % kLltSlots;
            if (!umma::mbar_wait(full0 + 8 * s, (uint32_t)(j / kLltStages) & 1u, bail ? kLltBailNs : kLltWaitNs)) {
                atomicExch(a.err, 1);
                bail = true;
            }
            const uint8_t *sb = sm + (size_t)s * L.stage;
            // Phase A: warp (chunk ch, row group grp) sums its rows, all-reduces
            // over the warp and pushes the chunk's partials to every rank.
            {
                float acc[EPC];
#pragma unroll
                for (int e = 0; e < EPC; ++e) acc[e] = 0.f;
#pragma unroll 4
                for (int r = grp * 32 + lane; r < a.rpc; r += 32 * NG) {
                    const uint4 u = *reinterpret_cast<const uint4 *>(sb + llt::swz<RB>(r, ch));
                    float f[EPC];
                    S::unpack(u, f);
                    const float yy = s_y[r];
#pragma unroll
                    for (int e = 0; e < EPC; ++e) acc[e] = fmaf(f[e], yy, acc[e]);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                    for (int e = 0; e < EPC; ++e) acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], o);
                if (lane < C * V4) {
                    const int dst = lane / V4, piece = lane % V4;
                    float4 v = make_float4(acc[0], acc[1], acc[2], acc[3]);
#pragma unroll
                    for (int k = 1; k < V4; ++k)
                        if (piece == k) v = make_float4(acc[4 * k], acc[4 * k + 1], acc[4 * k + 2], acc[4 * k + 3]);
                    const uint32_t local =
                        slots_u32 + (uint32_t)((((q * C + rank) * NG + grp) * W + ch * EPC + 4 * piece) * 4);
                    llt::st_async_v4(llt::mapa(local, (uint32_t)dst), v, llt::mapa(xchg0 + 8 * q, (uint32_t)dst));
                }
            }
            // Receive: z_b = sum over ranks and row groups, in a fixed order.
            float *zc = s_zc + (j & 1) * W;
            if (tid < W) {
                if (!llt::wait_cluster(xchg0 + 8 * q, (uint32_t)(j / kLltSlots) & 1u, bail ? kLltBailNs : kLltWaitNs)) {
                    atomicExch(a.err, 2);
                    bail = true;
                }
                const float *sl = slots + (size_t)q * C * NG * W + tid;
                float z = 0.f;
#pragma unroll
                for (int k = 0; k < C * NG; ++k) z += sl[k * W];
                zc[tid] = z;
                const int zcol = (cid + j * a.G) * W + tid;
                if (a.z != nullptr && rank == 0 && zcol < a.T) a.z[zcol] = z;
                if (tid == 0 && j + kLltSlots < nj) umma::mbar_arrive_expect_tx(xchg0 + 8 * q, xbytes);
            }
            llt::bar_consumers();
            // Phase B: g[rows] += L[rows, block j] z_b, one thread per row.  Under
            // the swizzle the 8 rows of a quarter-warp hit distinct bank groups,
            // while every thread reads the same z chunk (a broadcast).
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const int r = tid + k * kLltConsumers;
                if (r < a.rpc) {
                    float d0 = 0.f, d1 = 0.f;
#pragma unroll
                    for (int c = 0; c < NCH; ++c) {
                        const uint4 u = *reinterpret_cast<const uint4 *>(sb + llt::swz<RB>(r, c));
                        float f[EPC];
                        S::unpack(u, f);
#pragma unroll
                        for (int e = 0; e < EPC; e += 4) {
                            const float4 zq = *reinterpret_cast<const float4 *>(zc + c * EPC + e);
                            d0 = fmaf(f[e], zq.x, d0);
                            d1 = fmaf(f[e + 1], zq.y, d1);
                            d0 = fmaf(f[e + 2], zq.z, d0);
                            d1 = fmaf(f[e + 3], zq.w, d1);
                        }
                    }
                    const float yk = (d0 + d1) - gc[k];
                    const float tk = gs[k] + yk;
                    gc[k] = (tk - gs[k]) - yk;
                    gs[k] = tk;
                }
            }
            __syncwarp();
            if (lane == 0) llt::mbar_arrive(empty0 + 8 * s);      // this warp is done with the stage
        }
        // Per-cluster partial of g for this CTA's rows.
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int r = tid + k * kLltConsumers;
            if (r < a.rpc && row0 + r < a.n) a.gpart[(size_t)cid * a.n + row0 + r] = gs[k] - gc[k];
        }
    }

    llt_final_reduce(a, cid, rank, row0);
    cluster.sync();                                     // no CTA leaves while a peer may still push to it
}

// ------------------------------------------------------------------ transposed layout
// The same product over M = L^T stored T x n (row t = period t).  Column
// block b of L is the row block [b W, (b+1) W) of M with W * sizeof(elem) =
// 32 bytes (8 periods FP32, 16 BF16, 32 FP8); CTA rank r of a cluster holds
// the asset columns [r npc, (r+1) npc) of it, so each TMA box row is a run
// of kLltBoxCols contiguous assets (1 KB FP32) -- the access streams like a
// plain copy.  Stage layout: [box k][row w][kLltBoxCols elements].
//   A. warp (row w, part h) dots its row's chunks with y: z_b[w] partial,
//      pushed to every rank (RW floats per warp);
//   B. one thread per 16-byte column chunk: g[cols] += sum_w M[bW+w, cols] z_b[w].
constexpr int kLltBoxCols = 256;                 // elements per TMA box row
// Phase A rows per warp of the transposed pass: FP32 (8 periods per block),
// BF16 and FP8 (16 and 32 periods).
constexpr int kLltRowsA32 = 2, kLltRowsA16 = 4;
constexpr int kLltMaxRowsA = 8;                  // bound the exchange slots are sized for

__host__ __device__ inline LltSmem lltt_smem_layout(int npc, int C) {
    LltSmem m{};
    m.stage = (size_t)npc * 32;                  // W rows x npc elements, W * esize = 32 bytes
    size_t off = m.stage * kLltStages;
    m.o_slots = off;
    off += (size_t)kLltSlots * C * kLltConsumerWarps * kLltMaxRowsA * 4;   // [2][C][16 warps x RW floats]
    m.o_y = off;
    off += (size_t)npc * 4;
    m.o_zc = off;
    off += (size_t)2 * 32 * 4;
    off = (off + 15) / 16 * 16;
    m.o_bars = off;
    off += 8 * (size_t)(2 * kLltStages + kLltSlots);
    m.total = off + 1024;
    return m;
}

// The transposed pass of cluster cid (of a.G) over the tensor map tm.  With
// kGlobalMap the map lives in global memory (one per problem of a grouped
// launch) and the producer orders the tensor-map proxy after the host's
// copy of it before its first load.
template <int DT, int C, bool kGlobalMap>
__device__ __forceinline__ void lltt_body(const CUtensorMap *tm, const LltArgs &a, const int cid) {
    using S = Store<DT>;
    constexpr int ES = (int)sizeof(typename S::elem);
    constexpr int EPC = S::VEC;                          // elements per 16-byte chunk
    constexpr int W = 32 / ES;                           // periods per column block
    // Phase A: a warp dots RW rows of the block with the same chunks of y,
    // so each y load (EPC FP32 values per 16-byte chunk of L) serves RW rows;
    // WPR warps share a row's chunks.  (One row per warp made the BF16 and
    // FP8 passes load as many bytes of y from shared memory as of L.)
    constexpr int RW = (ES == 4) ? kLltRowsA32 : kLltRowsA16;   // rows per warp
    constexpr int WPR = kLltConsumerWarps * RW / W;      // warps per row
    constexpr int NGR = W / RW;                          // row groups
    static_assert(NGR * WPR == kLltConsumerWarps && RW <= kLltMaxRowsA && RW % 2 == 0, "phase A split");
    constexpr int NP = kLltConsumerWarps * RW;           // partials per rank and block
    constexpr int CPB = kLltBoxCols * ES / 16;           // 16-byte chunks per box row
    constexpr int BOXB = W * kLltBoxCols * ES;           // bytes of one box
    constexpr int RPT = (ES == 4) ? 2 : 1;               // column chunks per thread in phase B
    namespace cg = cooperative_groups;
    if (a.done != nullptr && *(const volatile int *)a.done) return;

    extern __shared__ uint8_t smem_raw[];
    // aligned up to 1024 bytes by pointer arithmetic on the shared array (an
    // integer round trip would hide from the compiler that it is shared memory)
    uint8_t *sm = smem_raw + ((1024u - (uint32_t)(reinterpret_cast<uintptr_t>(smem_raw) & 1023u)) & 1023u);
    const int npc = a.rpc;                               // asset columns of this CTA
    const LltSmem L = lltt_smem_layout(npc, C);
    float *slots = reinterpret_cast<float *>(sm + L.o_slots);       // [2][C][NP]
    float *s_y = reinterpret_cast<float *>(sm + L.o_y);
    float *s_zc = reinterpret_cast<float *>(sm + L.o_zc);           // [2][W]
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L.o_bars);
    const uint32_t full0 = umma::smem_u32(bars), empty0 = umma::smem_u32(bars + kLltStages);
    const uint32_t xchg0 = umma::smem_u32(bars + 2 * kLltStages);
    const uint32_t slots_u32 = umma::smem_u32(slots);

    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int col0 = rank * npc;
    const int nj = (a.nb - cid + a.G - 1) / a.G;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nch = npc * ES / 16;                       // 16-byte chunks of one row of the stage
    const uint32_t xbytes = (uint32_t)(C * NP * 4);
    const uint32_t stage_tx = (uint32_t)(a.nbox * BOXB);

    if (tid == 0) {
        for (int s = 0; s < kLltStages; ++s) {
            umma::mbar_init(full0 + 8 * s, 1);
            umma::mbar_init(empty0 + 8 * s, kLltConsumerWarps);
        }
        for (int q = 0; q < kLltSlots; ++q) umma::mbar_init(xchg0 + 8 * q, 1);
        umma::mbar_fence_init();
        for (int q = 0; q < kLltSlots && q < nj; ++q) umma::mbar_arrive_expect_tx(xchg0 + 8 * q, xbytes);
    }
    __syncthreads();
    auto issue = [&](int j) {
        const int s = j % kLltStages;
        const int b = cid + j * a.G;
        const uint32_t dst = umma::smem_u32(sm + (size_t)s * L.stage);
        umma::mbar_arrive_expect_tx(full0 + 8 * s, stage_tx);
        for (int k = 0; k < a.nbox; ++k)
            umma::tma_load_2d(dst + (uint32_t)(k * BOXB), tm, col0 + k * kLltBoxCols, b * W, full0 + 8 * s);
    };
    const bool producer = warp == kLltConsumerWarps && lane == 0;
    if (producer) {                                        // first stages before the cluster barrier
        if constexpr (kGlobalMap)
            asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(tm))
                         : "memory");
        umma::prefetch_tensormap(tm);
        if (a.early) {
            // Launched while the previous kernel (the step or the power
            // normalisation, which read y and write the next one) still
            // runs: L is read-only, so its first stages stream meanwhile.
            // (Prefetching further blocks into L2 as well measured slower:
            // 21.2 against 20.8 ms per solve.)
            for (int j = 0; j < kLltStages && j < nj; ++j) issue(j);
        }
    }
    if (a.early) {
        umma::grid_dependency_wait();                      // y, done and the scratch are the predecessor's
        if (a.done != nullptr && *(const volatile int *)a.done) {
            if (producer)                                  // the issued stages land before the CTA leaves
                for (int j = 0; j < kLltStages && j < nj; ++j)
                    if (!umma::mbar_wait(full0 + 8 * j, 0u, kLltWaitNs)) atomicExch(a.err, 4);
            return;
        }
    } else if (producer) {
        for (int j = 0; j < kLltStages && j < nj; ++j) issue(j);
    }
    for (int i = tid; i < npc; i += kLltThreads) s_y[i] = col0 + i < a.n ? a.y32[col0 + i] : 0.f;
    cluster.sync();

    float gs[RPT][EPC], gc[RPT][EPC];
#pragma unroll
    for (int k = 0; k < RPT; ++k)
#pragma unroll
        for (int e = 0; e < EPC; ++e) gs[k][e] = gc[k][e] = 0.f;

    if (warp == kLltConsumerWarps) {
        if (lane == 0) {
            bool bail = false;
            for (int j = kLltStages; j < nj; ++j) {
                const int s = j % kLltStages;
                if (!umma::mbar_wait(empty0 + 8 * s, (uint32_t)(j / kLltStages - 1) & 1u,
                                     bail ? kLltBailNs : kLltWaitNs)) {
                    atomicExch(a.err, 3);
                    bail = true;
                }
                issue(j);
            }
            for (int j = nj - kLltStages < 0 ? 0 : nj - kLltStages; j < nj; ++j)
                if (!umma::mbar_wait(full0 + 8 * (j % kLltStages), (uint32_t)(j / kLltStages) & 1u, kLltWaitNs))
                    atomicExch(a.err, 4);
        }
        __syncwarp();
    } else {
        bool bail = false;
        for (int j = 0; j < nj; ++j) {
            const int s = j % kLltStages, q = j % kLltSlots;
            if (!umma::mbar_wait(full0 + 8 * s, (uint32_t)(j / kLltStages) & 1u, bail ? kLltBailNs : kLltWaitNs)) {
                atomicExch(a.err, 1);
                bail = true;
            }
            const uint8_t *sb = sm + (size_t)s * L.stage;
            // Phase A.
            {
                float acc[RW];
#pragma unroll
                for (int r = 0; r < RW; ++r) acc[r] = 0.f;
                const int w0 = (warp % NGR) * RW, h = warp / NGR;
#pragma unroll 2
                for (int c = h * 32 + lane; c < nch; c += 32 * WPR) {
                    const int off = (c / CPB) * BOXB + (c % CPB) * 16;
                    float yv[EPC];
#pragma unroll
                    for (int e = 0; e < EPC; e += 4) {
                        const float4 q4 = *reinterpret_cast<const float4 *>(s_y + c * EPC + e);
                        yv[e] = q4.x;
                        yv[e + 1] = q4.y;
                        yv[e + 2] = q4.z;
                        yv[e + 3] = q4.w;
                    }
#pragma unroll
                    for (int r = 0; r < RW; ++r) {
                        const uint4 u =
                            *reinterpret_cast<const uint4 *>(sb + off + (w0 + r) * (kLltBoxCols * ES));
                        float f[EPC];
                        S::unpack(u, f);
#pragma unroll
                        for (int e = 0; e < EPC; ++e) acc[r] = fmaf(f[e], yv[e], acc[r]);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                    for (int r = 0; r < RW; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
                if (lane < C) {
                    const uint32_t local = slots_u32 + (uint32_t)(((q * C + rank) * NP + warp * RW) * 4);
                    const uint32_t rdst = llt::mapa(local, (uint32_t)lane), rbar = llt::mapa(xchg0 + 8 * q, (uint32_t)lane);
                    if constexpr (RW == 2) {
                        llt::st_async_v2(rdst, acc[0], acc[1], rbar);
                    } else {
#pragma unroll
                        for (int v = 0; v < RW; v += 4)
                            llt::st_async_v4(llt::mapa(local + (uint32_t)(4 * v), (uint32_t)lane),
                                             make_float4(acc[v], acc[v + 1], acc[v + 2], acc[v + 3]), rbar);
                    }
                }
            }
            // Receive: z_b[w] = sum over ranks and the row's warps, fixed order.
            float *zc = s_zc + (j & 1) * W;
            if (tid < W) {
                if (!llt::wait_cluster(xchg0 + 8 * q, (uint32_t)(j / kLltSlots) & 1u, bail ? kLltBailNs : kLltWaitNs)) {
                    atomicExch(a.err, 2);
                    bail = true;
                }
                const float *sl = slots + (size_t)q * C * NP;
                float z = 0.f;
#pragma unroll
                for (int r = 0; r < C; ++r)
#pragma unroll
                    for (int hh = 0; hh < WPR; ++hh) z += sl[r * NP + hh * W + tid];
                zc[tid] = z;
                const int zcol = (cid + j * a.G) * W + tid;
                if (a.z != nullptr && rank == 0 && zcol < a.T) a.z[zcol] = z;
                if (tid == 0 && j + kLltSlots < nj) umma::mbar_arrive_expect_tx(xchg0 + 8 * q, xbytes);
            }
            llt::bar_consumers();
            // Phase B: one thread per 16-byte column chunk, all W rows of the block.
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const int c = tid + k * kLltConsumers;
                if (c < nch) {
                    const int off = (c / CPB) * BOXB + (c % CPB) * 16;
                    float d[EPC];
#pragma unroll
                    for (int e = 0; e < EPC; ++e) d[e] = 0.f;
#pragma unroll
                    for (int w = 0; w < W; ++w) {
                        const uint4 u = *reinterpret_cast<const uint4 *>(sb + off + w * (kLltBoxCols * ES));
                        float f[EPC];
                        S::unpack(u, f);
                        const float zw = zc[w];
#pragma unroll
                        for (int e = 0; e < EPC; ++e) d[e] = fmaf(f[e], zw, d[e]);
                    }
#pragma unroll
                    for (int e = 0; e < EPC; ++e) {             // compensated running sums over blocks
                        const float yk = d[e] - gc[k][e];
                        const float tk = gs[k][e] + yk;
                        gc[k][e] = (tk - gs[k][e]) - yk;
                        gs[k][e] = tk;
                    }
                }
            }
            __syncwarp();
            if (lane == 0) llt::mbar_arrive(empty0 + 8 * s);
        }
        // Per-cluster partial of g for this CTA's asset columns.
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int c = tid + k * kLltConsumers;
            if (c < nch) {
#pragma unroll
                for (int e = 0; e < EPC; ++e) {
                    const int col = col0 + c * EPC + e;
                    if (col < a.n) a.gpart[(size_t)cid * a.n + col] = gs[k][e] - gc[k][e];
                }
            }
        }
    }
    llt_final_reduce(a, cid, rank, col0);
    cluster.sync();
}

template <int DT, int C>
__global__ void __launch_bounds__(kLltThreads, 1)
lltt_kernel(const __grid_constant__ CUtensorMap tmM, const LltArgs a) {
    lltt_body<DT, C, false>(&tmM, a, (int)(blockIdx.x / C));
}

// Grouped transposed pass: many problems (each its own L^T, n, T, vectors
// and scratch) in one launch.  Cluster c works on problem clusters[c].x as
// its cluster clusters[c].y of that problem's G.  Descriptors keep the
// tensor map's alignment (at least the 64 bytes TMA requires; the
// workspace places the array on a 256-byte boundary) and are written by the
// host before the launch.
struct LltGroup {
    CUtensorMap map;
    LltArgs a;
};
static_assert(alignof(LltGroup) >= 64 && sizeof(LltGroup) % 64 == 0, "tensor-map descriptors must stay aligned");

template <int DT, int C>
__global__ void __launch_bounds__(kLltThreads, 1)
lltt_grouped_kernel(const LltGroup *__restrict__ groups, const int2 *__restrict__ clusters) {
    const int2 w = clusters[blockIdx.x / C];
    const LltGroup *gd = groups + w.x;
    const LltArgs a = gd->a;
    lltt_body<DT, C, true>(&gd->map, a, w.y);
}

// ------------------------------------------------------------------ host
constexpr size_t kLltSmemCap = 221 * 1024;

// Geometry for one (cluster size C, row-segment bytes RB) choice.
inline bool llt_shape(int64_t n, int64_t T, int esize, int C, int RB, LltPlan *p) {
    const int W = RB / esize;
    const int64_t rpc0 = (n + C - 1) / C;
    const int nbox = (int)((rpc0 + 255) / 256);
    const int box_rows = (int)(((rpc0 + nbox - 1) / nbox + 7) / 8 * 8);
    const int rpc = nbox * box_rows;
    if (rpc > kLltRowsPerThread * kLltConsumers) return false;
    const size_t smem = llt_smem_layout(rpc, RB, W, C).total;
    if (smem > kLltSmemCap) return false;
    p->C = C;
    p->RB = RB;
    p->rpc = rpc;
    p->box_rows = box_rows;
    p->nbox = nbox;
    p->nb = (int)((T + W - 1) / W);
    p->smem = smem;
    return true;
}

// Geometry of the transposed-layout pass for cluster size C: npc asset
// columns per CTA (a multiple of kLltBoxCols), boxes per stage, blocks of
// W = 32 / esize periods.
inline bool lltt_shape(int64_t n, int64_t T, int esize, int C, LltPlan *p) {
    const int64_t npc = ((n + C - 1) / C + kLltBoxCols - 1) / kLltBoxCols * kLltBoxCols;
    if (npc * esize / 16 > (esize == 4 ? 2 : 1) * kLltConsumers) return false;
    const size_t smem = lltt_smem_layout((int)npc, C).total;
    if (smem > kLltSmemCap) return false;
    const int W = 32 / esize;
    p->C = C;
    p->RB = 0;                                  // marks the transposed layout
    p->rpc = (int)npc;
    p->box_rows = W;
    p->nbox = (int)(npc / kLltBoxCols);
    p->nb = (int)((T + W - 1) / W);
    p->smem = smem;
    return true;
}

// The (C, RB) pairs the library instantiates, in order of preference: the
// widest row segment that fits two stages (TMA row requests of 128 bytes
// stream near the copy peak, 32-byte ones far below it), then the smaller
// cluster (a cluster of 2 is a TPC pair, so clusters of 2 tile every SM;
// clusters of 8 leave SMs of each GPC idle).
constexpr int kLltShapes[][2] = {{2, 128}, {4, 128}, {2, 64}, {4, 64}, {2, 32}, {8, 128}};
constexpr int kLltNumShapes = (int)(sizeof(kLltShapes) / sizeof(kLltShapes[0]));

// 2-D tensor map over L for the fused pass: box = RB bytes of columns x box_rows rows,
// RB-byte swizzle (RB = 32, 64 or 128).
inline int make_map_llt(CUtensorMap *map, int dt, const void *base, int64_t n, int64_t T, int64_t ld, int box_rows,
                        int RB) {
    auto enc = tensor_map_encoder();
    if (enc == nullptr) return record_message(MV_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    const int es = dtype_size(dt);
    const CUtensorMapDataType ty = dt == MV_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : dt == MV_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                   : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    const CUtensorMapSwizzle sw = RB == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                                  : RB == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                             : CU_TENSOR_MAP_SWIZZLE_128B;
    cuuint64_t dims[2] = {(cuuint64_t)T, (cuuint64_t)n};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * es)};
    cuuint32_t box[2] = {(cuuint32_t)(RB / es), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, ty, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        char msg[128];
        snprintf(msg, sizeof(msg), "cuTensorMapEncodeTiled (fused pass) failed (%d)", (int)r);
        return record_message(MV_ERR_CUDA, msg);
    }
    return MV_OK;
}

// 2-D tensor map over M = L^T (T x n, leading dim ld) for the transposed pass:
// box = kLltBoxCols assets x W periods, no swizzle.
inline int make_map_lltt(CUtensorMap *map, int dt, const void *base, int64_t n, int64_t T, int64_t ld, int W) {
    auto enc = tensor_map_encoder();
    if (enc == nullptr) return record_message(MV_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    const int es = dtype_size(dt);
    const CUtensorMapDataType ty = dt == MV_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : dt == MV_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                   : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)T};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * es)};
    cuuint32_t box[2] = {(cuuint32_t)kLltBoxCols, (cuuint32_t)W};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, ty, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        char msg[128];
        snprintf(msg, sizeof(msg), "cuTensorMapEncodeTiled (transposed pass) failed (%d)", (int)r);
        return record_message(MV_ERR_CUDA, msg);
    }
    return MV_OK;
}

}  // namespace mv
