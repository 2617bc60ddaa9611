// Host side of the fused single-pass Gram product (llt.cuh): shape choice,
// device occupancy query, tensor map and launch.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>

#include <algorithm>
#include <mutex>
#include <unordered_map>

#include "llt.cuh"

namespace mv {

size_t llt_ticket_bytes() { return 4 * (size_t)kLltMaxCluster * (kLltMaxGroups + 1); }

size_t llt_scratch_bytes(int64_t n) {
    return align_up(4 * (size_t)n * kLltMaxClusters, 256) + align_up(8 * (size_t)n * kLltMaxGroups, 256) +
           align_up(llt_ticket_bytes(), 256) + 256;
}

LltScratch llt_scratch(void *base, int64_t n) {
    char *p = reinterpret_cast<char *>(base);
    LltScratch sc;
    sc.gpart = reinterpret_cast<float *>(p);
    p += align_up(4 * (size_t)n * kLltMaxClusters, 256);
    sc.gq = reinterpret_cast<double *>(p);
    p += align_up(8 * (size_t)n * kLltMaxGroups, 256);
    sc.tickets = reinterpret_cast<unsigned *>(p);
    p += align_up(llt_ticket_bytes(), 256);
    sc.err = reinterpret_cast<int *>(p);
    return sc;
}

static int max_clusters(int dt, int C, int RB, size_t smem) {   // RB = 0: transposed-layout kernel
    static std::mutex mu;
    static std::unordered_map<uint64_t, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    const uint64_t key = ((uint64_t)dev << 56) ^ ((uint64_t)dt << 48) ^ ((uint64_t)C << 40) ^ ((uint64_t)RB << 32) ^
                         (uint64_t)smem;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int v;
    if (RB == 0)
        v = dt == MV_F32 ? llt_max_clusters_tn_f32(C, smem)
            : dt == MV_BF16 ? llt_max_clusters_tn_bf16(C, smem)
                            : llt_max_clusters_tn_fp8(C, smem);
    else
        v = dt == MV_F32 ? llt_max_clusters_f32(C, RB, smem)
            : dt == MV_BF16 ? llt_max_clusters_bf16(C, RB, smem)
                            : llt_max_clusters_fp8(C, RB, smem);
    v = std::min(v, kLltMaxClusters);
    cache.emplace(key, v);
    return v;
}

// Transposed layout: the smallest cluster (1, 2, 4 or 8 CTAs) whose asset
// share fits two stages.
static LltPlan plan_tn(int dt, int64_t n, int64_t T, bool with_device) {
    LltPlan p{};
    p.ok = false;
    const int es = dtype_size(dt);
    for (int C = 1; C <= kLltMaxCluster; C *= 2) {
        LltPlan q{};
        if (!lltt_shape(n, T, es, C, &q)) continue;
        q.tn = true;
        if (!with_device) {
            q.ok = true;
            q.G = 1;
            return q;
        }
        const int mc = max_clusters(dt, C, 0, q.smem);
        if (mc < 1) continue;
        q.G = std::max(1, std::min(mc, q.nb));
        q.ok = true;
        return q;
    }
    return p;
}

LltPlan llt_plan(int dt, int64_t n, int64_t T, bool with_device, bool tn) {
    LltPlan p{};
    p.ok = false;
    const int es = dtype_size(dt);
    if (es == 0 || n < kLltMinN || T < kLltMinT) return p;
    if (tn) return plan_tn(dt, n, T, with_device);
    int fC = 0, fRB = 0;
    if (const char *env = getenv("MV_LLT_SHAPE")) {
        if (sscanf(env, "%d,%d", &fC, &fRB) != 2) fC = fRB = 0;
    }
    for (int pass = 0; pass < 2; ++pass) {
        for (int i = 0; i < kLltNumShapes; ++i) {
            const int C = kLltShapes[i][0], RB = kLltShapes[i][1];
            if (pass == 0 && fC != 0 && (C != fC || RB != fRB)) continue;
            LltPlan q{};
            if (!llt_shape(n, T, es, C, RB, &q)) continue;
            if (!with_device) {
                q.ok = true;
                q.G = 1;
                return q;
            }
            const int mc = max_clusters(dt, C, RB, q.smem);
            if (mc < 1) continue;
            q.G = std::max(1, std::min(mc, q.nb));
            q.ok = true;
            return q;
        }
        if (fC == 0) break;                  // no override: one pass over the preference list
    }
    return p;
}

int llt_launch(const LltPlan &lp, int dt, const void *L, int64_t n, int64_t T, int64_t ld, const float *y32,
               const float *row_scale, const LltScratch &sc, const int *done, double *g, float *g32, cudaStream_t s,
               float *z, bool pdl) {
    if (!lp.ok) return record_message(MV_ERR_UNSUPPORTED, "fused pass: no cluster shape fits this n and T");
    CUtensorMap map;
    if (lp.tn)
        MV_TRY(make_map_lltt(&map, dt, L, n, T, ld, lp.box_rows));
    else
        MV_TRY(make_map_llt(&map, dt, L, n, T, ld, lp.box_rows, lp.RB));
    LltArgs a;
    a.y32 = y32;
    a.row_scale = row_scale;
    a.gpart = sc.gpart;
    a.gq = sc.gq;
    a.g = g;
    a.g32 = g32;
    a.z = z;
    a.tick1 = sc.tickets;
    a.tick2 = sc.tickets + (size_t)kLltMaxCluster * kLltMaxGroups;
    a.err = sc.err;
    a.done = done;
    a.n = (int)n;
    a.T = (int)T;
    a.rpc = lp.rpc;
    a.box_rows = lp.box_rows;
    a.nbox = lp.nbox;
    a.nb = lp.nb;
    a.G = lp.G;
    a.early = (pdl && lp.tn) ? 1 : 0;
    cudaError_t e;
    if (lp.tn)
        e = dt == MV_F32    ? llt_launch_tn_f32(lp.C, lp.G, lp.smem, &map, a, s)
            : dt == MV_BF16 ? llt_launch_tn_bf16(lp.C, lp.G, lp.smem, &map, a, s)
                            : llt_launch_tn_fp8(lp.C, lp.G, lp.smem, &map, a, s);
    else
        e = dt == MV_F32    ? llt_launch_f32(lp.C, lp.RB, lp.G, lp.smem, &map, a, s)
            : dt == MV_BF16 ? llt_launch_bf16(lp.C, lp.RB, lp.G, lp.smem, &map, a, s)
                            : llt_launch_fp8(lp.C, lp.RB, lp.G, lp.smem, &map, a, s);
    if (e != cudaSuccess) return record_cuda_error(e, "fused L L^T pass launch", __FILE__, __LINE__);
    return MV_OK;
}

// ------------------------------------------------------------------ grouped transposed pass
// Clusters per problem: about 8 MB of the factor and at most 64 column
// blocks each, so no cluster runs long enough to leave a tail, and the fixed
// cost of a cluster (two stage fills, the partial of g) stays a few percent.
constexpr double kGroupBytesPerCluster = 8.0 * 1024 * 1024;
constexpr int kGroupMaxBlocks = 64;

bool llt_group_plan(int dt, int64_t n, int64_t T, LltGroupPlan *gp) {
    const int es = dtype_size(dt);
    if (es == 0 || n < 1 || T < 1) return false;
    for (int C = 1; C <= kLltMaxCluster; C *= 2) {
        LltPlan q{};
        if (!lltt_shape(n, T, es, C, &q)) continue;
        const double bytes = (double)n * (double)T * es;
        int64_t G = std::max<int64_t>((int64_t)std::ceil(bytes / kGroupBytesPerCluster),
                                      (q.nb + kGroupMaxBlocks - 1) / kGroupMaxBlocks);
        G = std::max<int64_t>(1, std::min<int64_t>(G, std::min<int64_t>(kLltMaxClusters, q.nb)));
        gp->C = C;
        gp->G = (int)G;
        gp->npc = q.rpc;
        gp->nb = q.nb;
        gp->smem = q.smem;
        // a block's stage is 32 bytes x npc per CTA; below ~40 KB a block costs
        // about a microsecond of latency whatever its size
        const int64_t per = (q.nb + G - 1) / G;
        gp->est_us = (double)per * std::max(1.0, 32.0 * q.rpc / 40000.0);
        return true;
    }
    return false;
}

size_t llt_group_bytes() { return sizeof(LltGroup); }

size_t llt_group_ticket_offset(int64_t n, int G) {
    const int ngrp = (G + kLltFan - 1) / kLltFan;
    return align_up(4 * (size_t)n * G, 256) + align_up(8 * (size_t)n * ngrp, 256);
}

size_t llt_group_scratch_bytes(int64_t n, int G) { return llt_group_ticket_offset(n, G) + align_up(llt_ticket_bytes(), 256); }

int llt_group_write(void *dst, const LltGroupPlan &gp, int dt, const void *L, int64_t n, int64_t T, int64_t ld,
                    const float *y32, const float *row_scale, void *scratch, int *err, const int *done, double *g,
                    float *g32, float *z, bool early) {
    LltGroup d;
    memset(&d, 0, sizeof(d));
    MV_TRY(make_map_lltt(&d.map, dt, L, n, T, ld, 32 / dtype_size(dt)));
    char *sp = reinterpret_cast<char *>(scratch);
    LltArgs &a = d.a;
    a.y32 = y32;
    a.row_scale = row_scale;
    a.gpart = reinterpret_cast<float *>(sp);
    a.gq = reinterpret_cast<double *>(sp + align_up(4 * (size_t)n * gp.G, 256));
    unsigned *tickets = reinterpret_cast<unsigned *>(sp + llt_group_ticket_offset(n, gp.G));
    a.tick1 = tickets;
    a.tick2 = tickets + (size_t)kLltMaxCluster * kLltMaxGroups;
    a.g = g;
    a.g32 = g32;
    a.z = z;
    a.err = err;
    a.done = done;
    a.n = (int)n;
    a.T = (int)T;
    a.rpc = gp.npc;
    a.box_rows = 32 / dtype_size(dt);
    a.nbox = gp.npc / kLltBoxCols;
    a.nb = gp.nb;
    a.G = gp.G;
    a.early = early ? 1 : 0;
    memcpy(dst, &d, sizeof(d));
    return MV_OK;
}

cudaError_t llt_launch_grouped(int dt, int C, int nclusters, size_t smem, const void *groups, const int2 *clusters,
                               cudaStream_t s, bool pdl) {
    if (nclusters < 1) return cudaSuccess;
    if (dt == MV_F32) return llt_launch_grouped_f32(C, nclusters, smem, groups, clusters, s, pdl);
    if (dt == MV_BF16) return llt_launch_grouped_bf16(C, nclusters, smem, groups, clusters, s, pdl);
    return llt_launch_grouped_fp8(C, nclusters, smem, groups, clusters, s, pdl);
}

}  // namespace mv
