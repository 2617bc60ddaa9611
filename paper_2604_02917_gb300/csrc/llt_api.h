// Host interface of the fused single-pass Gram product g = L L^T y
// (llt.cuh holds the kernel; llt_host.cu and llt_<dtype>.cu instantiate it).
// Internal to libmv, not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace mv {

constexpr int kLltMaxCluster = 8;          // largest cluster the pass uses
constexpr int kLltMaxClusters = 128;       // clusters per launch (upper bound)
constexpr int kLltFan = 8;                 // clusters per group of the final reduction
constexpr int kLltMaxGroups = kLltMaxClusters / kLltFan;
constexpr int64_t kLltMinN = 1024, kLltMinT = 4096;

struct LltPlan {
    bool ok;
    bool tn;                   // transposed layout (L^T stored T x n)
    int C, RB;                 // cluster size, bytes of one row per column block (NT)
    int rpc, box_rows, nbox;   // rows per CTA, TMA box rows, boxes per stage
    int nb, G;                 // column blocks, clusters launched
    size_t smem;               // dynamic shared memory per CTA
};

// Scratch of the pass inside a caller workspace (offsets from its base).
struct LltScratch {
    float *gpart;              // [kLltMaxClusters x n]
    double *gq;                // [kLltMaxGroups x n]
    unsigned *tickets;         // zero between launches
    int *err;                  // error word
};
size_t llt_scratch_bytes(int64_t n);
LltScratch llt_scratch(void *base, int64_t n);
size_t llt_ticket_bytes();     // bytes of sc.tickets to zero before the first launch

// Geometry for an n x T factor of dtype dt (ok = false where the pass does
// not apply).  with_device = false skips the device query and only decides
// whether a shape exists (workspace sizing must not depend on the device).
// MV_LLT_SHAPE="C,RB" in the environment forces one shape (tuning).
LltPlan llt_plan(int dt, int64_t n, int64_t T, bool with_device, bool tn = false);

// Enqueues g = L L^T y (row-scaled; FP8 y32 pre-multiplied by the scale) on
// stream s; capturable.  done (nullable): the launch returns at once if *done.
// z (nullable): also writes z = L^T y (T floats), which the pass forms anyway.
// For a transposed plan, L points at L^T (T x n, leading dim ld).
// pdl (transposed plans): launch as a programmatic dependent of the previous
// kernel, whose early trigger lets the pass stream its first blocks of L
// while that kernel finishes.  Only where no predecessor since the last
// ordinary launch writes L.
int llt_launch(const LltPlan &lp, int dt, const void *L, int64_t n, int64_t T, int64_t ld, const float *y32,
               const float *row_scale, const LltScratch &sc, const int *done, double *g, float *g32, cudaStream_t s,
               float *z = nullptr, bool pdl = false);

// ---- grouped transposed pass: many problems (each L^T stored T x n) in one
// launch per cluster size; the batch solve's product.
struct LltGroupPlan {
    int C;                     // cluster size (the transposed plan's)
    int G;                     // clusters of this problem
    int npc, nb;               // asset columns per CTA, column blocks
    size_t smem;               // dynamic shared memory per CTA
    double est_us;             // estimated time of one cluster (longest first)
};
// Geometry of one problem (ok = false where no cluster size fits n).
bool llt_group_plan(int dt, int64_t n, int64_t T, LltGroupPlan *gp);
size_t llt_group_bytes();                                   // one descriptor (64-byte multiple)
size_t llt_group_scratch_bytes(int64_t n, int G);           // per-problem partials and tickets
size_t llt_group_ticket_offset(int64_t n, int G);           // tickets inside that scratch
// Writes the descriptor of one problem (tensor map + arguments) into host
// memory dst (llt_group_bytes() bytes).  done, z: nullable as in llt_launch.
// early: the descriptor is for launches with pdl (see llt_launch).
int llt_group_write(void *dst, const LltGroupPlan &gp, int dt, const void *L, int64_t n, int64_t T, int64_t ld,
                    const float *y32, const float *row_scale, void *scratch, int *err, const int *done, double *g,
                    float *g32, float *z, bool early = false);
// One grouped launch over nclusters clusters of size C (descriptors and the
// (problem, cluster) list in device memory); pdl as in llt_launch, with
// descriptors written with early = true.
cudaError_t llt_launch_grouped(int dt, int C, int nclusters, size_t smem, const void *groups, const int2 *clusters,
                               cudaStream_t s, bool pdl = false);

// Per-dtype entry points (llt_<dtype>.cu).
int llt_max_clusters_f32(int C, int RB, size_t smem);
int llt_max_clusters_bf16(int C, int RB, size_t smem);
int llt_max_clusters_fp8(int C, int RB, size_t smem);
struct LltArgs;
cudaError_t llt_launch_f32(int C, int RB, int G, size_t smem, const void *map, const LltArgs &a, cudaStream_t s);
cudaError_t llt_launch_bf16(int C, int RB, int G, size_t smem, const void *map, const LltArgs &a, cudaStream_t s);
cudaError_t llt_launch_fp8(int C, int RB, int G, size_t smem, const void *map, const LltArgs &a, cudaStream_t s);
int llt_max_clusters_tn_f32(int C, size_t smem);
int llt_max_clusters_tn_bf16(int C, size_t smem);
int llt_max_clusters_tn_fp8(int C, size_t smem);
cudaError_t llt_launch_tn_f32(int C, int G, size_t smem, const void *map, const LltArgs &a, cudaStream_t s);
cudaError_t llt_launch_tn_bf16(int C, int G, size_t smem, const void *map, const LltArgs &a, cudaStream_t s);
cudaError_t llt_launch_tn_fp8(int C, int G, size_t smem, const void *map, const LltArgs &a, cudaStream_t s);
cudaError_t llt_launch_grouped_f32(int C, int nclusters, size_t smem, const void *groups, const int2 *clusters,
                                   cudaStream_t s, bool pdl);
cudaError_t llt_launch_grouped_bf16(int C, int nclusters, size_t smem, const void *groups, const int2 *clusters,
                                    cudaStream_t s, bool pdl);
cudaError_t llt_launch_grouped_fp8(int C, int nclusters, size_t smem, const void *groups, const int2 *clusters,
                                   cudaStream_t s, bool pdl);

}  // namespace mv
