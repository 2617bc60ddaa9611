// Instantiates the fused pass for one element type (MV_LLT_DT, MV_LLT_SUFFIX):
// kernel attributes, the occupancy query and the launch for every shape.
#pragma once

#include "llt.cuh"

#define MV_LLT_CAT2(a, b) a##b
#define MV_LLT_CAT(a, b) MV_LLT_CAT2(a, b)

namespace mv {
namespace {

template <int C, int RB>
int attrs() {
    static int st = -1;
    if (st < 0) {
        const int smem = (int)(kLltSmemCap + 256);
        st = (cudaFuncSetAttribute(llt_kernel<MV_LLT_DT, C, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
                  cudaSuccess &&
              cudaFuncSetAttribute(llt_kernel<MV_LLT_DT, C, RB>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                  cudaSuccess)
                 ? MV_OK
                 : MV_ERR_CUDA;
        if (st != MV_OK) (void)cudaGetLastError();
    }
    return st;
}

// attr: room for two attributes.  pdl: launch as a programmatic dependent
// of the previous kernel in the stream (the kernel's early-load path).
cudaLaunchConfig_t config(int C, int G, size_t smem, cudaStream_t s, cudaLaunchAttribute *attr, bool pdl = false) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(C * G));
    cfg.blockDim = dim3(kLltThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (pdl) {
        attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.numAttrs = 2;
    }
    return cfg;
}

template <int C, int RB>
int max_clusters(size_t smem) {
    if (attrs<C, RB>() != MV_OK) return 0;
    cudaLaunchAttribute attr[2];
    const cudaLaunchConfig_t cfg = config(C, kLltMaxClusters, smem, nullptr, attr);
    int num = 0;
    if (cudaOccupancyMaxActiveClusters(&num, llt_kernel<MV_LLT_DT, C, RB>, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return num;
}

template <int C, int RB>
cudaError_t launch(int G, size_t smem, const void *map, const LltArgs &a, cudaStream_t s) {
    if (attrs<C, RB>() != MV_OK) return cudaErrorInvalidValue;
    cudaLaunchAttribute attr[2];
    const cudaLaunchConfig_t cfg = config(C, G, smem, s, attr);
    return cudaLaunchKernelEx(&cfg, llt_kernel<MV_LLT_DT, C, RB>, *reinterpret_cast<const CUtensorMap *>(map), a);
}

template <int C>
int attrs_tn() {
    static int st = -1;
    if (st < 0) {
        const int smem = (int)(kLltSmemCap + 256);
        st = (cudaFuncSetAttribute(lltt_kernel<MV_LLT_DT, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
                  cudaSuccess &&
              cudaFuncSetAttribute(lltt_kernel<MV_LLT_DT, C>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                  cudaSuccess)
                 ? MV_OK
                 : MV_ERR_CUDA;
        if (st != MV_OK) (void)cudaGetLastError();
    }
    return st;
}

template <int C>
int max_clusters_tn(size_t smem) {
    if (attrs_tn<C>() != MV_OK) return 0;
    cudaLaunchAttribute attr[2];
    const cudaLaunchConfig_t cfg = config(C, kLltMaxClusters, smem, nullptr, attr);
    int num = 0;
    if (cudaOccupancyMaxActiveClusters(&num, lltt_kernel<MV_LLT_DT, C>, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return num;
}

template <int C>
cudaError_t launch_tn(int G, size_t smem, const void *map, const LltArgs &a, cudaStream_t s) {
    if (attrs_tn<C>() != MV_OK) return cudaErrorInvalidValue;
    cudaLaunchAttribute attr[2];
    const cudaLaunchConfig_t cfg = config(C, G, smem, s, attr, a.early != 0);
    return cudaLaunchKernelEx(&cfg, lltt_kernel<MV_LLT_DT, C>, *reinterpret_cast<const CUtensorMap *>(map), a);
}

template <int C>
int attrs_grouped() {
    static int st = -1;
    if (st < 0) {
        const int smem = (int)(kLltSmemCap + 256);
        st = (cudaFuncSetAttribute(lltt_grouped_kernel<MV_LLT_DT, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   smem) == cudaSuccess &&
              cudaFuncSetAttribute(lltt_grouped_kernel<MV_LLT_DT, C>, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                   1) == cudaSuccess)
                 ? MV_OK
                 : MV_ERR_CUDA;
        if (st != MV_OK) (void)cudaGetLastError();
    }
    return st;
}

template <int C>
cudaError_t launch_grouped(int nclusters, size_t smem, const void *groups, const int2 *clusters, cudaStream_t s,
                           bool pdl) {
    if (attrs_grouped<C>() != MV_OK) return cudaErrorInvalidValue;
    cudaLaunchAttribute attr[2];
    const cudaLaunchConfig_t cfg = config(C, nclusters, smem, s, attr, pdl);
    return cudaLaunchKernelEx(&cfg, lltt_grouped_kernel<MV_LLT_DT, C>, reinterpret_cast<const LltGroup *>(groups),
                              clusters);
}

}  // namespace

// The instantiated shapes (kLltShapes).
#define MV_LLT_SWITCH(C, RB, F, ...)                                     \
    if (C == 2 && RB == 128) return F<2, 128>(__VA_ARGS__);              \
    if (C == 4 && RB == 128) return F<4, 128>(__VA_ARGS__);              \
    if (C == 2 && RB == 64) return F<2, 64>(__VA_ARGS__);                \
    if (C == 4 && RB == 64) return F<4, 64>(__VA_ARGS__);                \
    if (C == 2 && RB == 32) return F<2, 32>(__VA_ARGS__);                \
    if (C == 8 && RB == 128) return F<8, 128>(__VA_ARGS__);

int MV_LLT_CAT(llt_max_clusters_, MV_LLT_SUFFIX)(int C, int RB, size_t smem) {
    MV_LLT_SWITCH(C, RB, max_clusters, smem)
    return 0;
}

cudaError_t MV_LLT_CAT(llt_launch_, MV_LLT_SUFFIX)(int C, int RB, int G, size_t smem, const void *map,
                                                    const LltArgs &a, cudaStream_t s) {
    MV_LLT_SWITCH(C, RB, launch, G, smem, map, a, s)
    return cudaErrorInvalidValue;
}

#define MV_LLT_SWITCH_TN(C, F, ...)                   \
    if (C == 1) return F<1>(__VA_ARGS__);             \
    if (C == 2) return F<2>(__VA_ARGS__);             \
    if (C == 4) return F<4>(__VA_ARGS__);             \
    if (C == 8) return F<8>(__VA_ARGS__);

int MV_LLT_CAT(llt_max_clusters_tn_, MV_LLT_SUFFIX)(int C, size_t smem) {
    MV_LLT_SWITCH_TN(C, max_clusters_tn, smem)
    return 0;
}

cudaError_t MV_LLT_CAT(llt_launch_tn_, MV_LLT_SUFFIX)(int C, int G, size_t smem, const void *map, const LltArgs &a,
                                                       cudaStream_t s) {
    MV_LLT_SWITCH_TN(C, launch_tn, G, smem, map, a, s)
    return cudaErrorInvalidValue;
}

cudaError_t MV_LLT_CAT(llt_launch_grouped_, MV_LLT_SUFFIX)(int C, int nclusters, size_t smem, const void *groups,
                                                            const int2 *clusters, cudaStream_t s, bool pdl) {
    MV_LLT_SWITCH_TN(C, launch_grouped, nclusters, smem, groups, clusters, s, pdl)
    return cudaErrorInvalidValue;
}

}  // namespace mv
