// Fused single-pass Gram product, bf16 factor (see llt.cuh).
#define MV_LLT_DT MV_BF16
#define MV_LLT_SUFFIX bf16
#include "llt_inst.cuh"
