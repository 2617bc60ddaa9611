// Fused single-pass Gram product, fp8 factor (see llt.cuh).
#define MV_LLT_DT MV_FP8_E4M3
#define MV_LLT_SUFFIX fp8
#include "llt_inst.cuh"
