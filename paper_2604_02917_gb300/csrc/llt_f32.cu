// Fused single-pass Gram product, f32 factor (see llt.cuh).
#define MV_LLT_DT MV_F32
#define MV_LLT_SUFFIX f32
#include "llt_inst.cuh"
