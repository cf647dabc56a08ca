// usp_fused.cu -- placeholder translation unit for the fused FP32 pipeline.
#include "usp_internal.cuh"
