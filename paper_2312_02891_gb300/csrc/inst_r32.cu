// inst_r32.cu - real shifts, float32 basis and sweeps, float64 outer iteration.
#define SYLV_SUFFIX r32
#define SYLV_T double
#define SYLV_S float
#define SYLV_C float
#include "inst.cuh"
