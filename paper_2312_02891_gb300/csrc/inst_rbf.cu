// inst_rbf.cu - real shifts, bfloat16 basis, float32 sweeps, float64 outer iteration.
#define SYLV_SUFFIX rbf
#define SYLV_T double
#define SYLV_S bf16
#define SYLV_C float
#include "inst.cuh"
