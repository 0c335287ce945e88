// inst_cbf.cu - complex shifts, bfloat16-pair basis, complex64 sweeps, complex128 outer iteration.
#define SYLV_SUFFIX cbf
#define SYLV_T cplx
#define SYLV_S cbf16
#define SYLV_C cflt
#include "inst.cuh"
