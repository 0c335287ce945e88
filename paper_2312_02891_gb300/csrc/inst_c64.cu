// inst_c64.cu - complex shifts, complex64 basis and sweeps, complex128 outer iteration.
#define SYLV_SUFFIX c64
#define SYLV_T cplx
#define SYLV_S cflt
#define SYLV_C cflt
#include "inst.cuh"
