// Multi-system solver kernels for the FP32 storage precision (see mrhs.cuh).
#include "mrhs.cuh"

MR_DEFINE(p32, P32, P32)
