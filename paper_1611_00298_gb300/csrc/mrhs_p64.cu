// Multi-system solver kernels for the FP64 storage precision (see mrhs.cuh).
#include "mrhs.cuh"

MR_DEFINE(p64, P64, P64)
