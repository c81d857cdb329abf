// Multi-system solver kernels for the FP16 storage precision (see mrhs.cuh).
#include "mrhs.cuh"

MR_DEFINE(p16, P16, P32)
