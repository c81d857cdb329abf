// Fused dslash kernels for the FP32 storage precision (see dslash_impl.cuh).
#include "dslash_impl.cuh"

DSL_DEFINE(p32, P32, P32)
