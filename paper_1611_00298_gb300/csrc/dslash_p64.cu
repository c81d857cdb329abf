// Fused dslash kernels for the FP64 storage precision (see dslash_impl.cuh).
#include "dslash_impl.cuh"

DSL_DEFINE(p64, P64, P64)
