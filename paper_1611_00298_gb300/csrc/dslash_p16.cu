// Fused dslash kernels for the FP16 storage precision (see dslash_impl.cuh).
#include "dslash_impl.cuh"

DSL_DEFINE(p16, P16, P32)
