// Multi-right-hand-side solver kernels (mrhs.cuh) and the batched group
// solver built on them (batch.cu).
#pragma once
#include "internal.h"

// systems iterated together in one launch
#define MR_MAX 16

// Per-system field pointers of one multi-system launch (kernel argument).
// dslash: in -> out (+ b y); local5: out2 = x updated in place with y = z,
// out = block output; xp update: x = out2, p = out, s = in.
struct MRPtrs {
    const void* in[MR_MAX];
    void* out[MR_MAX];
    void* out2[MR_MAX];
    const void* y[MR_MAX];
    double* red[MR_MAX];
};

// shared-memory layout of the multi-system kernels: Op5 records, the
// rank-one vectors (4 Ls per system, FP32 or FP64), per-system partial sums
// and last-block flags, then the 5D columns
__host__ __device__ inline size_t mr_round16(size_t n) { return (n + 15) & ~size_t(15); }
__host__ __device__ inline size_t mr_ops_bytes(int RB) { return mr_round16((size_t)RB * sizeof(Op5)); }
__host__ __device__ inline size_t mr_wv_bytes(int RB, int Ls) { return mr_round16((size_t)RB * 4 * Ls * sizeof(double)); }
__host__ __device__ inline size_t mr_head_bytes(int RB, int Ls) {
    return mr_ops_bytes(RB) + mr_wv_bytes(RB, Ls) + mr_round16((size_t)RB * (sizeof(double) + sizeof(unsigned)));
}

// Launchers per storage precision (mrhs_p64.cu, mrhs_p32.cu, mrhs_p16.cu).
// ops: device array of nr finalised Op5 (op_finalize), one per system.
//   dslash:  out_r = a_out (-1/2) B_r hop(in_r) + b_in y_r, |out_r|^2 -> red_r[slot] (slot >= 0)
//   local5:  x_r -= alpha_r z_r (CG scalars of system r at iteration it), |x_r|^2 -> red_r[slot],
//            out_r = B_r x_r
//   xp:      x_r += alpha_r p_r, p_r = s_r + beta_r p_r
#define MR_DECLARE(NAME)                                                                                     \
    void mr_dslash_##NAME(const eofa_ctx* ctx, int par, int dag, const MRPtrs& a, const Op5* ops, int nr,   \
                          bool hasop, double a_out, double b_in, int slot, cudaStream_t st);               \
    void mr_local5_##NAME(const eofa_ctx* ctx, const MRPtrs& a, const Op5* ops, int nr, int it, int slot,   \
                          cudaStream_t st);                                                                 \
    void mr_xp_##NAME(const eofa_ctx* ctx, const MRPtrs& a, int nr, int it, cudaStream_t st);
MR_DECLARE(p64)
MR_DECLARE(p32)
MR_DECLARE(p16)
