// Multi-right-hand-side solver kernels (mrhs.cuh) and the batched group
// solver built on them (batch.cu).
#pragma once
#include "internal.h"

// systems iterated together in one launch
#define MR_MAX 16

// Per-system field pointers of one multi-system launch (kernel argument).
// dslash: in -> out (+ b y), out2 = second output (MODE 1); the in-place
// updates of MODE 2 read and write out and out2.  xp update: x = out2,
// p = out, s = in.
struct MRPtrs {
    const void* in[MR_MAX];
    void* out[MR_MAX];
    void* out2[MR_MAX];
    const void* y[MR_MAX];
    double* red[MR_MAX];
};

// shared-memory layout of the multi-system kernels: two sets of Op5 records
// and rank-one vectors (4 Ls per system, FP32 or FP64), per-system partial
// sums and last-block flags, then the 5D columns
__host__ __device__ inline size_t mr_round16(size_t n) { return (n + 15) & ~size_t(15); }
__host__ __device__ inline size_t mr_ops_bytes(int RB) { return mr_round16((size_t)RB * sizeof(Op5)); }
__host__ __device__ inline size_t mr_wv_bytes(int RB, int Ls) { return mr_round16((size_t)RB * 4 * Ls * sizeof(double)); }
__host__ __device__ inline size_t mr_head_bytes(int RB, int Ls) {
    return 2 * mr_ops_bytes(RB) + 2 * mr_wv_bytes(RB, Ls) +
           mr_round16((size_t)RB * (2 * sizeof(double) + sizeof(unsigned)));
}

// Launchers per storage precision (mrhs_p64.cu, mrhs_p32.cu, mrhs_p16.cu).
// ops, ops2: device arrays of nr finalised Op5 (op_finalize), one per system.
//   dslash, mode 0: out_r = a_out (-1/2) B_r hop(in_r) + b_in y_r, |out_r|^2 -> red_r[slot] (slot >= 0)
//           mode 1: the same, and out2_r = B2_r out_r (B2 from ops2)
//           mode 2: out_r <- out_r - alpha_r (a_out (-1/2) hop(in_r) + b_in y_r) (B = 1), |out_r|^2 ->
//                   red_r[slot]; out2_r <- out2_r - alpha_r y_r, |out2_r|^2 -> red_r[slot2]
//           (alpha_r: system r's CG scalar at iteration it)
//   xp:     x_r += alpha_r p_r, p_r = s_r + beta_r p_r
#define MR_DECLARE(NAME)                                                                                       \
    void mr_dslash_##NAME(const eofa_ctx* ctx, int par, int dag, int mode, const MRPtrs& a, const Op5* ops,   \
                          const Op5* ops2, int nr, bool hasop, double a_out, double b_in, int slot, int it,   \
                          int slot2, cudaStream_t st);                                                        \
    void mr_xp_##NAME(const eofa_ctx* ctx, const MRPtrs& a, int nr, int it, cudaStream_t st);
MR_DECLARE(p64)
MR_DECLARE(p32)
MR_DECLARE(p16)
