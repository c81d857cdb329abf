// Fused kernels of the solver hot loop (dslash.cu) and the device-scalar layout.
#pragma once
#include "internal.h"

// Layout of ctx->red (doubles):
//   [0, 64)              results of the generic reductions (blas.cu)
//   [SC_RRH, +32)        |r|^2 history ring of the CG (index it % 32)
//   SC_GAMMA, +1         gamma = |A^+ r|^2, double-buffered by iteration parity
//   SC_DELTA             delta = |A p|^2
//   [128, 1344), 1344    partials and ticket of the generic reductions
//   [RED_PART, +RED_MAX_BLOCKS), RED_TICKET   partials and ticket of the fused kernels
//   RED_ERRWORD          device error word (bounded waits that ran out)
//   [RED_PART2, +RED_MAX_BLOCKS)  partials of the second sum of the two-sum launches
#define SC_RRH 64
#define SC_GAMMA 96
#define SC_DELTA 98
#define RED_PART 2048
#define RED_MAX_BLOCKS 4096
#define RED_TICKET (RED_PART + RED_MAX_BLOCKS)
#define RED_ERRWORD (RED_TICKET + 2)  // int: nonzero after a device wait timed out
#define RED_PART2 (RED_TICKET + 8)
#define RED_TOTAL_DOUBLES (RED_PART2 + RED_MAX_BLOCKS)

// out = a_out * (-1/2) B[hop(in)] + b_in * y ; |out|^2 -> red[slot] if red
void fused_dslash(const eofa_ctx* ctx, int prec, int out_parity, int dagger, const void* in, void* out, const Op5& op,
                  const void* y, double a_out, double b_in, double* red, int slot, cudaStream_t st);
// The two launches of the CG iteration that carry more than one output
// (solver.cu):
//   fused_dslash_to: out = a_out (-1/2) B[hop(in)] + b_in y, |out|^2 -> red[slot],
//                    out2 = B2 out (a second 5D-local block applied in the epilogue)
//   fused_dslash_z:  with alpha = alpha(red, it) and w = a_out (-1/2) B[hop(in)] + b_in y:
//                    z <- z - alpha w, |z|^2 -> red[slot];  when r is not null also
//                    r <- r - alpha y, |r|^2 -> red[rslot]
void fused_dslash_to(const eofa_ctx* ctx, int prec, int out_parity, int dagger, const void* in, void* out,
                     const Op5& op, const void* y, double a_out, double b_in, double* red, int slot, const Op5& op2,
                     void* out2, cudaStream_t st);
void fused_dslash_z(const eofa_ctx* ctx, int prec, int out_parity, int dagger, const void* in, void* z, const Op5& op,
                    const void* y, double a_out, double b_in, double* red, int slot, int it, void* r, int rslot,
                    cudaStream_t st);
//   fused_dslash_x:  out = (-1/2) B[hop(in)], and x <- x + alpha(red, it) p and (r not null)
//                    r <- r - alpha q elementwise at the same (j, s), |r|^2 -> red[rslot] (x in
//                    the solution precision: FP32 for FP16 fields)
void fused_dslash_x(const eofa_ctx* ctx, int prec, int out_parity, int dagger, const void* in, void* out,
                    const Op5& op, double* red, int it, void* x, const void* p, void* r, const void* q, int rslot,
                    cudaStream_t st);
// x' = x + c z (c = -alpha(sc, it) if use_alpha else c0); xw <- x'; |x'|^2 -> red[slot]; out = a_out B x'
void fused_local5(const eofa_ctx* ctx, int prec, const Op5& op, const void* x, const void* z, double c0,
                  const double* sc, int it, int use_alpha, void* xw, void* out, double a_out, double* red, int slot,
                  cudaStream_t st);
// x += alpha p (skipped when x is null); p = s + beta p   (alpha, beta from sc at iteration it)
void fused_xp_update(const eofa_ctx* ctx, int prec, int precx, const double* sc, int it, void* x, void* p,
                     const void* s, cudaStream_t st);
Op5 op_identity();

// throws EOFA_ETIMEOUT (and clears the word) when a kernel's bounded wait ran out
void check_device_error(const eofa_ctx* ctx, cudaStream_t st);
