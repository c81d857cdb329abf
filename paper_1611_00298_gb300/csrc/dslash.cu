// Precision dispatch of the fused solver kernels (dslash_impl.cuh).
#include "dslash_impl.cuh"

Op5 op_identity() {
    Op5 op;
    for (int h = 0; h < 2; h++) {
        op.inv[h] = op.fwd[h] = 0;
        op.p1[h] = op.q1[h] = op.p2[h] = op.q2[h] = 0.0;
        op.dir1[h] = op.dir2[h] = 0;
        op.sigma[h] = 0.0;
        op.w[h] = op.v[h] = nullptr;
    }
    op.mass = 0.0;
    op.a_out = 1.0;
    op.b_in = 0.0;
    return op;
}

// bytes of one spinor (site, slice) as stored, per precision (FP16 with its scale)
static double spinor_bytes(int prec) { return prec == P64 ? 192.0 : prec == P32 ? 96.0 : 52.0; }

void fused_dslash(const eofa_ctx* ctx, int prec, int out_parity, int dagger, const void* in, void* out, const Op5& op,
                  const void* y, double a_out, double b_in, double* red, int slot, cudaStream_t st) {
    const Op5 opf = op_finalize(op, ctx->Ls);
    const double n5h = (double)ctx->Vh * ctx->Ls;
    const double bytes = n5h * spinor_bytes(prec) * (y ? 3.0 : 2.0) + 8.0 * ctx->Vh * (prec == P64 ? 144.0 : 72.0);
    prof_begin(ctx, prec, st, bytes);
    if (prec == P64) dslash_p64(ctx, out_parity, dagger, in, out, opf, y, a_out, b_in, red, slot, st);
    else if (prec == P32) dslash_p32(ctx, out_parity, dagger, in, out, opf, y, a_out, b_in, red, slot, st);
    else dslash_p16(ctx, out_parity, dagger, in, out, opf, y, a_out, b_in, red, slot, st);
    prof_end(ctx, st);
}

void fused_local5(const eofa_ctx* ctx, int prec, const Op5& op, const void* x, const void* z, double c0,
                  const double* sc, int it, int use_alpha, void* xw, void* out, double a_out, double* red, int slot,
                  cudaStream_t st) {
    const Op5 opf = op_finalize(op, ctx->Ls);
    const double nf = 1.0 + (z ? 1.0 : 0.0) + (xw ? 1.0 : 0.0) + (out ? 1.0 : 0.0);
    prof_begin(ctx, 3 + prec, st, (double)ctx->Vh * ctx->Ls * spinor_bytes(prec) * nf);
    if (prec == P64) local5_p64(ctx, opf, x, z, c0, sc, it, use_alpha, xw, out, a_out, red, slot, st);
    else if (prec == P32) local5_p32(ctx, opf, x, z, c0, sc, it, use_alpha, xw, out, a_out, red, slot, st);
    else local5_p16(ctx, opf, x, z, c0, sc, it, use_alpha, xw, out, a_out, red, slot, st);
    prof_end(ctx, st);
}

void fused_xp_update(const eofa_ctx* ctx, int prec, int precx, const double* sc, int it, void* x, void* p,
                     const void* s, cudaStream_t st) {
    if (prec == P64) xp_update_p64(ctx, sc, it, x, p, s, st);
    else if (prec == P32) xp_update_p32(ctx, sc, it, x, p, s, st);
    else xp_update_p16(ctx, sc, it, x, p, s, st);
}

void fused_dslash_to(const eofa_ctx* ctx, int prec, int out_parity, int dagger, const void* in, void* out,
                     const Op5& op, const void* y, double a_out, double b_in, double* red, int slot, const Op5& op2,
                     void* out2, cudaStream_t st) {
    const Op5 opf = op_finalize(op, ctx->Ls);
    const Op5 op2f = op_finalize(op2, ctx->Ls);
    const double n5h = (double)ctx->Vh * ctx->Ls;
    // in, out, out2 (+ y): one spinor each per output site, links once per 4D site
    const double bytes = n5h * spinor_bytes(prec) * (y ? 4.0 : 3.0) + 8.0 * ctx->Vh * (prec == P64 ? 144.0 : 72.0);
    prof_begin(ctx, prec, st, bytes);
    if (prec == P64) dslash_to_p64(ctx, out_parity, dagger, in, out, opf, y, a_out, b_in, red, slot, op2f, out2, st);
    else if (prec == P32) dslash_to_p32(ctx, out_parity, dagger, in, out, opf, y, a_out, b_in, red, slot, op2f, out2, st);
    else dslash_to_p16(ctx, out_parity, dagger, in, out, opf, y, a_out, b_in, red, slot, op2f, out2, st);
    prof_end(ctx, st);
}

void fused_dslash_z(const eofa_ctx* ctx, int prec, int out_parity, int dagger, const void* in, void* z, const Op5& op,
                    const void* y, double a_out, double b_in, double* red, int slot, int it, void* r, int rslot,
                    cudaStream_t st) {
    const Op5 opf = op_finalize(op, ctx->Ls);
    const double n5h = (double)ctx->Vh * ctx->Ls;
    // in, y and z read, z written; r read and written when given
    const double bytes = n5h * spinor_bytes(prec) * (r ? 6.0 : 4.0) + 8.0 * ctx->Vh * (prec == P64 ? 144.0 : 72.0);
    prof_begin(ctx, prec, st, bytes);
    if (prec == P64) dslash_z_p64(ctx, out_parity, dagger, in, z, opf, y, a_out, b_in, red, slot, it, r, rslot, st);
    else if (prec == P32) dslash_z_p32(ctx, out_parity, dagger, in, z, opf, y, a_out, b_in, red, slot, it, r, rslot, st);
    else dslash_z_p16(ctx, out_parity, dagger, in, z, opf, y, a_out, b_in, red, slot, it, r, rslot, st);
    prof_end(ctx, st);
}

void fused_dslash_x(const eofa_ctx* ctx, int prec, int out_parity, int dagger, const void* in, void* out,
                    const Op5& op, double* red, int it, void* x, const void* p, void* r, const void* q, int rslot,
                    cudaStream_t st) {
    const Op5 opf = op_finalize(op, ctx->Ls);
    const double n5h = (double)ctx->Vh * ctx->Ls;
    // in, out, p read, x read and written; with r: q read, r read and written (x in FP32 when the field is FP16)
    const double xb = prec == P16 ? 96.0 : spinor_bytes(prec);
    const double bytes = n5h * (spinor_bytes(prec) * (r ? 6.0 : 3.0) + 2.0 * xb) +
                         8.0 * ctx->Vh * (prec == P64 ? 144.0 : 72.0);
    prof_begin(ctx, prec, st, bytes);
    if (prec == P64) dslash_x_p64(ctx, out_parity, dagger, in, out, opf, red, it, x, p, r, q, rslot, st);
    else if (prec == P32) dslash_x_p32(ctx, out_parity, dagger, in, out, opf, red, it, x, p, r, q, rslot, st);
    else dslash_x_p16(ctx, out_parity, dagger, in, out, opf, red, it, x, p, r, q, rslot, st);
    prof_end(ctx, st);
}
