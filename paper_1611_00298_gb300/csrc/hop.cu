// Even-odd Wilson hop on every s-slice (the hopping part of D_w, Sec. 2):
//   out(x, s) = -1/2 sum_mu [ (1 - g_mu) U_mu(x) in(x + mu, s)
//                            + (1 + g_mu) U_mu(x - mu)^+ in(x - mu, s) ]
// on the output sites of one parity (dagger: projectors swapped).  This is
// the fused dslash kernel of dslash.cu with the identity as 5D-local block.
#include "fused.h"

void launch_hop(const eofa_ctx* ctx, int prec, int out_parity, int dagger, const void* in, void* out,
                cudaStream_t st) {
    fused_dslash(ctx, prec, out_parity, dagger, in, out, op_identity(), nullptr, 1.0, 0.0, nullptr, 0, st);
}
