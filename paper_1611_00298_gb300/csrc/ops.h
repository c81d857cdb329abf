// Host-side composition of the 5D-local operators of Eq. (3) and of the
// EOFA rank-one terms (Sec. 2, Eq. (8)).
#pragma once
#include "internal.h"

// Scalars of one Moebius operator at mass m: D-tilde = b + c5 L and the
// even-odd diagonal block M = (4 - M5) D-tilde + 1 - L = p + q L.
struct Coeffs {
    double b, c5, p, q, mass;
};
Coeffs make_coeffs(double alpha, double M5, double m);

// The 5D-local block G' of a system (D_hop + G') psi = f with
// G = M D-tilde^{-1} and an optional rank-one term on one chirality:
// G' = G + sg w v^T (w, v real Ls-vectors) on chirality r1_h (0 = P_+, 1 = P_-).
struct System5 {
    Coeffs c;
    int r1_h;  // -1: no rank-one term
    double sg;
    std::vector<double> w, v;
};

System5 system_dwf(double alpha, double M5, double mf);
// EOFA system (H(m) + a Delta_chi P_chi): which = EOFA_SYS_EOFA_L (m = m1,
// chirality -) or EOFA_SYS_EOFA_R (m = m2, chirality +).
System5 system_eofa(int Ls, double alpha, double M5, double m1, double m2, int which, double a);

// EOFA closed forms: k and Omega_pm (Delta_pm = k Omega_pm Omega_pm^T).
double eofa_k(int Ls, double alpha, double m1, double m2);
void eofa_omega(int Ls, double alpha, double* Op, double* Om);

// Op5 descriptors; rank-one vectors are uploaded to ctx->coef at slot*Ls.
Op5 op_plain(const Coeffs& c, int inv_which, int fwd_which, int transpose);
// which: 0 none, 1 D-tilde, 2 M
Op5 op_G(eofa_ctx* ctx, const System5& S, int slot, cudaStream_t st);
Op5 op_Ginv(eofa_ctx* ctx, const System5& S, int slot, cudaStream_t st);
Op5 op_GinvT(eofa_ctx* ctx, const System5& S, int slot, cudaStream_t st);
