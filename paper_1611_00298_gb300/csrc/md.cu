// Molecular dynamics with the EOFA action: the pseudofermion solutions of
// Eq. (5) and (7), the momentum update and the leapfrog trajectory
// H = sum_links tr P^2 + S_EOFA (P traceless Hermitian, U <- exp(i dtau P) U).
#include "api_util.h"

#include <cmath>

namespace {

// P <- P - eps F (flat complex arrays)
__global__ void mom_update_kernel(long long n, double eps, const double2* __restrict__ F, double2* P) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= n) return;
    double2 f = F[t], p = P[t];
    P[t] = make_double2(p.x - eps * f.x, p.y - eps * f.y);
}

inline unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

int eofa_chis_to(eofa_ctx* ctx, int Ls, double alpha, double M5, double m1, double m2, int precision, double tol,
                 const double* phi_dev, double* chiL, double* chiR, double* S, eofa_solve_info info[2], cudaStream_t st);

extern "C" {

int eofa_pseudofermion_solutions_dev(eofa_ctx* ctx, int Ls, double alpha, double M5, double m1, double m2,
                                     int precision, double tol, const double* phi_dev, double* chiL_dev,
                                     double* chiR_dev, double* S, eofa_solve_info info[2], void* stream) {
    if (!ctx || !phi_dev || !chiL_dev || !chiR_dev) return fail(ctx, EOFA_EINVAL, "null argument");
    eofa_solve_info loc[2];
    try {
        return eofa_chis_to(ctx, Ls, alpha, M5, m1, m2, precision, tol, phi_dev, chiL_dev, chiR_dev, S,
                            info ? info : loc, (cudaStream_t)stream);
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
}

int eofa_leapfrog_dev(eofa_ctx* ctx, int Ls, double alpha, double M5, double m1, double m2, int precision, double tol,
                      int nsteps, double dtau, const double* phi_dev, double* P_dev, double* U_dev, double* dH,
                      double* H0_out, void* stream) {
    if (!ctx || !phi_dev || !P_dev || !dH || nsteps < 1 || !(dtau > 0)) return fail(ctx, EOFA_EINVAL, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    try {
        require_gauge(ctx);
        const long long nP = 4LL * ctx->V * 9;  // complex entries of P and F
        double* F = (double*)ctx_buffer(ctx, "md_F", (size_t)nP * 16);
        eofa_solve_info info[2];
        auto kinetic = [&]() {
            blas_flat_dot(ctx, nP, P_dev, P_dev, 12, st);
            return red_fetch(ctx, 12, st);
        };
        auto force = [&](double* S) {
            int rc = eofa_force_dev(ctx, Ls, alpha, M5, m1, m2, precision, tol, phi_dev, F, S, info, st);
            if (rc != EOFA_OK) throw eofa_error(rc, "force evaluation failed in the trajectory: " + ctx->err);
        };
        auto mom = [&](double eps) {
            mom_update_kernel<<<nblk(nP, 256), 256, 0, st>>>(nP, eps, (const double2*)F, (double2*)P_dev);
            EOFA_LAUNCHED();
        };
        auto links = [&]() {
            int rc = eofa_link_update_dev(ctx, dtau, P_dev, U_dev, st);
            if (rc != EOFA_OK) throw eofa_error(rc, ctx->err);
        };
        double S0 = 0, S1 = 0;
        double K0 = kinetic();
        force(&S0);
        mom(0.5 * dtau);
        for (int step = 0; step < nsteps; step++) {
            links();
            force(&S1);
            mom(step < nsteps - 1 ? dtau : 0.5 * dtau);
        }
        double K1 = kinetic();
        *dH = (K1 + S1) - (K0 + S0);
        if (H0_out) *H0_out = K0 + S0;
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return EOFA_OK;
}

}  // extern "C"
