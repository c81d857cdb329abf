// The HMC Markov chain with the EOFA pseudofermion (Sec. 3, Sec. 5):
// per trajectory a fresh pseudofermion from the EOFA heatbath of Eq. (6),
// fresh Gaussian momenta, one molecular-dynamics trajectory of
// H = sum tr P^2 + S_g + S_EOFA (eofa_hmc_trajectory_dev) and a Metropolis
// accept/reject step with probability min(1, exp(-dH)).  The random
// numbers (momenta, heatbath noise, the uniforms of the accept test) are
// inputs, so that a chain can be replayed exactly.
#include "api_util.h"

#include <chrono>
#include <cmath>
#include <vector>

extern "C" int eofa_hmc_dev(eofa_ctx* ctx, const eofa_md_params* md, int ntraj, double alpha0, int npoles,
                            const double* alphas, const double* betas, const double* P_dev, const double* eta_dev,
                            const double* u, double* U_dev, eofa_hmc_traj_info* info, void* stream) {
    if (!ctx || !md || ntraj < 0 || !P_dev || !u || !info) return fail(ctx, EOFA_EINVAL, "null argument");
    if (npoles < 0 || (npoles > 0 && (!alphas || !betas || !eta_dev)))
        return fail(ctx, EOFA_EINVAL, "the heatbath needs npoles >= 1, alphas, betas and eta");
    if (npoles == 0 && md->beta == 0.0) return fail(ctx, EOFA_EINVAL, "nothing to integrate");
    for (int k = 0; k < ntraj; k++)
        if (!(u[k] >= 0.0 && u[k] < 1.0)) return fail(ctx, EOFA_EINVAL, "Metropolis uniforms must lie in [0, 1)");
    cudaStream_t st = (cudaStream_t)stream;
    try {
        require_gauge(ctx);
        const long long nP = 4LL * ctx->V * 9;     // complex entries of a momentum field
        const long long n4 = (long long)ctx->V * 12;  // complex entries of a 4D field
        double* Uc = (double*)ctx_buffer(ctx, "U", 0);
        double* Uold = (double*)ctx_buffer(ctx, "hmc_Uold", (size_t)nP * 16);
        double* Pw = (double*)ctx_buffer(ctx, "hmc_P", (size_t)nP * 16);
        double* phi = npoles > 0 ? (double*)ctx_buffer(ctx, "hmc_phi", (size_t)n4 * 16) : nullptr;
        std::vector<eofa_solve_info> hb(2 * (npoles > 0 ? npoles : 1));
        for (int k = 0; k < ntraj; k++) {
            auto t0 = std::chrono::steady_clock::now();
            eofa_hmc_traj_info r{};
            int iters = 0;
            // pseudofermion refresh: phi = f(M_EOFA) eta, f ~ x^-1/2 (Eq. (6))
            if (npoles > 0) {
                const double* eta = eta_dev + (size_t)k * n4 * 2;
                blas_flat_dot(ctx, n4, eta, eta, 12, st);
                r.eta_norm2 = red_fetch(ctx, 12, st);
                int rc = eofa_heatbath_dev(ctx, md->Ls, md->alpha, md->M5, md->m1, md->m2, md->precision, md->tol,
                                           npoles, alpha0, alphas, betas, eta, phi, 1, hb.data(), st);
                if (rc != EOFA_OK) throw eofa_error(rc, "heatbath failed in trajectory " + std::to_string(k) + ": " + ctx->err);
                for (int l = 0; l < 2 * npoles; l++) iters += hb[l].iters;
            }
            // momentum refresh (given) and the trajectory from the saved links
            EOFA_CUDA(cudaMemcpyAsync(Uold, Uc, (size_t)nP * 16, cudaMemcpyDeviceToDevice, st));
            EOFA_CUDA(cudaMemcpyAsync(Pw, P_dev + (size_t)k * nP * 2, (size_t)nP * 16, cudaMemcpyDeviceToDevice, st));
            eofa_md_info mi{};
            int rc = eofa_hmc_trajectory_dev(ctx, md, phi, Pw, nullptr, &mi, st);
            if (rc != EOFA_OK) throw eofa_error(rc, "trajectory " + std::to_string(k) + " failed: " + ctx->err);
            iters += mi.solver_iters;
            r.H0 = mi.H0;
            r.dH = mi.dH;
            r.S_eofa_start = mi.S_eofa0;
            r.exp_minus_dH = std::exp(-mi.dH);
            // Metropolis: accept with probability min(1, exp(-dH)); a NaN dH is rejected
            r.accepted = (std::isfinite(mi.dH) && u[k] < r.exp_minus_dH) ? 1 : 0;
            if (!r.accepted) {
                EOFA_CUDA(cudaMemcpyAsync(Uc, Uold, (size_t)nP * 16, cudaMemcpyDeviceToDevice, st));
                launch_gauge_pack(ctx, Uc, st);
            }
            // average plaquette Re tr U_p / 3 of the chain's links: S_g(beta = 3) = sum_p (3 - Re tr U_p)
            double Sg3 = 0.0;
            rc = eofa_gauge_action_dev(ctx, 3.0, nullptr, &Sg3, st);
            if (rc != EOFA_OK) throw eofa_error(rc, "plaquette failed: " + ctx->err);
            r.plaquette = 1.0 - Sg3 / (18.0 * ctx->V);
            r.solver_iters = iters;
            EOFA_CUDA(cudaStreamSynchronize(st));
            r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            info[k] = r;
        }
        if (U_dev) EOFA_CUDA(cudaMemcpyAsync(U_dev, Uc, (size_t)nP * 16, cudaMemcpyDeviceToDevice, st));
        EOFA_CUDA(cudaStreamSynchronize(st));
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return EOFA_OK;
}
