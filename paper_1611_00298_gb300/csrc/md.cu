// Molecular dynamics with the EOFA action: the pseudofermion solutions of
// Eq. (5) and (7), the momentum update and the leapfrog trajectory
// H = sum_links tr P^2 + S_EOFA (P traceless Hermitian, U <- exp(i dtau P) U).
#include "api_util.h"

#include <cmath>
#include <vector>

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

// ---------------------------------------------------------------- force-gradient HMC trajectory
//
// H = sum tr P^2 + S_g (Wilson plaquette, beta) + S_EOFA (Eq. (5)), with the
// fourth-order force-gradient integrators (Sec. 5 runs a nested QPQPQ one):
//   PQPQP:  P(h/6) Q(h/2) P~(2h/3) Q(h/2) P(h/6)
//   QPQPQ:  Q(lam h) P~(h/2) Q((1 - 2 lam) h) P~(h/2) Q(lam h),  lam = 1/2 - sqrt(3)/6
// P~(c) is a kick with the force at the displaced links U' = exp(-i z F(U)) U
// (z = h^2/24, PQPQP; (2 - sqrt 3) h^2/12, QPQPQ): to first order in z it is
// the force-gradient correction.  Leapfrog: P(h/2) Q(h) P(h/2).
//
// Time scales are a list of levels, outermost first; every drift of a level
// is the next level's integration (a link update at the innermost one), and
// a level's displacement uses its own force only (the forces commute):
//   one level:     EOFA + gauge (or gauge alone without phi)
//   n_inner > 0:   EOFA | gauge
//   split_lr = 1:  S_R force | S_L force | gauge (asymmetric L/R integration)
//   split_lr = 2:  S_L force | S_R force | gauge
enum Force { F_EOFA_AND_GAUGE, F_EOFA, F_EOFA_L, F_EOFA_R, F_GAUGE };

struct Trajectory {
    eofa_ctx* ctx;
    const eofa_md_params& p;
    const double* phi;
    double* P;
    cudaStream_t st;
    long long nP;
    double *F, *Fz, *Uc, *Usave;
    std::vector<Force> kind;
    std::vector<int> nsub;
    int nferm = 0, ngauge = 0, iters = 0;

    Trajectory(eofa_ctx* c, const eofa_md_params& pp, const double* ph, double* Pd, cudaStream_t s)
        : ctx(c), p(pp), phi(ph), P(Pd), st(s) {
        nP = 4LL * ctx->V * 9;
        F = (double*)ctx_buffer(ctx, "md_F", (size_t)nP * 16);
        Fz = (double*)ctx_buffer(ctx, "md_Fz", (size_t)nP * 16);
        Usave = (double*)ctx_buffer(ctx, "md_Usave", (size_t)nP * 16);
        Uc = (double*)ctx_buffer(ctx, "U", 0);
        if (!phi) {
            kind = {F_GAUGE};
            nsub = {p.nsteps};
        } else if (p.split_lr) {
            // 1: S_R outermost, S_L in the middle; 2: the reverse
            kind = p.split_lr == 2 ? std::vector<Force>{F_EOFA_L, F_EOFA_R} : std::vector<Force>{F_EOFA_R, F_EOFA_L};
            nsub = {p.nsteps, p.n_middle};
            if (p.beta != 0.0) {
                kind.push_back(F_GAUGE);
                nsub.push_back(p.n_inner);
            }
        } else if (p.n_inner > 0) {
            kind = {F_EOFA, F_GAUGE};
            nsub = {p.nsteps, p.n_inner};
        } else {
            kind = {p.beta != 0.0 ? F_EOFA_AND_GAUGE : F_EOFA};
            nsub = {p.nsteps};
        }
    }
    void force(int level, double* out) {
        const Force k = kind[level];
        if (k == F_GAUGE) {
            gauge_force_launch(ctx, Uc, p.beta, 0, out, st);
            ngauge++;
            return;
        }
        eofa_solve_info info[2];
        int rc;
        if (k == F_EOFA_L || k == F_EOFA_R)
            rc = eofa_force_parts_dev(ctx, p.Ls, p.alpha, p.M5, p.m1, p.m2, p.precision, p.tol, phi,
                                      k == F_EOFA_L ? out : nullptr, k == F_EOFA_R ? out : nullptr, info, st);
        else
            rc = eofa_force_dev(ctx, p.Ls, p.alpha, p.M5, p.m1, p.m2, p.precision, p.tol, phi, out, nullptr, info,
                                st);
        if (rc != EOFA_OK) throw eofa_error(rc, "force evaluation failed in the trajectory: " + ctx->err);
        nferm++;
        iters += info[0].iters + info[1].iters;
        if (k == F_EOFA_AND_GAUGE) {
            gauge_force_launch(ctx, Uc, p.beta, 1, out, st);
            ngauge++;
        }
    }
    void links(double eps, const double* Q) {
        int rc = eofa_link_update_dev(ctx, eps, Q, nullptr, st);
        if (rc != EOFA_OK) throw eofa_error(rc, ctx->err);
    }
    // P <- P - c F(U'), U' = exp(-i z F(U)) U
    void kick(int level, double c, double z) {
        if (z != 0.0) {
            force(level, Fz);
            EOFA_CUDA(cudaMemcpyAsync(Usave, Uc, (size_t)nP * 16, cudaMemcpyDeviceToDevice, st));
            links(-z, Fz);
            force(level, F);
            EOFA_CUDA(cudaMemcpyAsync(Uc, Usave, (size_t)nP * 16, cudaMemcpyDeviceToDevice, st));
            launch_gauge_pack(ctx, Uc, st);
        } else {
            force(level, F);
        }
        mom_update_kernel<<<nblk(nP, 256), 256, 0, st>>>(nP, c, (const double2*)F, (double2*)P);
        EOFA_LAUNCHED();
    }
    void drift(int level, double t) {
        if (level + 1 < (int)kind.size()) steps(level + 1, t);
        else links(t, P);
    }
    void steps(int level, double t) {
        const int n = nsub[level];
        const double h = t / n;
        for (int k = 0; k < n; k++) {
            if (p.integrator == EOFA_INT_FG_PQPQP) {
                kick(level, h / 6, 0.0);
                drift(level, h / 2);
                kick(level, 2 * h / 3, h * h / 24);
                drift(level, h / 2);
                kick(level, h / 6, 0.0);
            } else if (p.integrator == EOFA_INT_FG_QPQPQ) {
                const double lam = 0.5 - std::sqrt(3.0) / 6.0, z = (2.0 - std::sqrt(3.0)) / 12.0 * h * h;
                drift(level, lam * h);
                kick(level, h / 2, z);
                drift(level, (1 - 2 * lam) * h);
                kick(level, h / 2, z);
                drift(level, lam * h);
            } else {
                kick(level, h / 2, 0.0);
                drift(level, h);
                kick(level, h / 2, 0.0);
            }
        }
    }
    void energy(double* K, double* Sg, double* Sf) {
        blas_flat_dot(ctx, nP, P, P, 12, st);
        *K = red_fetch(ctx, 12, st);
        *Sg = p.beta != 0.0 ? gauge_action_now(ctx, Uc, p.beta, st) : 0.0;
        *Sf = 0.0;
        if (phi) {
            eofa_solve_info info[2];
            int rc = eofa_action_dev(ctx, p.Ls, p.alpha, p.M5, p.m1, p.m2, p.precision, p.tol, phi, Sf, info, st);
            if (rc != EOFA_OK) throw eofa_error(rc, "action failed in the trajectory: " + ctx->err);
            iters += info[0].iters + info[1].iters;
        }
    }
};

extern "C" int eofa_hmc_trajectory_dev(eofa_ctx* ctx, const eofa_md_params* p, const double* phi_dev, double* P_dev,
                                       double* U_dev, eofa_md_info* info, void* stream) {
    if (!ctx || !p || !P_dev || !info) return fail(ctx, EOFA_EINVAL, "null argument");
    const bool bad_split = p->split_lr < 0 || p->split_lr > 2 ||
                           (p->split_lr && (!phi_dev || p->n_middle < 1 || (p->beta != 0.0 && p->n_inner < 1)));
    if (p->nsteps < 1 || !(p->tau > 0) || p->n_inner < 0 || p->integrator < EOFA_INT_LEAPFROG ||
        p->integrator > EOFA_INT_FG_QPQPQ || (!p->split_lr && p->n_inner > 0 && (!phi_dev || p->beta == 0.0)) ||
        (!phi_dev && p->beta == 0.0) || bad_split)
        return fail(ctx, EOFA_EINVAL, "bad trajectory parameters");
    cudaStream_t st = (cudaStream_t)stream;
    try {
        require_gauge(ctx);
        Trajectory T(ctx, *p, phi_dev, P_dev, st);
        eofa_md_info r{};
        T.energy(&r.kinetic0, &r.S_gauge0, &r.S_eofa0);
        T.steps(0, p->tau);
        T.energy(&r.kinetic1, &r.S_gauge1, &r.S_eofa1);
        r.H0 = r.kinetic0 + r.S_gauge0 + r.S_eofa0;
        r.dH = (r.kinetic1 + r.S_gauge1 + r.S_eofa1) - r.H0;
        r.fermion_forces = T.nferm;
        r.gauge_forces = T.ngauge;
        r.solver_iters = T.iters;
        if (U_dev) EOFA_CUDA(cudaMemcpyAsync(U_dev, T.Uc, (size_t)T.nP * 16, cudaMemcpyDeviceToDevice, st));
        EOFA_CUDA(cudaStreamSynchronize(st));
        *info = r;
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return EOFA_OK;
}

}  // extern "C"
