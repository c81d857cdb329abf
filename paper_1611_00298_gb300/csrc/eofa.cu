// EOFA action (Eq. (5)), pseudofermion force (Eq. (7)) and the molecular-
// dynamics link update.
//
// Action: with chi_L = H(m1)^{-1} Omega_- P_- phi and
// chi_R = [H(m2) - Delta_+ P_+]^{-1} Omega_+ P_+ phi,
//   S = |phi|^2 - k <Omega_- P_- phi, chi_L> + k <Omega_+ P_+ phi, chi_R>.
//
// Force: d D_w under U_mu(x) -> U + dU touches the forward hop at x and the
// backward hop at x + mu.  With zeta = gamma_5 R_5 chi, the two terms of
// chi^+ gamma_5 R_5 (dD_w) chi are complex conjugates, so
//   chi^+ g5 R5 (dD_w) chi = -Re tr(dU Y1),
//   Y1_{ba} = sum_s sum_{i=0,1} h_{ib}(x + mu, s) conj(g_{ia}(x, Ls-1-s)),
// h = chi_u - A_mu chi_l (the (1 - gamma_mu) half spinor at x + mu) and
// g = chi_u + A_mu chi_l at (x, Ls-1-s).  With Y = k (Y1[chi_L] - Y1[chi_R])
// (times the boundary phase), dS = -Re tr(dU Y): for dU = i w T^a U,
// F^a = Im tr(T^a U Y) and F = sum_a F^a T^a = -(i/4)[(X - X^+) - tr(X - X^+)/3]
// with X = U Y; the real-view gradient is dS/dRe U + i dS/dIm U = -Y^+.
#include "api_util.h"

#include <cmath>

namespace {

struct Coords {
    int X, Y, Z, T;
};

// embed: out(s, i) = Om[s] P_chi phi(i); chirality chi = +1 keeps spins 0,1
__global__ void embed_kernel(long long V, int Ls, const double2* __restrict__ phi, const double* __restrict__ Om, int chi,
                             double2* __restrict__ out) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long n = V * 12 * Ls;
    if (t >= n) return;
    int s = (int)(t / (V * 12));
    long long r = t - (long long)s * V * 12;
    int c = (int)(r % 12);
    bool keep = chi > 0 ? (c < 6) : (c >= 6);
    double2 z = phi[r];
    double w = keep ? Om[s] : 0.0;
    out[t] = make_double2(w * z.x, w * z.y);
}

template <int MU>
__device__ __forceinline__ void proj_A(const cpx<double>* v, int sg, cpx<double> out[6]) {
    // out = v_u + sg A_mu v_l (two spins x three colours)
    for (int c = 0; c < 3; c++) {
        cpx<double> l0 = v[6 + c], l1 = v[9 + c], a0, a1;
        if (MU == 0) { a0 = mitimes(l1); a1 = mitimes(l0); }
        if (MU == 1) { a0 = mk(-l1.re, -l1.im); a1 = l0; }
        if (MU == 2) { a0 = mitimes(l0); a1 = itimes(l1); }
        if (MU == 3) { a0 = l0; a1 = l1; }
        out[c] = sg > 0 ? v[c] + a0 : v[c] - a0;
        out[3 + c] = sg > 0 ? v[3 + c] + a1 : v[3 + c] - a1;
    }
}

template <int MU>
__device__ void accumulate_Y(const double2* chi, long long V, int Ls, long long i, long long ifw, double coef,
                             cpx<double> Y[9]) {
    for (int s = 0; s < Ls; s++) {
        cpx<double> vf[12], vb[12], h[6], g[6];
        const double2* pf = chi + ((long long)s * V + ifw) * 12;
        const double2* pb = chi + ((long long)(Ls - 1 - s) * V + i) * 12;
        for (int c = 0; c < 12; c++) {
            vf[c] = mk(pf[c].x, pf[c].y);
            vb[c] = mk(pb[c].x, pb[c].y);
        }
        proj_A<MU>(vf, -1, h);
        proj_A<MU>(vb, +1, g);
        for (int b = 0; b < 3; b++)
            for (int a = 0; a < 3; a++) {
                cpx<double> acc = cjmul(g[a], h[b]);
                acc = acc + cjmul(g[3 + a], h[3 + b]);
                Y[3 * b + a] = Y[3 * b + a] + coef * acc;
            }
    }
}

// mode 0: traceless Hermitian force F; mode 1: real-view gradient -Y^+
__global__ void force_kernel(Coords d, int Ls, int bc_t, double k, const double2* __restrict__ U,
                             const double2* __restrict__ chiL, const double2* __restrict__ chiR, double2* __restrict__ F,
                             int mode) {
    long long V = (long long)d.X * d.Y * d.Z * d.T;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= 4 * V) return;
    long long i = t / 4;
    int mu = (int)(t % 4);
    int x = (int)(i % d.X), y = (int)((i / d.X) % d.Y), z = (int)((i / ((long long)d.X * d.Y)) % d.Z),
        tt = (int)(i / ((long long)d.X * d.Y * d.Z));
    int c[4] = {x, y, z, tt};
    int n[4] = {d.X, d.Y, d.Z, d.T};
    double phase = 1.0;
    c[mu] += 1;
    if (c[mu] == n[mu]) {
        c[mu] = 0;
        if (mu == 3) phase = (double)bc_t;
    }
    long long ifw = c[0] + (long long)d.X * (c[1] + (long long)d.Y * (c[2] + (long long)d.Z * c[3]));
    cpx<double> Y[9];
    for (int e = 0; e < 9; e++) Y[e] = mk(0.0, 0.0);
    switch (mu) {
        // a null chi drops its term (the force of S_L or S_R alone)
        case 0:
            if (chiL) accumulate_Y<0>(chiL, V, Ls, i, ifw, k, Y);
            if (chiR) accumulate_Y<0>(chiR, V, Ls, i, ifw, -k, Y);
            break;
        case 1:
            if (chiL) accumulate_Y<1>(chiL, V, Ls, i, ifw, k, Y);
            if (chiR) accumulate_Y<1>(chiR, V, Ls, i, ifw, -k, Y);
            break;
        case 2:
            if (chiL) accumulate_Y<2>(chiL, V, Ls, i, ifw, k, Y);
            if (chiR) accumulate_Y<2>(chiR, V, Ls, i, ifw, -k, Y);
            break;
        default:
            if (chiL) accumulate_Y<3>(chiL, V, Ls, i, ifw, k, Y);
            if (chiR) accumulate_Y<3>(chiR, V, Ls, i, ifw, -k, Y);
            break;
    }
    for (int e = 0; e < 9; e++) Y[e] = phase * Y[e];
    double2* out = F + t * 9;
    if (mode == 1) {
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) out[3 * a + b] = make_double2(-Y[3 * b + a].re, Y[3 * b + a].im);
        return;
    }
    const double2* u = U + t * 9;
    cpx<double> X[9];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            cpx<double> acc = mk(0.0, 0.0);
            for (int e = 0; e < 3; e++) acc = acc + cmul(mk(u[3 * a + e].x, u[3 * a + e].y), Y[3 * e + b]);
            X[3 * a + b] = acc;
        }
    // A = X - X^+ (anti-Hermitian), F = -(i/4)(A - tr(A)/3)
    cpx<double> A[9];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) A[3 * a + b] = X[3 * a + b] - mk(X[3 * b + a].re, -X[3 * b + a].im);
    cpx<double> tr3 = (1.0 / 3.0) * (A[0] + A[4] + A[8]);
    for (int a = 0; a < 3; a++) A[4 * a] = A[4 * a] - tr3;
    for (int e = 0; e < 9; e++) {
        cpx<double> f = mk(0.25 * A[e].im, -0.25 * A[e].re);  // -(i/4) A
        out[e] = make_double2(f.re, f.im);
    }
}

// U <- exp(i eps P) U, exp by Taylor series with scaling and squaring
// (Moler and Van Loan, "Nineteen dubious ways to compute the exponential of
// a matrix", method 3); P Hermitian.
__device__ void mat3_mul(const cpx<double>* a, const cpx<double>* b, cpx<double>* c) {
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cpx<double> acc = mk(0.0, 0.0);
            for (int k = 0; k < 3; k++) acc = acc + cmul(a[3 * i + k], b[3 * k + j]);
            c[3 * i + j] = acc;
        }
}

__global__ void link_update_kernel(long long nlinks, double eps, const double2* __restrict__ P, double2* Uc,
                                   double2* Ux) {
    long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (l >= nlinks) return;
    cpx<double> A[9];
    double nrm = 0;
    for (int e = 0; e < 9; e++) {
        double2 p = P[l * 9 + e];
        A[e] = mk(-eps * p.y, eps * p.x);  // i eps P
        nrm += A[e].re * A[e].re + A[e].im * A[e].im;
    }
    nrm = sqrt(nrm);
    int sq = 0;
    while (nrm > 0.25 && sq < 60) { nrm *= 0.5; sq++; }
    double sc = ldexp(1.0, -sq);
    for (int e = 0; e < 9; e++) A[e] = sc * A[e];
    cpx<double> E[9], term[9], tmp[9];
    for (int e = 0; e < 9; e++) { E[e] = mk(e % 4 == 0 ? 1.0 : 0.0, 0.0); term[e] = E[e]; }
    for (int n = 1; n <= 14; n++) {
        mat3_mul(term, A, tmp);
        for (int e = 0; e < 9; e++) { term[e] = (1.0 / n) * tmp[e]; E[e] = E[e] + term[e]; }
    }
    for (int k = 0; k < sq; k++) {
        mat3_mul(E, E, tmp);
        for (int e = 0; e < 9; e++) E[e] = tmp[e];
    }
    cpx<double> u[9], out[9];
    for (int e = 0; e < 9; e++) u[e] = mk(Uc[l * 9 + e].x, Uc[l * 9 + e].y);
    mat3_mul(E, u, out);
    for (int e = 0; e < 9; e++) {
        Uc[l * 9 + e] = make_double2(out[e].re, out[e].im);
        if (Ux) Ux[l * 9 + e] = make_double2(out[e].re, out[e].im);
    }
}

inline unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

struct ChiBufs {
    double *bL, *bR, *chiL, *chiR;
};

// The two solves behind Eq. (5) and Eq. (7); fills S if requested.
// parts: 1 = chi_L only, 2 = chi_R only, 3 = both (S needs both).
ChiBufs eofa_chis(eofa_ctx* ctx, int Ls, double alpha, double M5, double m1, double m2, int precision, double tol,
                  const double* phi_dev, double* S, eofa_solve_info info[2], cudaStream_t st, int* rc_out,
                  double* chiL_out = nullptr, double* chiR_out = nullptr, int parts = 3) {
    check_ls(ctx, Ls);
    require_gauge(ctx);
    if (!(m1 < m2)) throw eofa_error(EOFA_EINVAL, "EOFA needs m1 < m2 (k > 0)");
    long long V = ctx->V;
    size_t b5 = (size_t)V * Ls * 12 * 16;
    ChiBufs c;
    c.bL = (double*)ctx_buffer(ctx, "eo_bL", b5);
    c.bR = (double*)ctx_buffer(ctx, "eo_bR", b5);
    c.chiL = chiL_out ? chiL_out : (double*)ctx_buffer(ctx, "eo_chiL", b5);
    c.chiR = chiR_out ? chiR_out : (double*)ctx_buffer(ctx, "eo_chiR", b5);
    double* om = (double*)ctx_buffer(ctx, "eo_omega", 2 * EOFA_MAX_LS * sizeof(double));
    std::vector<double> Op(Ls), Om(Ls);
    eofa_omega(Ls, alpha, Op.data(), Om.data());
    EOFA_CUDA(cudaMemcpyAsync(om, Op.data(), Ls * sizeof(double), cudaMemcpyHostToDevice, st));
    EOFA_CUDA(cudaMemcpyAsync(om + EOFA_MAX_LS, Om.data(), Ls * sizeof(double), cudaMemcpyHostToDevice, st));
    long long n = V * 12 * Ls;
    embed_kernel<<<nblk(n, 256), 256, 0, st>>>(V, Ls, (const double2*)phi_dev, om + EOFA_MAX_LS, -1, (double2*)c.bL);
    EOFA_LAUNCHED();
    embed_kernel<<<nblk(n, 256), 256, 0, st>>>(V, Ls, (const double2*)phi_dev, om, +1, (double2*)c.bR);
    EOFA_LAUNCHED();
    eofa_solve_params p;
    p.Ls = Ls;
    p.alpha = alpha;
    p.M5 = M5;
    p.mf = 0;
    p.m1 = m1;
    p.m2 = m2;
    p.precision = precision;
    p.tol = tol;
    p.maxiter = 100000;
    p.delta = ctx->rel_delta;
    p.use_x0 = 0;
    p.system = EOFA_SYS_EOFA_L;
    p.shift = 0.0;
    int rc1 = EOFA_OK, rc2 = EOFA_OK;
    info[0] = info[1] = eofa_solve_info{};
    if (parts & 1) rc1 = solve_dev_impl(ctx, &p, c.bL, c.chiL, &info[0], st);
    p.system = EOFA_SYS_EOFA_R;
    p.shift = -1.0;
    if (parts & 2) rc2 = solve_dev_impl(ctx, &p, c.bR, c.chiR, &info[1], st);
    *rc_out = rc1 != EOFA_OK ? rc1 : rc2;
    if (S && parts == 3) {
        double k = eofa_k(Ls, alpha, m1, m2);
        blas_flat_dot(ctx, V * 12, phi_dev, phi_dev, 6, st);
        blas_flat_dot(ctx, n, c.bL, c.chiL, 8, st);
        blas_flat_dot(ctx, n, c.bR, c.chiR, 10, st);
        double v[6];
        red_fetch_many(ctx, 6, 6, v, st);
        *S = v[0] - k * v[2] + k * v[4];
    }
    return c;
}

}  // namespace

void eofa_embed(eofa_ctx* ctx, const double* phi, const double* Om_dev, int chi, double* out, cudaStream_t st) {
    long long V = ctx->V, n = V * 12 * ctx->Ls;
    embed_kernel<<<nblk(n, 256), 256, 0, st>>>(V, ctx->Ls, (const double2*)phi, Om_dev, chi, (double2*)out);
    EOFA_LAUNCHED();
}

int eofa_chis_to(eofa_ctx* ctx, int Ls, double alpha, double M5, double m1, double m2, int precision, double tol,
                 const double* phi_dev, double* chiL, double* chiR, double* S, eofa_solve_info info[2], cudaStream_t st) {
    int rc = EOFA_OK;
    eofa_chis(ctx, Ls, alpha, M5, m1, m2, precision, tol, phi_dev, S, info, st, &rc, chiL, chiR);
    EOFA_CUDA(cudaStreamSynchronize(st));
    return rc;
}

extern "C" {

int eofa_action_dev(eofa_ctx* ctx, int Ls, double alpha, double M5, double m1, double m2, int precision, double tol,
                    const double* phi_dev, double* S, eofa_solve_info info[2], void* stream) {
    if (!ctx || !phi_dev || !S) return fail(ctx, EOFA_EINVAL, "null argument");
    eofa_solve_info loc[2];
    if (!info) info = loc;
    try {
        int rc = EOFA_OK;
        eofa_chis(ctx, Ls, alpha, M5, m1, m2, precision, tol, phi_dev, S, info, (cudaStream_t)stream, &rc);
        return rc;
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
}

int eofa_action(eofa_ctx* ctx, int Ls, double alpha, double M5, double m1, double m2, int precision, double tol,
                const double* phi, double* S, eofa_solve_info info[2]) {
    if (!ctx || !phi || !S) return fail(ctx, EOFA_EINVAL, "null argument");
    try {
        size_t b4 = (size_t)ctx->V * 12 * 16;
        double* dphi = (double*)ctx_buffer(ctx, "host_phi", b4);
        EOFA_CUDA(cudaMemcpyAsync(dphi, phi, b4, cudaMemcpyHostToDevice, ctx->stream));
        return eofa_action_dev(ctx, Ls, alpha, M5, m1, m2, precision, tol, dphi, S, info, ctx->stream);
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
}

static void launch_force(eofa_ctx* ctx, double k, const double* chiL, const double* chiR, double* F, int mode,
                         cudaStream_t st) {
    require_gauge(ctx);
    Coords d = {ctx->dims[0], ctx->dims[1], ctx->dims[2], ctx->dims[3]};
    const double* U = (const double*)ctx_buffer(ctx, "U", 0);
    long long nl = 4LL * ctx->V;
    force_kernel<<<nblk(nl, 128), 128, 0, st>>>(d, ctx->Ls, ctx->bc_t, k, (const double2*)U, (const double2*)chiL,
                                                (const double2*)chiR, (double2*)F, mode);
    EOFA_LAUNCHED();
}

int eofa_force_from_chi_dev(eofa_ctx* ctx, double k, const double* chiL_dev, const double* chiR_dev, double* F_dev,
                            void* stream) {
    if (!ctx || !chiL_dev || !chiR_dev || !F_dev) return fail(ctx, EOFA_EINVAL, "null argument");
    try {
        launch_force(ctx, k, chiL_dev, chiR_dev, F_dev, 0, (cudaStream_t)stream);
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return EOFA_OK;
}

int eofa_grad_from_chi_dev(eofa_ctx* ctx, double k, const double* chiL_dev, const double* chiR_dev, double* G_dev,
                           void* stream) {
    if (!ctx || !chiL_dev || !chiR_dev || !G_dev) return fail(ctx, EOFA_EINVAL, "null argument");
    try {
        launch_force(ctx, k, chiL_dev, chiR_dev, G_dev, 1, (cudaStream_t)stream);
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return EOFA_OK;
}

int eofa_force_dev(eofa_ctx* ctx, int Ls, double alpha, double M5, double m1, double m2, int precision, double tol,
                   const double* phi_dev, double* F_dev, double* S, eofa_solve_info info[2], void* stream) {
    if (!ctx || !phi_dev || !F_dev) return fail(ctx, EOFA_EINVAL, "null argument");
    eofa_solve_info loc[2];
    if (!info) info = loc;
    cudaStream_t st = (cudaStream_t)stream;
    try {
        int rc = EOFA_OK;
        ChiBufs c = eofa_chis(ctx, Ls, alpha, M5, m1, m2, precision, tol, phi_dev, S, info, st, &rc);
        launch_force(ctx, eofa_k(Ls, alpha, m1, m2), c.chiL, c.chiR, F_dev, 0, st);
        EOFA_CUDA(cudaStreamSynchronize(st));
        return rc;
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
}

int eofa_force_parts_dev(eofa_ctx* ctx, int Ls, double alpha, double M5, double m1, double m2, int precision,
                         double tol, const double* phi_dev, double* FL_dev, double* FR_dev, eofa_solve_info info[2],
                         void* stream) {
    if (!ctx || !phi_dev || (!FL_dev && !FR_dev)) return fail(ctx, EOFA_EINVAL, "null argument");
    eofa_solve_info loc[2];
    if (!info) info = loc;
    cudaStream_t st = (cudaStream_t)stream;
    try {
        int rc = EOFA_OK;
        const int parts = (FL_dev ? 1 : 0) | (FR_dev ? 2 : 0);
        ChiBufs c = eofa_chis(ctx, Ls, alpha, M5, m1, m2, precision, tol, phi_dev, nullptr, info, st, &rc, nullptr,
                              nullptr, parts);
        const double k = eofa_k(Ls, alpha, m1, m2);
        if (FL_dev) launch_force(ctx, k, c.chiL, nullptr, FL_dev, 0, st);
        if (FR_dev) launch_force(ctx, k, nullptr, c.chiR, FR_dev, 0, st);
        EOFA_CUDA(cudaStreamSynchronize(st));
        return rc;
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
}

int eofa_force(eofa_ctx* ctx, int Ls, double alpha, double M5, double m1, double m2, int precision, double tol,
               const double* phi, double* F, double* S, eofa_solve_info info[2]) {
    if (!ctx || !phi || !F) return fail(ctx, EOFA_EINVAL, "null argument");
    try {
        size_t b4 = (size_t)ctx->V * 12 * 16;
        size_t bf = (size_t)ctx->V * 4 * 9 * 16;
        double* dphi = (double*)ctx_buffer(ctx, "host_phi", b4);
        double* dF = (double*)ctx_buffer(ctx, "host_F", bf);
        EOFA_CUDA(cudaMemcpyAsync(dphi, phi, b4, cudaMemcpyHostToDevice, ctx->stream));
        int rc = eofa_force_dev(ctx, Ls, alpha, M5, m1, m2, precision, tol, dphi, dF, S, info, ctx->stream);
        if (rc == EOFA_OK || rc == EOFA_ENOTCONV) {
            EOFA_CUDA(cudaMemcpyAsync(F, dF, bf, cudaMemcpyDeviceToHost, ctx->stream));
            EOFA_CUDA(cudaStreamSynchronize(ctx->stream));
        }
        return rc;
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
}

int eofa_link_update_dev(eofa_ctx* ctx, double eps, const double* P_dev, double* U_dev, void* stream) {
    if (!ctx || !P_dev) return fail(ctx, EOFA_EINVAL, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    try {
        require_gauge(ctx);
        double* Uc = (double*)ctx_buffer(ctx, "U", 0);
        long long nl = 4LL * ctx->V;
        link_update_kernel<<<nblk(nl, 128), 128, 0, st>>>(nl, eps, (const double2*)P_dev, (double2*)Uc, (double2*)U_dev);
        EOFA_LAUNCHED();
        launch_gauge_pack(ctx, Uc, st);
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return EOFA_OK;
}

}  // extern "C"
