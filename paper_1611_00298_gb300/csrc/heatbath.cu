// EOFA heatbath (Sec. 3.2, Eq. (6)): phi = f(M_EOFA) eta for a rational
// f(x) = alpha_0 + sum_l alpha_l / (x + beta_l) ~ x^{-1/2}.  With
// gamma_l = 1 / (1 + beta_l),
//   phi = alpha_0 eta + sum_l alpha_l gamma_l [eta + k gamma_l P_- Omega_-^+ psi_L,l
//                                                  - k gamma_l P_+ Omega_+^+ psi_R,l],
//   (H(m1) - gamma_l Delta_- P_-) psi_L,l = Omega_- P_- eta,
//   (H(m2) - gamma_l beta_l Delta_+ P_+) psi_R,l = Omega_+ P_+ eta,
// i.e. 2 N_p solves of Eq. (8).  Initial guesses (Sec. 5.2) come from the
// chronological method: the earlier solutions chi_i of the same family span
// the guess x0 = sum_i c_i chi_i with c minimising |b - A x0| (A the new
// system), a small least-squares problem built from <A chi_i, A chi_j> and
// <A chi_i, b>.
#include "api_util.h"

#include <cmath>
#include <complex>

#define HB_HIST 6

namespace {

inline unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

// out(i, c) += coef sum_s Om[s] psi(s, i, c) on the components of one chirality
__global__ void contract_kernel(long long V12, int Ls, const double2* __restrict__ psi, const double* __restrict__ Om,
                                int chi, double coef, double2* out) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= V12) return;
    int c = (int)(t % 12);
    bool keep = chi > 0 ? (c < 6) : (c >= 6);
    if (!keep) return;
    double re = 0, im = 0;
    for (int s = 0; s < Ls; s++) {
        double2 z = psi[(long long)s * V12 + t];
        re += Om[s] * z.x;
        im += Om[s] * z.y;
    }
    double2 o = out[t];
    out[t] = make_double2(o.x + coef * re, o.y + coef * im);
}

// y = a x + b y (real a, b) on flat complex arrays
__global__ void flat_axpby_kernel(long long n, double a, const double2* __restrict__ x, double b, double2* y) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= n) return;
    double2 u = x[t], v = y[t];
    y[t] = make_double2(a * u.x + b * v.x, a * u.y + b * v.y);
}

// y += (cr + i ci) x on flat complex arrays
__global__ void flat_caxpy_kernel(long long n, double cr, double ci, const double2* __restrict__ x, double2* y) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= n) return;
    double2 u = x[t], v = y[t];
    y[t] = make_double2(v.x + cr * u.x - ci * u.y, v.y + cr * u.y + ci * u.x);
}

// out = (H(m) + a Delta P) x on canonical 5D fields: gamma5 R5 (D_hop + G') x
void system_apply(eofa_ctx* ctx, const System5& S, const double* x, double* out, cudaStream_t st) {
    const size_t f64 = field_bytes(P64, ctx->Vh, ctx->Ls);
    void* xe = ctx_buffer(ctx, "hb_xe", f64);
    void* xo = ctx_buffer(ctx, "hb_xo", f64);
    void* ye = ctx_buffer(ctx, "hb_ye", f64);
    void* yo = ctx_buffer(ctx, "hb_yo", f64);
    double* tmp = (double*)ctx_buffer(ctx, "hb_tmp", (size_t)ctx->V * ctx->Ls * 12 * 16);
    double* saved = ctx->coef;
    ctx->coef = (double*)ctx_buffer(ctx, "coef_hb", 16 * EOFA_MAX_LS * sizeof(double));
    Op5 G = op_G(ctx, S, 4, st);
    ctx->coef = saved;
    launch_pack(ctx, P64, x, xe, xo, st);
    apply_eofa_fields(ctx, G, xe, xo, ye, yo, st);
    launch_unpack(ctx, P64, ye, yo, tmp, st);
    launch_rs5(ctx, tmp, out, st);
}

std::complex<double> cdot(eofa_ctx* ctx, long long n, const double* a, const double* b, cudaStream_t st) {
    blas_flat_dot(ctx, n, a, b, 14, st);
    double v[2];
    red_fetch_many(ctx, 14, 2, v, st);
    return {v[0], v[1]};
}

// Solve G c = r (m x m complex) by Gaussian elimination with partial pivoting;
// false when the Gram matrix is numerically singular (a pivot below 1e-13 of
// the largest diagonal entry).
bool small_solve(std::vector<std::complex<double>> G, std::vector<std::complex<double>>& r, int m) {
    double scale = 0;
    for (int i = 0; i < m; i++) scale = std::fmax(scale, std::abs(G[i * m + i]));
    for (int c = 0; c < m; c++) {
        int piv = c;
        for (int i = c + 1; i < m; i++)
            if (std::abs(G[i * m + c]) > std::abs(G[piv * m + c])) piv = i;
        if (std::abs(G[piv * m + c]) <= 1e-13 * scale) return false;
        if (piv != c) {
            for (int j = 0; j < m; j++) std::swap(G[c * m + j], G[piv * m + j]);
            std::swap(r[c], r[piv]);
        }
        for (int i = c + 1; i < m; i++) {
            std::complex<double> f = G[i * m + c] / G[c * m + c];
            for (int j = c; j < m; j++) G[i * m + j] -= f * G[c * m + j];
            r[i] -= f * r[c];
        }
    }
    for (int i = m - 1; i >= 0; i--) {
        for (int j = i + 1; j < m; j++) r[i] -= G[i * m + j] * r[j];
        r[i] /= G[i * m + i];
    }
    return true;
}

}  // namespace

extern "C" int eofa_heatbath_dev(eofa_ctx* ctx, int Ls, double alpha, double M5, double m1, double m2, int precision,
                                 double tol, int npoles, double alpha0, const double* alphas, const double* betas,
                                 const double* eta_dev, double* phi_dev, int forecast, eofa_solve_info* info,
                                 void* stream) {
    if (!ctx || npoles < 1 || !alphas || !betas || !eta_dev || !phi_dev) return fail(ctx, EOFA_EINVAL, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    try {
        check_ls(ctx, Ls);
        require_gauge(ctx);
        if (!(m1 < m2)) throw eofa_error(EOFA_EINVAL, "EOFA needs m1 < m2 (k > 0)");
        for (int l = 0; l < npoles; l++)
            if (!(betas[l] > 0)) throw eofa_error(EOFA_EINVAL, "heatbath poles beta_l must be positive");
        const long long V12 = 12LL * ctx->V;
        const long long n5 = V12 * Ls;
        const size_t b5 = (size_t)n5 * 16;
        double* om = (double*)ctx_buffer(ctx, "hb_omega", 2 * EOFA_MAX_LS * sizeof(double));
        std::vector<double> Op(Ls), Om(Ls);
        eofa_omega(Ls, alpha, Op.data(), Om.data());
        EOFA_CUDA(cudaMemcpyAsync(om, Op.data(), Ls * sizeof(double), cudaMemcpyHostToDevice, st));
        EOFA_CUDA(cudaMemcpyAsync(om + EOFA_MAX_LS, Om.data(), Ls * sizeof(double), cudaMemcpyHostToDevice, st));
        const double k = eofa_k(Ls, alpha, m1, m2);
        // right-hand sides Omega_-+ P_-+ eta (the same embedding as the action)
        double* bL = (double*)ctx_buffer(ctx, "hb_bL", b5);
        double* bR = (double*)ctx_buffer(ctx, "hb_bR", b5);
        eofa_embed(ctx, eta_dev, om + EOFA_MAX_LS, -1, bL, st);
        eofa_embed(ctx, eta_dev, om, +1, bR, st);
        // phi = alpha0 eta
        flat_axpby_kernel<<<nblk(V12, 256), 256, 0, st>>>(V12, alpha0, (const double2*)eta_dev, 0.0, (double2*)phi_dev);
        EOFA_LAUNCHED();
        const int hist = forecast ? HB_HIST : 0;
        std::vector<double*> chiL(hist ? npoles : 1), chiR(hist ? npoles : 1), W(hist);
        double* psi = (double*)ctx_buffer(ctx, "hb_psi", b5);
        for (int i = 0; i < hist; i++) W[i] = (double*)ctx_buffer(ctx, "hb_W" + std::to_string(i), b5);
        for (int l = 0; l < npoles; l++) {
            const double g = 1.0 / (1.0 + betas[l]);
            for (int fam = 0; fam < 2; fam++) {  // 0: L (P_-), 1: R (P_+)
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
                p.system = fam == 0 ? EOFA_SYS_EOFA_L : EOFA_SYS_EOFA_R;
                p.shift = fam == 0 ? -g : -g * betas[l];
                const double* b = fam == 0 ? bL : bR;
                std::vector<double*>& prev = fam == 0 ? chiL : chiR;
                // the last HB_HIST solutions of each family are kept in a ring of buffers
                double* x = hist ? (double*)ctx_buffer(ctx, std::string(fam ? "hb_chiR" : "hb_chiL") +
                                                                std::to_string(l % (HB_HIST + 1)), b5)
                                 : psi;
                p.use_x0 = 0;
                const int m = std::min(l, hist);
                if (m > 0) {
                    // chronological guess from the last m solutions of this family
                    System5 S = system_eofa(Ls, alpha, M5, m1, m2, p.system, p.shift);
                    for (int i = 0; i < m; i++) system_apply(ctx, S, prev[l - m + i], W[i], st);
                    std::vector<std::complex<double>> Gm(m * m), r(m);
                    for (int i = 0; i < m; i++) {
                        r[i] = cdot(ctx, n5, W[i], b, st);
                        for (int j = i; j < m; j++) {
                            Gm[i * m + j] = cdot(ctx, n5, W[i], W[j], st);
                            Gm[j * m + i] = std::conj(Gm[i * m + j]);
                        }
                    }
                    // nearly dependent history makes the normal equations singular:
                    // drop the oldest solutions until the system is solvable
                    for (int kk = m; kk >= 1 && !p.use_x0; kk--) {
                        const int o = m - kk;  // first kept vector
                        std::vector<std::complex<double>> Gk(kk * kk), rk(kk);
                        for (int i = 0; i < kk; i++) {
                            rk[i] = r[o + i];
                            for (int j = 0; j < kk; j++) Gk[i * kk + j] = Gm[(o + i) * m + (o + j)];
                        }
                        if (!small_solve(Gk, rk, kk)) continue;
                        EOFA_CUDA(cudaMemsetAsync(x, 0, b5, st));
                        for (int i = 0; i < kk; i++) {
                            flat_caxpy_kernel<<<nblk(n5, 256), 256, 0, st>>>(n5, rk[i].real(), rk[i].imag(),
                                                                             (const double2*)prev[l - kk + i],
                                                                             (double2*)x);
                            EOFA_LAUNCHED();
                        }
                        p.use_x0 = 1;
                    }
                }
                eofa_solve_info inf;
                int rc = solve_dev_impl(ctx, &p, b, x, &inf, st);
                if (info) info[2 * l + fam] = inf;
                if (rc != EOFA_OK) throw eofa_error(rc, "heatbath solve failed: " + ctx->err);
                if (hist) prev[l] = x;
                // phi += alpha_l gamma_l eta (once per pole) +- alpha_l gamma_l^2 k P Omega^+ x
                if (fam == 0) {
                    flat_axpby_kernel<<<nblk(V12, 256), 256, 0, st>>>(V12, alphas[l] * g, (const double2*)eta_dev, 1.0,
                                                                      (double2*)phi_dev);
                    EOFA_LAUNCHED();
                }
                const double coef = (fam == 0 ? 1.0 : -1.0) * alphas[l] * g * g * k;
                contract_kernel<<<nblk(V12, 256), 256, 0, st>>>(V12, Ls, (const double2*)x,
                                                                fam == 0 ? om + EOFA_MAX_LS : om, fam == 0 ? -1 : 1,
                                                                coef, (double2*)phi_dev);
                EOFA_LAUNCHED();
            }
        }
        EOFA_CUDA(cudaStreamSynchronize(st));
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return EOFA_OK;
}
