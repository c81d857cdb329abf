// Rational approximation x^{-1/2} ~ alpha_0 + sum_l alpha_l / (x + beta_l) on
// [lmin, lmax] for the EOFA heatbath (Sec. 3.2, Eq. (6)).
//
// Zolotarev's optimal (n, n) relative approximation of 1/sqrt(y) on [1, b]
// (b = lmax / lmin): with the modulus k' = sqrt(1 - 1/b), K' = K(k') and
//   c_l = sn^2(l K' / (2n + 1); k') / cn^2(l K' / (2n + 1); k'),  l = 1 .. 2n,
// the approximant is D prod_{l=1}^{n} (y + c_{2l}) / (y + c_{2l-1}), D fixing
// the equioscillating relative error.  K, sn and cn come from the
// arithmetic-geometric mean and the descending Landen transformation
// (Abramowitz and Stegun 17.6 and 16.4).  Partial fractions give alpha_0,
// alpha_l, beta_l, rescaled from [1, b] to [lmin, lmax].
#include "api_util.h"

#include <cmath>
#include <vector>

namespace {

double ellipK(double k) {
    double a = 1.0, b = std::sqrt(1.0 - k * k);
    for (int i = 0; i < 60 && std::fabs(a - b) > 1e-16 * a; i++) {
        double an = 0.5 * (a + b);
        b = std::sqrt(a * b);
        a = an;
    }
    return M_PI / (2.0 * a);
}

void sncn(double u, double k, double* sn, double* cn) {
    double a[64], c[64];
    a[0] = 1.0;
    double b = std::sqrt(1.0 - k * k);
    c[0] = k;
    int N = 0;
    while (std::fabs(c[N]) > 1e-16 && N < 62) {
        a[N + 1] = 0.5 * (a[N] + b);
        c[N + 1] = 0.5 * (a[N] - b);
        b = std::sqrt(a[N] * b);
        N++;
    }
    double phi = std::ldexp(a[N] * u, N);
    for (int i = N; i > 0; i--) phi = 0.5 * (phi + std::asin(c[i] * std::sin(phi) / a[i]));
    *sn = std::sin(phi);
    *cn = std::cos(phi);
}

}  // namespace

extern "C" int eofa_rational_inv_sqrt(int npoles, double lmin, double lmax, double* alpha0, double* alpha,
                                      double* beta, double* max_rel_err) {
    if (npoles < 1 || npoles > 64 || !(lmin > 0) || !(lmax > lmin) || !alpha0 || !alpha || !beta) return EOFA_EINVAL;
    const int n = npoles;
    const double bnd = lmax / lmin;
    const double kp = std::sqrt(1.0 - 1.0 / bnd);
    const double Kp = ellipK(kp);
    std::vector<double> c(2 * n + 1);
    for (int l = 1; l <= 2 * n; l++) {
        double sn, cn;
        sncn(l * Kp / (2 * n + 1), kp, &sn, &cn);
        c[l] = sn * sn / (cn * cn);
    }
    auto R = [&](double y) {
        double r = 1.0;
        for (int l = 1; l <= n; l++) r *= (y + c[2 * l]) / (y + c[2 * l - 1]);
        return r;
    };
    // extremes of sqrt(y) R(y) on [1, b] (log-spaced scan refined around the extrema)
    double mn = 1e300, mx = -1e300;
    const int NS = 20000;
    for (int i = 0; i <= NS; i++) {
        double y = std::exp(std::log(bnd) * i / NS);
        double v = std::sqrt(y) * R(y);
        mn = std::fmin(mn, v);
        mx = std::fmax(mx, v);
    }
    const double D = 2.0 / (mn + mx);
    if (max_rel_err) *max_rel_err = (mx - mn) / (mx + mn);
    // partial fractions of D prod (y + c_2l) / (y + c_2l-1)
    const double sq = std::sqrt(lmin);
    *alpha0 = D / sq;
    for (int l = 1; l <= n; l++) {
        double A = 1.0;
        for (int m = 1; m <= n; m++) A *= (c[2 * m] - c[2 * l - 1]);
        for (int m = 1; m <= n; m++)
            if (m != l) A /= (c[2 * m - 1] - c[2 * l - 1]);
        alpha[l - 1] = D * A * sq;  // x = lmin y: A / (y + c) = A lmin / (x + lmin c)
        beta[l - 1] = lmin * c[2 * l - 1];
    }
    return EOFA_OK;
}
