// Host-side construction of the 5D-local operator descriptors.
//
// Eq. (3): D_DWF = D_w D-tilde + (1 - L) with D-tilde = d(1 - L) + c(1 + L)
// = b + c5 L (b = c + d, c5 = c - d).  Writing D_w = (4 - M5) + D_hop gives
// D_DWF = D_hop D-tilde + M with the 5D-local M = (4 - M5) D-tilde + 1 - L,
// and D_EOFA = D_DWF D-tilde^{-1} = D_hop + G with G = M D-tilde^{-1}.  The
// EOFA systems of Eq. (8), multiplied by R_5 gamma_5, read
//   (D_hop + G + a chi k (R_5 Omega_chi) Omega_chi^T P_chi) psi = R_5 gamma_5 phi,
// so every solve is an even-odd solve of D_hop + G' with a 5D-local G'.
#include "ops.h"

#include <cmath>

namespace {

typedef std::vector<double> Mat;

Mat bidiag(int Ls, double p, double q, int dir, double mass) {
    Mat A(Ls * Ls, 0.0);
    for (int s = 0; s < Ls; s++) A[s * Ls + s] = p;
    if (dir == 0) {  // L_+: (L y)_s = y_{s-1}, (L y)_0 = -mass y_{Ls-1}
        for (int s = 1; s < Ls; s++) A[s * Ls + s - 1] += q;
        A[0 * Ls + Ls - 1] += -q * mass;
    } else {  // L_- = L_+^T
        for (int s = 0; s + 1 < Ls; s++) A[s * Ls + s + 1] += q;
        A[(Ls - 1) * Ls + 0] += -q * mass;
    }
    return A;
}

Mat matmul(const Mat& A, const Mat& B, int n) {
    Mat C(n * n, 0.0);
    for (int i = 0; i < n; i++)
        for (int k = 0; k < n; k++)
            for (int j = 0; j < n; j++) C[i * n + j] += A[i * n + k] * B[k * n + j];
    return C;
}

Mat transpose(const Mat& A, int n) {
    Mat T(n * n);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) T[j * n + i] = A[i * n + j];
    return T;
}

// Gauss-Jordan inverse with partial pivoting
Mat inverse(Mat A, int n) {
    Mat I(n * n, 0.0);
    for (int i = 0; i < n; i++) I[i * n + i] = 1.0;
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++)
            if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0.0) throw eofa_error(EOFA_EINVAL, "singular 5D-local block (check alpha, M5, mass)");
        if (piv != c)
            for (int j = 0; j < n; j++) {
                std::swap(A[c * n + j], A[piv * n + j]);
                std::swap(I[c * n + j], I[piv * n + j]);
            }
        double d = 1.0 / A[c * n + c];
        for (int j = 0; j < n; j++) { A[c * n + j] *= d; I[c * n + j] *= d; }
        for (int r = 0; r < n; r++) {
            if (r == c) continue;
            double f = A[r * n + c];
            if (f == 0.0) continue;
            for (int j = 0; j < n; j++) { A[r * n + j] -= f * A[c * n + j]; I[r * n + j] -= f * I[c * n + j]; }
        }
    }
    return I;
}

std::vector<double> matvec(const Mat& A, const std::vector<double>& x, int n) {
    std::vector<double> y(n, 0.0);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) y[i] += A[i * n + j] * x[j];
    return y;
}

double dotv(const std::vector<double>& a, const std::vector<double>& b) {
    double s = 0;
    for (size_t i = 0; i < a.size(); i++) s += a[i] * b[i];
    return s;
}

// chirality h (0: P_+ -> L_+ shape, 1: P_- -> L_- shape), optionally transposed
inline int dir_of(int h, int transpose) { return h ^ transpose; }

void upload(eofa_ctx* ctx, int slot, const std::vector<double>& v, cudaStream_t st) {
    EOFA_CUDA(cudaMemcpyAsync(ctx->coef + (size_t)slot * EOFA_MAX_LS, v.data(), v.size() * sizeof(double),
                              cudaMemcpyHostToDevice, st));
}

Op5 op_base() {
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

}  // namespace

Op5 op_finalize(Op5 op, int Ls) {
    for (int h = 0; h < 2; h++) {
        if (op.inv[h]) {
            op.mr[h] = -op.q1[h] / op.p1[h];
            op.invp[h] = 1.0 / op.p1[h];
            op.invN[h] = 1.0 / (op.p1[h] * (1.0 + op.mass * std::pow(op.mr[h], Ls)));
        } else {
            op.mr[h] = op.invp[h] = op.invN[h] = 0.0;
        }
    }
    return op;
}

Coeffs make_coeffs(double alpha, double M5, double m) {
    Coeffs k;
    double c = 0.5 * alpha, d = 0.5;
    k.b = c + d;
    k.c5 = c - d;
    k.p = (4.0 - M5) * k.b + 1.0;
    k.q = (4.0 - M5) * k.c5 - 1.0;
    k.mass = m;
    return k;
}

double eofa_k(int Ls, double alpha, double m1, double m2) {
    double c = 0.5 * alpha, d = 0.5;
    double beta = -(c - d) / (c + d);
    double bL = std::pow(beta, Ls);
    return alpha * (m2 - m1) / ((1.0 + m1 * bL) * (1.0 + m2 * bL));
}

void eofa_omega(int Ls, double alpha, double* Op, double* Om) {
    double c = 0.5 * alpha, d = 0.5;
    double b = c + d, beta = -(c - d) / b;
    for (int s = 0; s < Ls; s++) {
        if (Op) Op[s] = std::pow(beta, Ls - 1 - s) / b;
        if (Om) Om[s] = std::pow(beta, s) / b;
    }
}

System5 system_dwf(double alpha, double M5, double mf) {
    System5 S;
    S.c = make_coeffs(alpha, M5, mf);
    S.r1_h = -1;
    S.sg = 0.0;
    return S;
}

System5 system_eofa(int Ls, double alpha, double M5, double m1, double m2, int which, double a) {
    System5 S;
    bool left = which == EOFA_SYS_EOFA_L;
    S.c = make_coeffs(alpha, M5, left ? m1 : m2);
    S.r1_h = -1;
    S.sg = 0.0;
    if (a != 0.0) {
        std::vector<double> Op(Ls), Om(Ls);
        eofa_omega(Ls, alpha, Op.data(), Om.data());
        const std::vector<double>& Om_chi = left ? Om : Op;
        double chi = left ? -1.0 : 1.0;
        S.r1_h = left ? 1 : 0;
        S.sg = a * chi * eofa_k(Ls, alpha, m1, m2);
        S.v = Om_chi;
        S.w.resize(Ls);
        for (int s = 0; s < Ls; s++) S.w[s] = Om_chi[Ls - 1 - s];  // R_5 Omega
    }
    return S;
}

Op5 op_plain(const Coeffs& c, int inv_which, int fwd_which, int transpose) {
    Op5 op = op_base();
    op.mass = c.mass;
    for (int h = 0; h < 2; h++) {
        if (inv_which) {
            op.inv[h] = 1;
            op.p1[h] = inv_which == 1 ? c.b : c.p;
            op.q1[h] = inv_which == 1 ? c.c5 : c.q;
            op.dir1[h] = dir_of(h, transpose);
        }
        if (fwd_which) {
            op.fwd[h] = 1;
            op.p2[h] = fwd_which == 1 ? c.b : c.p;
            op.q2[h] = fwd_which == 1 ? c.c5 : c.q;
            op.dir2[h] = dir_of(h, transpose);
        }
    }
    return op;
}

// G' = M D-tilde^{-1} + sg w v^T:  u = D-tilde^{-1} x, out = M u + sg w ((D-tilde^T v) . u)
Op5 op_G(eofa_ctx* ctx, const System5& S, int slot, cudaStream_t st) {
    Op5 op = op_plain(S.c, 1, 2, 0);
    if (S.r1_h >= 0) {
        int Ls = ctx->Ls, h = S.r1_h;
        Mat Dt = bidiag(Ls, S.c.b, S.c.c5, dir_of(h, 0), S.c.mass);
        std::vector<double> vd = matvec(transpose(Dt, Ls), S.v, Ls);
        upload(ctx, slot, S.w, st);
        upload(ctx, slot + 1, vd, st);
        op.sigma[h] = S.sg;
        op.w[h] = ctx->coef + (size_t)slot * EOFA_MAX_LS;
        op.v[h] = ctx->coef + (size_t)(slot + 1) * EOFA_MAX_LS;
    }
    return op;
}

// G'^{-1} by Sherman-Morrison: G'^{-1} x = G^{-1} x + sm (G^{-1} w) (v^T G^{-1} x),
// sm = -sg / (1 + sg v^T G^{-1} w), G^{-1} = D-tilde M^{-1}.
Op5 op_Ginv(eofa_ctx* ctx, const System5& S, int slot, cudaStream_t st) {
    Op5 op = op_plain(S.c, 2, 1, 0);
    if (S.r1_h >= 0) {
        int Ls = ctx->Ls, h = S.r1_h;
        Mat Dt = bidiag(Ls, S.c.b, S.c.c5, dir_of(h, 0), S.c.mass);
        Mat M = bidiag(Ls, S.c.p, S.c.q, dir_of(h, 0), S.c.mass);
        Mat Gi = matmul(Dt, inverse(M, Ls), Ls);
        std::vector<double> Giw = matvec(Gi, S.w, Ls);
        double den = 1.0 + S.sg * dotv(S.v, Giw);
        if (den == 0.0) throw eofa_error(EOFA_EINVAL, "EOFA system is singular for this shift");
        std::vector<double> vd = matvec(transpose(Dt, Ls), S.v, Ls);
        upload(ctx, slot, Giw, st);
        upload(ctx, slot + 1, vd, st);
        op.sigma[h] = -S.sg / den;
        op.w[h] = ctx->coef + (size_t)slot * EOFA_MAX_LS;
        op.v[h] = ctx->coef + (size_t)(slot + 1) * EOFA_MAX_LS;
    }
    return op;
}

// (G'^{-1})^T x = G^{-T} x + sm (G^{-T} v) (w^T G^{-T} x),  G^{-T} = D-tilde^T M^{-T}:
// u = M^{-T} x, out = D-tilde^T u + sm (G^{-T} v) ((D-tilde w) . u)
Op5 op_GinvT(eofa_ctx* ctx, const System5& S, int slot, cudaStream_t st) {
    Op5 op = op_plain(S.c, 2, 1, 1);
    if (S.r1_h >= 0) {
        int Ls = ctx->Ls, h = S.r1_h;
        Mat Dt = bidiag(Ls, S.c.b, S.c.c5, dir_of(h, 0), S.c.mass);
        Mat M = bidiag(Ls, S.c.p, S.c.q, dir_of(h, 0), S.c.mass);
        Mat Gi = matmul(Dt, inverse(M, Ls), Ls);
        double den = 1.0 + S.sg * dotv(S.v, matvec(Gi, S.w, Ls));
        if (den == 0.0) throw eofa_error(EOFA_EINVAL, "EOFA system is singular for this shift");
        std::vector<double> GiTv = matvec(transpose(Gi, Ls), S.v, Ls);
        std::vector<double> Dw = matvec(Dt, S.w, Ls);
        upload(ctx, slot, GiTv, st);
        upload(ctx, slot + 1, Dw, st);
        op.sigma[h] = -S.sg / den;
        op.w[h] = ctx->coef + (size_t)slot * EOFA_MAX_LS;
        op.v[h] = ctx->coef + (size_t)(slot + 1) * EOFA_MAX_LS;
    }
    return op;
}
