// Linear solves (Sec. 5.1): even-odd preconditioning, Cayley-factorised
// 5D-local blocks, CG on the normal equations, mixed precision.
//
// Every system is brought to the form (D_hop + G') psi = f with a 5D-local
// G' (see ops.cu).  With even (e) and odd (o) sites,
//   psi_o solves  A psi_o = f^_o,  A = 1 - G'^{-1} D_oe G'^{-1} D_eo,
//                 f^_o = G'^{-1} (f_o - D_oe G'^{-1} f_e),
//   psi_e = G'^{-1} (f_e - D_eo psi_o),
// and the full residual is (0, G' (f^_o - A psi_o)).  A^+ follows from
// D_hop^+ = gamma_5 D_hop gamma_5 and the reality of G' in s:
//   A^+ = 1 - D^dag_oe G'^{-T} D^dag_eo G'^{-T}  (D^dag: hop with swapped projectors).
// CGLS (CG on A^+ A tracking r = f^ - A x) iterates in the inner precision;
// with mixed precision the residual is recomputed in FP64 whenever |r| has
// dropped by the factor delta since the last recomputation (reliable
// updates), and the solution accumulates in FP64.  The stopping test is the
// FP64 true residual of the full, unpreconditioned system.
#include "api_util.h"

#include <chrono>
#include <cmath>

namespace {

struct SchurOps {
    Op5 Gi, GiT;
};

struct Work {
    int prec;   // inner storage precision
    int precx;  // inner solution accumulator precision
    void *p, *q, *r, *s, *x, *te, *te2, *to;
};

// out = A in (odd -> odd), precision w.prec
void apply_A(eofa_ctx* ctx, const SchurOps& o, int prec, const void* in, void* out, void* te, void* te2, cudaStream_t st) {
    launch_hop(ctx, prec, 0, 0, in, te, st);
    launch_op5(ctx, prec, o.Gi, te, nullptr, te2, st);
    launch_hop(ctx, prec, 1, 0, te2, out, st);
    Op5 g = o.Gi;
    g.a_out = -1.0;
    g.b_in = 1.0;
    launch_op5(ctx, prec, g, out, in, out, st);
}

// out = A^+ in; to is an odd temporary
void apply_Adag(eofa_ctx* ctx, const SchurOps& o, int prec, const void* in, void* out, void* te, void* te2, void* to,
                cudaStream_t st) {
    launch_op5(ctx, prec, o.GiT, in, nullptr, to, st);
    launch_hop(ctx, prec, 0, 1, to, te, st);
    launch_op5(ctx, prec, o.GiT, te, nullptr, te2, st);
    launch_hop(ctx, prec, 1, 1, te2, out, st);
    blas_axpby(ctx, prec, 1.0, in, -1.0, out, st);
}

double norm2_now(eofa_ctx* ctx, int prec, const void* x, cudaStream_t st) {
    blas_norm2(ctx, prec, x, 0, st);
    return red_fetch(ctx, 0, st);
}

bool is_finite(double v) { return std::isfinite(v); }

}  // namespace

int solve_dev_impl(eofa_ctx* ctx, const eofa_solve_params* prm, const double* b_dev, double* x_dev,
                   eofa_solve_info* info, cudaStream_t st) {
    auto t0 = std::chrono::steady_clock::now();
    eofa_solve_info inf;
    inf.iters = 0;
    inf.reliable_updates = 0;
    inf.true_resid = -1.0;
    inf.seconds = 0.0;
    inf.status = EOFA_OK;
    const eofa_solve_params& P = *prm;
    check_ls(ctx, P.Ls);
    require_gauge(ctx);
    if (!(P.tol > 0) || P.maxiter < 1 || P.precision < 0 || P.precision > 2 || P.system < 0 || P.system > 2)
        throw eofa_error(EOFA_EINVAL, "bad solve parameters");
    if (P.system != EOFA_SYS_DWF && !(P.m1 < P.m2)) throw eofa_error(EOFA_EINVAL, "EOFA systems need m1 < m2");
    const bool mixed = P.precision != EOFA_PREC_F64;
    const int prec = P.precision == EOFA_PREC_F64 ? P64 : (P.precision == EOFA_PREC_MIXED_F32 ? P32 : P16);
    const int precx = mixed ? P32 : P64;
    const double delta = (P.delta > 0 && P.delta < 1) ? P.delta : 0.1;

    System5 S = P.system == EOFA_SYS_DWF ? system_dwf(P.alpha, P.M5, P.mf)
                                         : system_eofa(P.Ls, P.alpha, P.M5, P.m1, P.m2, P.system, P.shift);
    SchurOps ops;
    ops.Gi = op_Ginv(ctx, S, 0, st);
    ops.GiT = op_GinvT(ctx, S, 2, st);
    Op5 G = op_G(ctx, S, 4, st);

    const size_t f64 = field_bytes(P64, ctx->Vh, ctx->Ls);
    const long long n5full = (long long)ctx->V * ctx->Ls * 12;
    double* canon = (double*)ctx_buffer(ctx, "sv_canon", (size_t)n5full * 16);
    void* f_e = ctx_buffer(ctx, "sv_fe", f64);
    void* f_o = ctx_buffer(ctx, "sv_fo", f64);
    void* fh = ctx_buffer(ctx, "sv_fh", f64);
    void* x_e = ctx_buffer(ctx, "sv_xe", f64);
    void* x_o = ctx_buffer(ctx, "sv_xo", f64);
    void* r64 = ctx_buffer(ctx, "sv_r64", f64);
    void* a_e = ctx_buffer(ctx, "sv_ae", f64);
    void* a_e2 = ctx_buffer(ctx, "sv_ae2", f64);
    void* a_o = ctx_buffer(ctx, "sv_ao", f64);

    // right-hand side of (D_hop + G') psi = f
    const double* fsrc = b_dev;
    if (P.system != EOFA_SYS_DWF) {
        launch_rs5(ctx, b_dev, canon, st);  // f = R5 gamma5 b
        fsrc = canon;
    }
    launch_pack(ctx, P64, fsrc, f_e, f_o, st);
    double fnorm2 = norm2_now(ctx, P64, f_e, st) + norm2_now(ctx, P64, f_o, st);
    if (!is_finite(fnorm2)) throw eofa_error(EOFA_ENUMERIC, "right-hand side has NaN/Inf");
    if (fnorm2 == 0.0) {
        EOFA_CUDA(cudaMemsetAsync(x_dev, 0, (size_t)n5full * 16, st));
        EOFA_CUDA(cudaStreamSynchronize(st));
        inf.true_resid = 0.0;
        if (info) *info = inf;
        return EOFA_OK;
    }
    // initial guess
    if (P.use_x0) {
        launch_pack(ctx, P64, x_dev, x_e, x_o, st);
        if (P.system == EOFA_SYS_DWF) {  // iterate on y = D-tilde psi
            Op5 Dt = op_plain(S.c, 0, 1, 0);
            launch_op5(ctx, P64, Dt, x_o, nullptr, x_o, st);
        }
    } else {
        blas_zero(ctx, P64, x_o, st);
    }
    // f^_o = G'^{-1} (f_o - D_oe G'^{-1} f_e)
    launch_op5(ctx, P64, ops.Gi, f_e, nullptr, a_e, st);
    launch_hop(ctx, P64, 1, 0, a_e, a_o, st);
    blas_axpby(ctx, P64, 1.0, f_o, -1.0, a_o, st);
    launch_op5(ctx, P64, ops.Gi, a_o, nullptr, fh, st);
    const double fhn = std::sqrt(norm2_now(ctx, P64, fh, st));

    // inner work fields
    Work w;
    w.prec = prec;
    w.precx = precx;
    const size_t fbi = field_bytes(prec, ctx->Vh, ctx->Ls);
    std::string tag = "_" + std::to_string(prec);
    w.p = ctx_buffer(ctx, "sv_p" + tag, fbi);
    w.q = ctx_buffer(ctx, "sv_q" + tag, fbi);
    w.r = ctx_buffer(ctx, "sv_r" + tag, fbi);
    w.s = ctx_buffer(ctx, "sv_s" + tag, fbi);
    w.te = ctx_buffer(ctx, "sv_te" + tag, fbi);
    w.te2 = ctx_buffer(ctx, "sv_te2" + tag, fbi);
    w.to = ctx_buffer(ctx, "sv_to" + tag, fbi);
    w.x = mixed ? ctx_buffer(ctx, "sv_x32", field_bytes(P32, ctx->Vh, ctx->Ls)) : x_o;

    double target_rel = 0.5 * P.tol;  // on |r| / |f^|, refined by the true-residual check
    int restarts = 0;
    double true_rel = 1.0;
    for (;;) {
        // r64 = f^ - A x_o  (FP64)
        apply_A(ctx, ops, P64, x_o, r64, a_e, a_e2, st);
        blas_axpby(ctx, P64, 1.0, fh, -1.0, r64, st);
        double rr = norm2_now(ctx, P64, r64, st);
        if (!is_finite(rr)) throw eofa_error(EOFA_ENUMERIC, "NaN/Inf in the residual");
        double target = target_rel * fhn;
        if (mixed) {
            blas_copy(ctx, prec, w.r, P64, r64, st);
            blas_zero(ctx, precx, w.x, st);
        } else {
            blas_copy(ctx, P64, w.r, P64, r64, st);
        }
        double rmax = std::sqrt(rr);
        if (std::sqrt(rr) > target) {
            apply_Adag(ctx, ops, prec, w.r, w.s, w.te, w.te2, w.to, st);
            blas_copy(ctx, prec, w.p, prec, w.s, st);
            double gam = norm2_now(ctx, prec, w.s, st);
            while (inf.iters < P.maxiter) {
                apply_A(ctx, ops, prec, w.p, w.q, w.te, w.te2, st);
                double dl = norm2_now(ctx, prec, w.q, st);
                if (!is_finite(dl) || !is_finite(gam)) throw eofa_error(EOFA_ENUMERIC, "NaN/Inf in CG");
                if (dl == 0.0) break;
                double alpha = gam / dl;
                blas_cg_update(ctx, prec, precx, alpha, w.p, w.q, w.x, w.r, 2, st);
                apply_Adag(ctx, ops, prec, w.r, w.s, w.te, w.te2, w.to, st);
                blas_norm2(ctx, prec, w.s, 4, st);
                double vals[3];
                red_fetch_many(ctx, 2, 3, vals, st);
                rr = vals[0];
                double gnew = vals[2];
                inf.iters++;
                if (!is_finite(rr)) throw eofa_error(EOFA_ENUMERIC, "NaN/Inf in CG");
                if (mixed && (std::sqrt(rr) < delta * rmax || std::sqrt(rr) < target || inf.iters >= P.maxiter)) {
                    // reliable update: accumulate x in FP64, recompute r in FP64
                    blas_copy(ctx, P64, a_o, precx, w.x, st);
                    blas_axpby(ctx, P64, 1.0, a_o, 1.0, x_o, st);
                    blas_zero(ctx, precx, w.x, st);
                    apply_A(ctx, ops, P64, x_o, r64, a_e, a_e2, st);
                    blas_axpby(ctx, P64, 1.0, fh, -1.0, r64, st);
                    rr = norm2_now(ctx, P64, r64, st);
                    inf.reliable_updates++;
                    rmax = std::sqrt(rr);
                    if (std::sqrt(rr) < target) break;
                    blas_copy(ctx, prec, w.r, P64, r64, st);
                    apply_Adag(ctx, ops, prec, w.r, w.s, w.te, w.te2, w.to, st);
                    gnew = norm2_now(ctx, prec, w.s, st);
                } else if (!mixed && std::sqrt(rr) < target) {
                    break;
                }
                double beta = gnew / gam;
                gam = gnew;
                blas_axpby(ctx, prec, 1.0, w.s, beta, w.p, st);
            }
            if (mixed) {
                blas_copy(ctx, P64, a_o, precx, w.x, st);
                blas_axpby(ctx, P64, 1.0, a_o, 1.0, x_o, st);
                blas_zero(ctx, precx, w.x, st);
            }
        }
        // reconstruct psi_e = G'^{-1} (f_e - D_eo psi_o)
        launch_hop(ctx, P64, 0, 0, x_o, a_e, st);
        blas_axpby(ctx, P64, 1.0, f_e, -1.0, a_e, st);
        launch_op5(ctx, P64, ops.Gi, a_e, nullptr, x_e, st);
        // true residual of the full system
        if (P.system == EOFA_SYS_DWF) {
            // psi = D-tilde^{-1} y, residual b - D_DWF psi
            Op5 Dti = op_plain(S.c, 1, 0, 0);
            void* pe = ctx_buffer(ctx, "sv_pe", f64);
            void* po = ctx_buffer(ctx, "sv_po", f64);
            launch_op5(ctx, P64, Dti, x_e, nullptr, pe, st);
            launch_op5(ctx, P64, Dti, x_o, nullptr, po, st);
            void* re = ctx_buffer(ctx, "sv_re", f64);
            void* ro = ctx_buffer(ctx, "sv_ro", f64);
            apply_dwf_fields(ctx, S.c, 0, pe, po, re, ro, st);
            blas_axpby(ctx, P64, 1.0, f_e, -1.0, re, st);
            blas_axpby(ctx, P64, 1.0, f_o, -1.0, ro, st);
            double res2 = norm2_now(ctx, P64, re, st) + norm2_now(ctx, P64, ro, st);
            true_rel = std::sqrt(res2 / fnorm2);
            if (true_rel <= P.tol || inf.iters >= P.maxiter || restarts >= 8 || !is_finite(true_rel)) {
                launch_unpack(ctx, P64, pe, po, x_dev, st);
                break;
            }
        } else {
            void* re = ctx_buffer(ctx, "sv_re", f64);
            void* ro = ctx_buffer(ctx, "sv_ro", f64);
            apply_eofa_fields(ctx, G, x_e, x_o, re, ro, st);
            blas_axpby(ctx, P64, 1.0, f_e, -1.0, re, st);
            blas_axpby(ctx, P64, 1.0, f_o, -1.0, ro, st);
            double res2 = norm2_now(ctx, P64, re, st) + norm2_now(ctx, P64, ro, st);
            true_rel = std::sqrt(res2 / fnorm2);
            if (true_rel <= P.tol || inf.iters >= P.maxiter || restarts >= 8 || !is_finite(true_rel)) {
                launch_unpack(ctx, P64, x_e, x_o, x_dev, st);
                break;
            }
        }
        // not yet: tighten the inner target by the observed ratio and restart
        double rr_now = norm2_now(ctx, P64, r64, st);
        double ratio = std::sqrt(rr_now) / fhn / (true_rel > 0 ? true_rel : 1e-300);
        double nt = 0.5 * P.tol * ratio;
        target_rel = nt < 0.5 * target_rel ? nt : 0.5 * target_rel;
        restarts++;
    }
    EOFA_CUDA(cudaStreamSynchronize(st));
    inf.true_resid = true_rel;
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (!is_finite(true_rel)) inf.status = EOFA_ENUMERIC;
    else if (true_rel > P.tol) inf.status = EOFA_ENOTCONV;
    if (info) *info = inf;
    if (inf.status != EOFA_OK) {
        ctx->err = inf.status == EOFA_ENOTCONV ? "solver did not reach tol (true residual " + std::to_string(true_rel) + ")"
                                               : "NaN/Inf in the solution";
    }
    return inf.status;
}

extern "C" {

int eofa_solve_dev(eofa_ctx* ctx, const eofa_solve_params* p, const double* b_dev, double* x_dev, eofa_solve_info* info,
                   void* stream) {
    if (!ctx || !p || !b_dev || !x_dev) return fail(ctx, EOFA_EINVAL, "null argument");
    try {
        return solve_dev_impl(ctx, p, b_dev, x_dev, info, (cudaStream_t)stream);
    } catch (const eofa_error& e) {
        if (info) info->status = e.code;
        return fail(ctx, e.code, e.msg);
    }
}

int eofa_solve(eofa_ctx* ctx, const eofa_solve_params* p, const double* b, double* x, eofa_solve_info* info) {
    if (!ctx || !p || !b || !x) return fail(ctx, EOFA_EINVAL, "null argument");
    try {
        size_t bytes = (size_t)ctx->V * ctx->Ls * 12 * 16;
        double* db = (double*)ctx_buffer(ctx, "host_in", bytes);
        double* dx = (double*)ctx_buffer(ctx, "host_out", bytes);
        EOFA_CUDA(cudaMemcpyAsync(db, b, bytes, cudaMemcpyHostToDevice, ctx->stream));
        if (p->use_x0) EOFA_CUDA(cudaMemcpyAsync(dx, x, bytes, cudaMemcpyHostToDevice, ctx->stream));
        int rc = solve_dev_impl(ctx, p, db, dx, info, ctx->stream);
        if (rc == EOFA_OK || rc == EOFA_ENOTCONV) {
            EOFA_CUDA(cudaMemcpyAsync(x, dx, bytes, cudaMemcpyDeviceToHost, ctx->stream));
            EOFA_CUDA(cudaStreamSynchronize(ctx->stream));
        }
        return rc;
    } catch (const eofa_error& e) {
        if (info) info->status = e.code;
        return fail(ctx, e.code, e.msg);
    }
}

}  // extern "C"
