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
#include "fused.h"

#include <algorithm>

#include <chrono>
#include <cmath>

namespace {

struct SchurOps {
    Op5 Gi, GiT;
};

// out = A in (odd -> odd) with the fused kernels; |out|^2 -> red[slot] if red
void apply_A(eofa_ctx* ctx, const SchurOps& o, int prec, const void* in, void* out, void* te, double* red, int slot,
             cudaStream_t st) {
    fused_dslash(ctx, prec, 0, 0, in, te, o.Gi, nullptr, 1.0, 0.0, nullptr, 0, st);
    fused_dslash(ctx, prec, 1, 0, te, out, o.Gi, in, -1.0, 1.0, red, slot, st);
}

// s = A^+ r' where r' = r - alpha q (when q; written back to r) and |r'|^2 -> red[rslot];
// |s|^2 -> red[gslot]
void apply_Adag_cg(eofa_ctx* ctx, const SchurOps& o, int prec, void* r, const void* q, int it, void* s, void* te,
                   void* to, int rslot, int gslot, cudaStream_t st) {
    fused_local5(ctx, prec, o.GiT, r, q, 0.0, ctx->red, it, q != nullptr, q != nullptr ? r : nullptr, to, 1.0,
                 ctx->red, rslot, st);
    fused_dslash(ctx, prec, 0, 1, to, te, o.GiT, nullptr, 1.0, 0.0, nullptr, 0, st);
    fused_dslash(ctx, prec, 1, 1, te, s, op_identity(), r, -1.0, 1.0, ctx->red, gslot, st);
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
    const size_t fbi = field_bytes(prec, ctx->Vh, ctx->Ls);
    std::string tag = "_" + std::to_string(prec);
    void* p = ctx_buffer(ctx, "sv_p" + tag, fbi);
    void* q = ctx_buffer(ctx, "sv_q" + tag, fbi);
    void* r = ctx_buffer(ctx, "sv_r" + tag, fbi);
    void* s = ctx_buffer(ctx, "sv_s" + tag, fbi);
    void* te = ctx_buffer(ctx, "sv_te" + tag, fbi);
    void* to = ctx_buffer(ctx, "sv_to" + tag, fbi);
    void* x = mixed ? ctx_buffer(ctx, "sv_x32", field_bytes(P32, ctx->Vh, ctx->Ls)) : x_o;
    double* red = ctx->red;

    double target_rel = 0.5 * P.tol;  // on |r| / |f^|, refined by the true-residual check
    int restarts = 0;
    double true_rel = 1.0;
    double hist[32];
    for (;;) {
        // r64 = f^ - A x_o  (FP64)
        apply_A(ctx, ops, P64, x_o, r64, a_e, nullptr, 0, st);
        blas_axpby(ctx, P64, 1.0, fh, -1.0, r64, st);
        double rr = norm2_now(ctx, P64, r64, st);
        if (!is_finite(rr)) throw eofa_error(EOFA_ENUMERIC, "NaN/Inf in the residual");
        const double target = target_rel * fhn;
        blas_copy(ctx, prec, r, P64, r64, st);
        if (mixed) blas_zero(ctx, precx, x, st);
        double rmax = std::sqrt(rr);
        int it = 0;  // iteration index within this CG run (parity of the gamma slots)
        if (std::sqrt(rr) > target) {
            // s = A^+ r, gamma -> slot of iteration 0, p = s
            apply_Adag_cg(ctx, ops, prec, r, nullptr, 0, s, te, to, SC_RRH, SC_GAMMA, st);
            blas_copy(ctx, prec, p, prec, s, st);
            int chunk = 4;
            double rr_prev = rr;
            bool done = false;
            while (!done && inf.iters < P.maxiter) {
                int n = chunk;
                if (n > P.maxiter - inf.iters) n = P.maxiter - inf.iters;
                for (int k = 0; k < n; k++, it++) {
                    apply_A(ctx, ops, prec, p, q, te, red, SC_DELTA, st);
                    apply_Adag_cg(ctx, ops, prec, r, q, it, s, te, to, SC_RRH + (it & 31),
                                  SC_GAMMA + ((it + 1) & 1), st);
                    fused_xp_update(ctx, prec, precx, red, it, x, p, s, st);
                }
                inf.iters += n;
                red_fetch_many(ctx, SC_RRH, 32, hist, st);
                rr = hist[(it - 1) & 31];
                if (!is_finite(rr)) throw eofa_error(EOFA_ENUMERIC, "NaN/Inf in CG");
                double rn = std::sqrt(rr);
                bool want_update = mixed && (rn < delta * rmax || rn < target || inf.iters >= P.maxiter);
                if (!mixed && rn < target) done = true;
                if (want_update) {
                    // reliable update: x64 += x, r64 = f^ - A x64 (FP64), r = r64, s = A^+ r
                    blas_copy(ctx, P64, a_o, precx, x, st);
                    blas_axpby(ctx, P64, 1.0, a_o, 1.0, x_o, st);
                    blas_zero(ctx, precx, x, st);
                    apply_A(ctx, ops, P64, x_o, r64, a_e, nullptr, 0, st);
                    blas_axpby(ctx, P64, 1.0, fh, -1.0, r64, st);
                    rr = norm2_now(ctx, P64, r64, st);
                    inf.reliable_updates++;
                    rn = std::sqrt(rr);
                    rmax = rn;
                    if (rn < target || inf.iters >= P.maxiter) {
                        done = true;
                    } else {
                        blas_copy(ctx, prec, r, P64, r64, st);
                        apply_Adag_cg(ctx, ops, prec, r, nullptr, it, s, te, to, SC_RRH + ((it - 1) & 31),
                                      SC_GAMMA + (it & 1), st);
                    }
                }
                // next chunk: iterations predicted to reach the next threshold
                double thr = mixed ? std::max(delta * rmax, target) : target;
                double rate = (rr_prev > 0 && rr < rr_prev && n > 0) ? std::pow(rr / rr_prev, 1.0 / n) : 0.0;
                rr_prev = rr;
                if (rate > 0 && rate < 1 && rr > thr * thr) {
                    double need = std::log(thr * thr / rr) / std::log(rate);
                    chunk = (int)std::ceil(need);
                } else {
                    chunk = 4;
                }
                if (chunk < 1) chunk = 1;
                if (chunk > 32) chunk = 32;
            }
            if (mixed) {
                blas_copy(ctx, P64, a_o, precx, x, st);
                blas_axpby(ctx, P64, 1.0, a_o, 1.0, x_o, st);
                blas_zero(ctx, precx, x, st);
            }
        }
        // reconstruct psi_e = G'^{-1} (f_e - D_eo psi_o)
        launch_hop(ctx, P64, 0, 0, x_o, a_e, st);
        blas_axpby(ctx, P64, 1.0, f_e, -1.0, a_e, st);
        launch_op5(ctx, P64, ops.Gi, a_e, nullptr, x_e, st);
        // true residual of the full system
        void* re = ctx_buffer(ctx, "sv_re", f64);
        void* ro = ctx_buffer(ctx, "sv_ro", f64);
        const void* out_e = x_e;
        const void* out_o = x_o;
        if (P.system == EOFA_SYS_DWF) {
            // psi = D-tilde^{-1} y, residual b - D_DWF psi
            Op5 Dti = op_plain(S.c, 1, 0, 0);
            void* pe = ctx_buffer(ctx, "sv_pe", f64);
            void* po = ctx_buffer(ctx, "sv_po", f64);
            launch_op5(ctx, P64, Dti, x_e, nullptr, pe, st);
            launch_op5(ctx, P64, Dti, x_o, nullptr, po, st);
            apply_dwf_fields(ctx, S.c, 0, pe, po, re, ro, st);
            out_e = pe;
            out_o = po;
        } else {
            apply_eofa_fields(ctx, G, x_e, x_o, re, ro, st);
        }
        blas_axpby(ctx, P64, 1.0, f_e, -1.0, re, st);
        blas_axpby(ctx, P64, 1.0, f_o, -1.0, ro, st);
        double res2 = norm2_now(ctx, P64, re, st) + norm2_now(ctx, P64, ro, st);
        true_rel = std::sqrt(res2 / fnorm2);
        if (true_rel <= P.tol || inf.iters >= P.maxiter || restarts >= 8 || !is_finite(true_rel)) {
            launch_unpack(ctx, P64, out_e, out_o, x_dev, st);
            break;
        }
        // not yet: tighten the inner target by the observed ratio and restart
        apply_A(ctx, ops, P64, x_o, r64, a_e, nullptr, 0, st);
        blas_axpby(ctx, P64, 1.0, fh, -1.0, r64, st);
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
