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
// CG on the normal equations A^+ A x = A^+ f^ (the least-squares form,
// tracking r = f^ - A x and the normal residual s = A^+ r) iterates in the
// inner precision in one of two forms of fused launches (iterate):
// five launches,
//   te = G'^-1 D_eo p;  q = p - G'^-1 D_oe te, |q|^2 = delta, to = G'^-T q;
//   te = G'^-T D^+_eo to, with x += alpha p and r <- r - alpha q, |r|^2
//   elementwise in the same launch;
//   s <- s - alpha (q - D^+_oe te) = s - alpha A^+ q, gamma' = |s|^2;
//   p = s + beta p,
// or six launches that move fewer bytes (s is formed from r, not updated),
//   te = G'^-1 D_eo p;  q = p - G'^-1 D_oe te, |q|^2 = delta;
//   r <- r - alpha q, |r|^2, to = G'^-T r;
//   te = G'^-T D^+_eo to, with x += alpha p in the same launch;
//   s = r - D^+_oe te = A^+ r, gamma' = |s|^2;
//   p = s + beta p.
// Which one runs is timed per context (Solve::enqueue).
// With mixed precision the residual is recomputed in FP64 whenever |r| has
// dropped by the factor delta since the last recomputation (reliable
// updates; they also reset s = A^+ r), and the solution accumulates in
// FP64; delta splits the way to the target into equal segments.  With FP16
// inner storage (delta ~ 0.1) most recomputations are FP32 ones relative to
// the last FP64 residual, and an FP64 one follows every reduction by ~1e-4.  The stopping test is the FP64 true residual of the full,
// unpreconditioned system.
#include "solver.h"
#include "reliable.h"

#include <algorithm>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>

namespace {

// out = A in (odd -> odd) with the fused kernels; |out|^2 -> red[slot] if red
void apply_A(eofa_ctx* ctx, const Op5& Gi, int prec, const void* in, void* out, void* te, double* red, int slot,
             cudaStream_t st) {
    fused_dslash(ctx, prec, 0, 0, in, te, Gi, nullptr, 1.0, 0.0, nullptr, 0, st);
    fused_dslash(ctx, prec, 1, 0, te, out, Gi, in, -1.0, 1.0, red, slot, st);
}

// s = A^+ r' where r' = r - alpha q (when q; written back to r) and |r'|^2 -> red[rslot];
// |s|^2 -> red[gslot]
void apply_Adag_cg(eofa_ctx* ctx, const Op5& GiT, int prec, void* r, const void* q, double* red, int it, void* s,
                   void* te, void* to, int rslot, int gslot, cudaStream_t st) {
    fused_local5(ctx, prec, GiT, r, q, 0.0, red, it, q != nullptr, q != nullptr ? r : nullptr, to, 1.0, red, rslot,
                 st);
    fused_dslash(ctx, prec, 0, 1, to, te, GiT, nullptr, 1.0, 0.0, nullptr, 0, st);
    fused_dslash(ctx, prec, 1, 1, te, s, op_identity(), r, -1.0, 1.0, red, gslot, st);
}

double norm2_now(eofa_ctx* ctx, int prec, const void* x, cudaStream_t st) {
    blas_norm2(ctx, prec, x, 0, st);
    return red_fetch(ctx, 0, st);
}

bool is_finite(double v) { return std::isfinite(v); }

double fetch_one(const eofa_ctx* ctx, const double* dev, cudaStream_t st) {
    EOFA_CUDA(cudaMemcpyAsync(ctx->red_host, dev, sizeof(double), cudaMemcpyDeviceToHost, st));
    EOFA_CUDA(cudaStreamSynchronize(st));
    return ctx->red_host[0];
}

}  // namespace

// FP16 inner storage: largest reduction between FP64 reliable updates; the
// FP32 recomputations in between are accurate to ~1e-7 of the last FP64
// residual, so 1e-4 leaves a margin of three orders (5e-6 measured 0.4%
// faster at 24^3x64x24 but took 2.5% more iterations)
static constexpr double DELTA64_TWO_LEVEL = 1e-4;

// ---------------------------------------------------------------- Solve

void Solve::setup(eofa_ctx* c, const eofa_solve_params& prm, const double* b_dev, const double* x_dev,
                  const std::string& tg, double* red_scratch, int ring_len, cudaStream_t st) {
    ctx = c;
    P = prm;
    tag = tg;
    red = red_scratch;
    ring = ring_len;
    inf.iters = 0;
    inf.reliable_updates = 0;
    inf.low_updates = 0;
    inf.true_resid = -1.0;
    inf.seconds = 0.0;
    inf.status = EOFA_OK;
    check_ls(ctx, P.Ls);
    require_gauge(ctx);
    if (!(P.tol > 0) || P.maxiter < 1 || P.precision < 0 || P.precision > 2 || P.system < 0 || P.system > 2)
        throw eofa_error(EOFA_EINVAL, "bad solve parameters");
    if (P.system != EOFA_SYS_DWF && !(P.m1 < P.m2)) throw eofa_error(EOFA_EINVAL, "EOFA systems need m1 < m2");
    mixed = P.precision != EOFA_PREC_F64;
    prec = P.precision == EOFA_PREC_F64 ? P64 : (P.precision == EOFA_PREC_MIXED_F32 ? P32 : P16);
    precx = mixed ? P32 : P64;
    // largest residual reduction between reliable updates: P.delta <= 0 picks
    // the default of the inner precision.  An FP32 recursion follows the
    // residual down by 5e-6 without costing iterations (1e-6 cost a fifth
    // more at 24^3x64, Ls = 24); FP16 storage not much beyond ~1e-2.
    const double auto_delta = prec == P16 ? 0.1 : 5e-6;
    delta_max = (P.delta > 0 && P.delta < 1) ? P.delta : auto_delta;
    if (prec == P16 && delta_max < 0.05) delta_max = 0.05;
    delta = delta_max;
    S = P.system == EOFA_SYS_DWF ? system_dwf(P.alpha, P.M5, P.mf)
                                 : system_eofa(P.Ls, P.alpha, P.M5, P.m1, P.m2, P.system, P.shift);
    // per-solve coefficient slots so that concurrent solves on one context do not clash
    int base = 0;
    if (!tag.empty()) {
        double* coef = (double*)ctx_buffer(ctx, "coef" + tag, 16 * EOFA_MAX_LS * sizeof(double));
        double* saved = ctx->coef;
        ctx->coef = coef;
        Gi = op_Ginv(ctx, S, 0, st);
        GiT = op_GinvT(ctx, S, 2, st);
        G = op_G(ctx, S, 4, st);
        ctx->coef = saved;
    } else {
        Gi = op_Ginv(ctx, S, base, st);
        GiT = op_GinvT(ctx, S, base + 2, st);
        G = op_G(ctx, S, base + 4, st);
    }

    const size_t f64 = field_bytes(P64, ctx->Vh, ctx->Ls);
    const long long n5full = (long long)ctx->V * ctx->Ls * 12;
    f_e = ctx_buffer(ctx, "sv_fe" + tag, f64);
    f_o = ctx_buffer(ctx, "sv_fo" + tag, f64);
    fh = ctx_buffer(ctx, "sv_fh" + tag, f64);
    x_e = ctx_buffer(ctx, "sv_xe" + tag, f64);
    x_o = ctx_buffer(ctx, "sv_xo" + tag, f64);
    r64 = ctx_buffer(ctx, "sv_r64" + tag, f64);
    a_e = ctx_buffer(ctx, "sv_ae" + tag, f64);
    a_o = ctx_buffer(ctx, "sv_ao" + tag, f64);
    const double* fsrc = b_dev;
    if (P.system != EOFA_SYS_DWF) {
        double* canon = (double*)ctx_buffer(ctx, "sv_canon", (size_t)n5full * 16);
        launch_rs5(ctx, b_dev, canon, st);  // f = R5 gamma5 b
        fsrc = canon;
    }
    launch_pack(ctx, P64, fsrc, f_e, f_o, st);
    fnorm2 = norm2_now(ctx, P64, f_e, st) + norm2_now(ctx, P64, f_o, st);
    if (!is_finite(fnorm2)) throw eofa_error(EOFA_ENUMERIC, "right-hand side has NaN/Inf");
    trivial = fnorm2 == 0.0;
    done = trivial;
    x_zero = false;
    if (trivial) return;
    if (P.use_x0) {
        launch_pack(ctx, P64, x_dev, x_e, x_o, st);
        if (P.system == EOFA_SYS_DWF) {  // iterate on y = D-tilde psi
            Op5 Dt = op_plain(S.c, 0, 1, 0);
            launch_op5(ctx, P64, Dt, x_o, nullptr, x_o, st);
        }
    } else {
        blas_zero(ctx, P64, x_o, st);
    }
    x_zero = !P.use_x0;
    // f^_o = G'^{-1} (f_o - D_oe G'^{-1} f_e)
    launch_op5(ctx, P64, Gi, f_e, nullptr, a_e, st);
    launch_hop(ctx, P64, 1, 0, a_e, a_o, st);
    blas_axpby(ctx, P64, 1.0, f_o, -1.0, a_o, st);
    launch_op5(ctx, P64, Gi, a_o, nullptr, fh, st);
    fhn = std::sqrt(norm2_now(ctx, P64, fh, st));

    const size_t fbi = field_bytes(prec, ctx->Vh, ctx->Ls);
    std::string t = "_" + std::to_string(prec) + tag;
    p = ctx_buffer(ctx, "sv_p" + t, fbi);
    q = ctx_buffer(ctx, "sv_q" + t, fbi);
    r = ctx_buffer(ctx, "sv_r" + t, fbi);
    s = ctx_buffer(ctx, "sv_s" + t, fbi);
    te = ctx_buffer(ctx, "sv_te" + t, fbi);
    to = ctx_buffer(ctx, "sv_to" + t, fbi);
    x = mixed ? ctx_buffer(ctx, "sv_x32" + tag, field_bytes(P32, ctx->Vh, ctx->Ls)) : x_o;
    two_level = prec == P16;
    if (two_level) {
        const size_t f32 = field_bytes(P32, ctx->Vh, ctx->Ls);
        ra32 = ctx_buffer(ctx, "sv_ra32" + tag, f32);
        rt32 = ctx_buffer(ctx, "sv_rt32" + tag, f32);
        te32 = ctx_buffer(ctx, "sv_te32" + tag, f32);
    }
    target_rel = 0.5 * P.tol;  // on |r| / |f^|, refined by the true-residual check
    restarts = 0;
    true_rel = 1.0;
}

bool Solve::start_cg(cudaStream_t st) {
    // r64 = f^ - A x_o (FP64); with x_o = 0 it is f^ itself (two FP64 hops saved)
    if (x_zero) {
        blas_copy(ctx, P64, r64, P64, fh, st);
    } else {
        apply_A(ctx, Gi, P64, x_o, r64, a_e, nullptr, 0, st);
        blas_axpby(ctx, P64, 1.0, fh, -1.0, r64, st);
    }
    x_zero = false;
    double rr = norm2_now(ctx, P64, r64, st);
    if (!is_finite(rr)) throw eofa_error(EOFA_ENUMERIC, "NaN/Inf in the residual");
    target = target_rel * fhn;
    // split the reduction from |r| to the target into the fewest equal
    // segments of at most delta_max: a reliable update ends each segment but
    // the last, which ends at convergence (no update there, see check_value)
    auto segment = [&](double dmax) { return mixed ? equal_segment_reduction(std::sqrt(rr), target, dmax) : dmax; };
    delta = segment(delta_max);
    if (two_level) {
        // FP16 inner storage: FP32 recomputations every delta, FP64 ones every
        // delta64; the FP32 anchor is the FP64 residual of this start
        delta64 = segment(DELTA64_TWO_LEVEL);
        rmax64 = std::sqrt(rr);
        blas_copy(ctx, P32, ra32, P64, r64, st);
    }
    blas_copy(ctx, prec, r, P64, r64, st);
    if (mixed) blas_zero(ctx, precx, x, st);
    rmax = std::sqrt(rr);
    it = 0;
    if (std::sqrt(rr) <= target) {
        done = true;
        return false;
    }
    // s = A^+ r, gamma -> slot of iteration 0, p = s
    apply_Adag_cg(ctx, GiT, prec, r, nullptr, red, 0, s, te, to, SC_RRH, SC_GAMMA, st);
    blas_copy(ctx, prec, p, prec, s, st);
    done = false;
    return true;
}

static bool solve_log() {
    static const int v = getenv("EOFA_SOLVE_LOG") ? 1 : 0;
    return v != 0;
}

// One CG iteration in the given form.  Both forms leave the same state at
// the iteration boundary (x, r, p, s = A^+ r, |r|^2 in the ring slot of the
// iteration, gamma in the slot of the next parity), so a solve may switch
// between them at any iteration.
void Solve::iterate(int form, cudaStream_t st) {
    if (form == EOFA_CG_FORM_SIX) {
        // q = A p, |q|^2 -> delta
        apply_A(ctx, Gi, prec, p, q, te, red, SC_DELTA, st);
        // r -= alpha q, |r|^2 -> ring, to = G'^-T r
        fused_local5(ctx, prec, GiT, r, q, 0.0, red, it, 1, r, to, 1.0, red, SC_RRH + (it % ring), st);
        // te = G'^-T D^+_eo to, with x += alpha p riding along
        fused_dslash_x(ctx, prec, 0, 1, to, te, GiT, red, it, x, p, nullptr, nullptr, 0, st);
        // s = r - D^+_oe te = A^+ r, |s|^2 -> gamma (next parity)
        fused_dslash(ctx, prec, 1, 1, te, s, op_identity(), r, -1.0, 1.0, red, SC_GAMMA + ((it + 1) & 1), st);
    } else {
        // q = A p, |q|^2 -> delta, to = G'^-T q
        fused_dslash(ctx, prec, 0, 0, p, te, Gi, nullptr, 1.0, 0.0, nullptr, 0, st);
        fused_dslash_to(ctx, prec, 1, 0, te, q, Gi, p, -1.0, 1.0, red, SC_DELTA, GiT, to, st);
        // te = G'^-T D^+_eo to, with x += alpha p and r -= alpha q, |r|^2 -> ring riding along
        // (alpha is known once delta is)
        fused_dslash_x(ctx, prec, 0, 1, to, te, GiT, red, it, x, p, r, q, SC_RRH + (it % ring), st);
        // s -= alpha A^+ q, |s|^2 -> gamma (next parity)
        fused_dslash_z(ctx, prec, 1, 1, te, s, op_identity(), q, -1.0, 1.0, red, SC_GAMMA + ((it + 1) & 1), it,
                       nullptr, 0, st);
    }
    // p = s + beta p
    fused_xp_update(ctx, prec, precx, red, it, nullptr, p, s, st);
    it++;
}

// The iteration form of a context and inner precision: set by
// eofa_set_cg_form, else timed on the first chunk of at least
// FORM_TUNE_MIN iterations that runs outside stream capture.  The timing
// runs real CG iterations: one warm-up iteration per form (it lets the
// kernel autotuner settle), then blocks of m iterations in the order
// five, six, six, five with CUDA events on the solve's stream; the form
// with the smaller total wins.  Until then (short chunks, capture), the
// five-launch form runs below FORM_SIX_SITES sites per checkerboard and
// the six-launch form above, where bytes rather than launches set the
// iteration time.
static constexpr int FORM_TUNE_MIN = 6;
static constexpr long long FORM_SIX_SITES = 1LL << 22;

static long long form_key(int prec) { return -1 - (long long)prec; }

int Solve::tune_form(int n, cudaStream_t st) {
    iterate(EOFA_CG_FORM_FIVE, st);
    iterate(EOFA_CG_FORM_SIX, st);
    const int m = (n - 2) / 4;
    const int order[4] = {EOFA_CG_FORM_FIVE, EOFA_CG_FORM_SIX, EOFA_CG_FORM_SIX, EOFA_CG_FORM_FIVE};
    cudaEvent_t ev[5];
    for (auto& e : ev) EOFA_CUDA(cudaEventCreate(&e));
    EOFA_CUDA(cudaEventRecord(ev[0], st));
    for (int b = 0; b < 4; b++) {
        for (int k = 0; k < m; k++) iterate(order[b], st);
        EOFA_CUDA(cudaEventRecord(ev[b + 1], st));
    }
    EOFA_CUDA(cudaEventSynchronize(ev[4]));
    float ms[4];
    for (int b = 0; b < 4; b++) EOFA_CUDA(cudaEventElapsedTime(&ms[b], ev[b], ev[b + 1]));
    for (auto& e : ev) EOFA_CUDA(cudaEventDestroy(e));
    const int form = ms[0] + ms[3] <= ms[1] + ms[2] ? EOFA_CG_FORM_FIVE : EOFA_CG_FORM_SIX;
    (*ctx->tuned)[form_key(prec)] = form;
    if (getenv("EOFA_TUNE_LOG"))
        fprintf(stderr, "cg form (precision %d, %d iterations each): five %.4f ms, six %.4f ms per iteration -> %s\n",
                prec, 2 * m, (ms[0] + ms[3]) / (2 * m), (ms[1] + ms[2]) / (2 * m),
                form == EOFA_CG_FORM_FIVE ? "five" : "six");
    return 2 + 4 * m;
}

void Solve::enqueue(int n, cudaStream_t st) {
    int done_here = 0;
    int form;
    auto f = ctx->tuned->find(form_key(prec));
    if (f != ctx->tuned->end()) {
        form = f->second;
    } else {
        cudaStreamCaptureStatus cs;
        EOFA_CUDA(cudaStreamIsCapturing(st, &cs));
        if (cs == cudaStreamCaptureStatusNone && n >= FORM_TUNE_MIN) {
            done_here = tune_form(n, st);
            form = ctx->tuned->at(form_key(prec));
        } else {
            form = (long long)ctx->Vh * ctx->Ls >= FORM_SIX_SITES ? EOFA_CG_FORM_SIX : EOFA_CG_FORM_FIVE;
        }
    }
    for (int k = done_here; k < n; k++) iterate(form, st);
    inf.iters += n;
}

void Solve::check(int n, cudaStream_t st) { check_value(fetch_one(ctx, last_rr(), st), st); }

void Solve::check_value(double rr, cudaStream_t st) {
    if (!is_finite(rr)) throw eofa_error(EOFA_ENUMERIC, "NaN/Inf in CG");
    double rn = std::sqrt(rr);
    if (!mixed) {
        if (rn < target || inf.iters >= P.maxiter) done = true;
        return;
    }
    // a residual above the last recomputed one means the low-precision recursion
    // has lost track: recompute in FP64 and restart the search direction
    const bool diverging = rn > rmax;
    if (rn < target && !diverging) {
        // converged by the recursive residual, whose drift since the last
        // reliable update is far below the target: finish() folds x into x_o
        // and judges by the FP64 true residual of the full system (a CG
        // restart follows if that is not met), so the FP64 recomputation of
        // r here would be redundant
        done = true;
        return;
    }
    const bool due = rn < delta * rmax || rn < target || inf.iters >= P.maxiter || diverging;
    if (due && two_level && !diverging && rn >= target && inf.iters < P.maxiter && rn >= delta64 * rmax64) {
        // FP32 reliable update (FP16 inner storage): r = ra - A x in FP32, with
        // ra the residual of the last FP64 update and x the inner solution
        // accumulated since then; |r| stays above delta64 |ra|, far above the
        // FP32 rounding of ra - A x
        apply_A(ctx, Gi, P32, x, rt32, te32, nullptr, 0, st);
        blas_axpby(ctx, P32, 1.0, ra32, -1.0, rt32, st);
        rr = norm2_now(ctx, P32, rt32, st);
        if (!is_finite(rr)) throw eofa_error(EOFA_ENUMERIC, "NaN/Inf in the FP32 residual");
        inf.low_updates++;
        if (solve_log())
            fprintf(stderr, "FP32 update %d: iters %d, inner |r| %.3e, FP32 |r| %.3e, last %.3e\n", inf.low_updates,
                    inf.iters, rn, std::sqrt(rr), rmax);
        rmax = std::sqrt(rr);
        blas_copy(ctx, prec, r, P32, rt32, st);
        apply_Adag_cg(ctx, GiT, prec, r, nullptr, red, it, s, te, to, SC_RRH + ((it + ring - 1) % ring),
                      SC_GAMMA + (it & 1), st);
        return;
    }
    if (due) {
        // reliable update: x64 += x, r64 = f^ - A x64 (FP64), r = r64, s = A^+ r
        blas_copy(ctx, P64, a_o, precx, x, st);
        blas_axpby(ctx, P64, 1.0, a_o, 1.0, x_o, st);
        blas_zero(ctx, precx, x, st);
        apply_A(ctx, Gi, P64, x_o, r64, a_e, nullptr, 0, st);
        blas_axpby(ctx, P64, 1.0, fh, -1.0, r64, st);
        rr = norm2_now(ctx, P64, r64, st);
        inf.reliable_updates++;
        if (solve_log())
            fprintf(stderr, "reliable update %d: iters %d, inner |r| %.3e, true |r| %.3e, last true %.3e, target %.3e\n",
                    inf.reliable_updates, inf.iters, rn, std::sqrt(rr), rmax, target);
        rn = std::sqrt(rr);
        rmax = rn;
        if (two_level) {
            rmax64 = rn;
            blas_copy(ctx, P32, ra32, P64, r64, st);
        }
        if (rn < target || inf.iters >= P.maxiter) {
            done = true;
        } else {
            blas_copy(ctx, prec, r, P64, r64, st);
            apply_Adag_cg(ctx, GiT, prec, r, nullptr, red, it, s, te, to, SC_RRH + ((it + ring - 1) % ring),
                          SC_GAMMA + (it & 1), st);
            if (diverging) blas_copy(ctx, prec, p, prec, s, st);
        }
    }
}

bool Solve::finish(double* x_dev, cudaStream_t st) {
    check_device_error(ctx, st);
    if (trivial) {
        EOFA_CUDA(cudaMemsetAsync(x_dev, 0, (size_t)ctx->V * ctx->Ls * 12 * 16, st));
        true_rel = 0.0;
        return true;
    }
    if (mixed) {
        blas_copy(ctx, P64, a_o, precx, x, st);
        blas_axpby(ctx, P64, 1.0, a_o, 1.0, x_o, st);
        blas_zero(ctx, precx, x, st);
    }
    const size_t f64 = field_bytes(P64, ctx->Vh, ctx->Ls);
    // reconstruct psi_e = G'^{-1} (f_e - D_eo psi_o)
    launch_hop(ctx, P64, 0, 0, x_o, a_e, st);
    blas_axpby(ctx, P64, 1.0, f_e, -1.0, a_e, st);
    launch_op5(ctx, P64, Gi, a_e, nullptr, x_e, st);
    void* re = ctx_buffer(ctx, "sv_re" + tag, f64);
    void* ro = ctx_buffer(ctx, "sv_ro" + tag, f64);
    const void* out_e = x_e;
    const void* out_o = x_o;
    if (P.system == EOFA_SYS_DWF) {
        // psi = D-tilde^{-1} y, residual b - D_DWF psi
        Op5 Dti = op_plain(S.c, 1, 0, 0);
        void* pe = ctx_buffer(ctx, "sv_pe" + tag, f64);
        void* po = ctx_buffer(ctx, "sv_po" + tag, f64);
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
        return true;
    }
    // not yet: tighten the inner target by the observed ratio; the caller restarts the CG
    apply_A(ctx, Gi, P64, x_o, r64, a_e, nullptr, 0, st);
    blas_axpby(ctx, P64, 1.0, fh, -1.0, r64, st);
    double rr_now = norm2_now(ctx, P64, r64, st);
    double ratio = std::sqrt(rr_now) / fhn / (true_rel > 0 ? true_rel : 1e-300);
    double nt = 0.5 * P.tol * ratio;
    target_rel = nt < 0.5 * target_rel ? nt : 0.5 * target_rel;
    restarts++;
    return false;
}

int solve_dev_impl(eofa_ctx* ctx, const eofa_solve_params* prm, const double* b_dev, double* x_dev,
                   eofa_solve_info* info, cudaStream_t st) {
    auto t0 = std::chrono::steady_clock::now();
    Solve sv;
    sv.setup(ctx, *prm, b_dev, x_dev, "", ctx->red, 32, st);
    if (!sv.trivial) {
        for (;;) {
            if (sv.start_cg(st)) {
                int chunk = 4;
                double rr_prev = -1;
                while (!sv.done && sv.inf.iters < sv.P.maxiter) {
                    int n = std::min(chunk, sv.P.maxiter - sv.inf.iters);
                    sv.enqueue(n, st);
                    sv.check(n, st);
                    // next chunk: iterations predicted to reach the next threshold
                    double rr = fetch_one(ctx, sv.red + SC_RRH + ((sv.it - 1) % sv.ring), st);
                    double thr = sv.mixed ? std::max(sv.delta * sv.rmax, sv.target) : sv.target;
                    double rate = (rr_prev > 0 && rr < rr_prev && n > 0) ? std::pow(rr / rr_prev, 1.0 / n) : 0.0;
                    rr_prev = rr;
                    if (rate > 0 && rate < 1 && rr > thr * thr)
                        chunk = (int)std::ceil(std::log(thr * thr / rr) / std::log(rate));
                    else
                        chunk = 4;
                    chunk = std::max(1, std::min(chunk, 32));
                }
            }
            if (sv.finish(x_dev, st)) break;
        }
    } else {
        sv.finish(x_dev, st);
    }
    EOFA_CUDA(cudaStreamSynchronize(st));
    eofa_solve_info inf = sv.inf;
    inf.true_resid = sv.true_rel;
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (!is_finite(sv.true_rel)) inf.status = EOFA_ENUMERIC;
    else if (sv.true_rel > sv.P.tol) inf.status = EOFA_ENOTCONV;
    if (info) *info = inf;
    if (inf.status != EOFA_OK) {
        ctx->err = inf.status == EOFA_ENOTCONV
                       ? "solver did not reach tol (true residual " + std::to_string(sv.true_rel) + ")"
                       : "NaN/Inf in the solution";
    }
    return inf.status;
}

extern "C" {

int eofa_set_cg_form(eofa_ctx* ctx, int precision, int form) {
    if (!ctx) return EOFA_EINVAL;
    if (precision < EOFA_PREC_F64 || precision > EOFA_PREC_MIXED_F16)
        return fail(ctx, EOFA_EINVAL, "precision must be an EOFA_PREC_* value");
    if (form == EOFA_CG_FORM_AUTO) ctx->tuned->erase(form_key(precision));
    else if (form == EOFA_CG_FORM_FIVE || form == EOFA_CG_FORM_SIX) (*ctx->tuned)[form_key(precision)] = form;
    else return fail(ctx, EOFA_EINVAL, "form must be EOFA_CG_FORM_AUTO, _FIVE or _SIX");
    return EOFA_OK;
}

int eofa_get_cg_form(const eofa_ctx* ctx, int precision, int* form) {
    if (!ctx || !form || precision < EOFA_PREC_F64 || precision > EOFA_PREC_MIXED_F16) return EOFA_EINVAL;
    auto f = ctx->tuned->find(form_key(precision));
    *form = f != ctx->tuned->end() ? f->second : EOFA_CG_FORM_AUTO;
    return EOFA_OK;
}

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
