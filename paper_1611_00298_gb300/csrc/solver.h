// Solver state shared by single and batched solves (solver.cu, batch.cu).
#pragma once
#include "api_util.h"
#include "fused.h"

// One even-odd CG solve of (D_hop + G') psi = f (see solver.cu).  The
// iteration kernels read and write only this object's reduction scratch
// `red`, so several solves can run concurrently on one context.
struct Solve {
    eofa_ctx* ctx;
    eofa_solve_params P;
    int prec, precx;
    bool mixed;
    double delta_max;  // largest residual reduction between reliable updates
    bool two_level;    // FP16 inner storage: FP32 reliable updates between the FP64 ones
    double delta64, rmax64;       // two-level: reduction between FP64 updates, residual of the last one
    void *ra32, *rt32, *te32;     // two-level: FP32 anchor residual, FP32 residual, FP32 workspace
    double delta;      // the reduction of the current CG run (equal segments to the target)
    System5 S;
    Op5 Gi, GiT, G;
    double* red;       // reduction scratch / device scalars of this solve
    std::string tag;   // buffer-name suffix
    // FP64 half fields
    void *f_e, *f_o, *fh, *x_e, *x_o, *r64, *a_e, *a_o;
    // inner-precision fields
    void *p, *q, *r, *s, *te, *to, *x;
    double fnorm2, fhn, rmax, target_rel, target, true_rel;
    int it, ring, restarts;
    bool done, trivial;
    bool x_zero;       // x_o is known to be zero (no initial guess, CG not yet started)
    eofa_solve_info inf;

    // b_dev, x_dev: canonical 5D device fields (x_dev holds x0 when P.use_x0)
    void setup(eofa_ctx* c, const eofa_solve_params& p, const double* b_dev, const double* x_dev, const std::string& tg,
               double* red_scratch, int ring_len, cudaStream_t st);
    // start a CG run from the current FP64 iterate x_o; returns false if already converged
    bool start_cg(cudaStream_t st);
    // queue n CG iterations (no host synchronisation, except once per context and
    // precision when the iteration form is timed)
    void enqueue(int n, cudaStream_t st);
    // one CG iteration in form EOFA_CG_FORM_FIVE or EOFA_CG_FORM_SIX
    void iterate(int form, cudaStream_t st);
    // time both forms on real iterations of this solve; returns the iterations run
    int tune_form(int n, cudaStream_t st);
    // after a queued chunk: read |r|^2, do a reliable update if due; sets done when the inner target is met
    void check(int n, cudaStream_t st);
    // the same with |r|^2 already read back by the caller
    void check_value(double rr, cudaStream_t st);
    // device address of the |r|^2 written by the last queued iteration
    const double* last_rr() const { return red + SC_RRH + ((it + ring - 1) % ring); }
    // fold the inner solution into x_o, reconstruct, compute the true residual; true when finished
    bool finish(double* x_dev, cudaStream_t st);
};

int solve_dev_impl(eofa_ctx* ctx, const eofa_solve_params* p, const double* b_dev, double* x_dev,
                   eofa_solve_info* info, cudaStream_t st);
