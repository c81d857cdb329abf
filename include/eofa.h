/*
 * eofa.h -- C ABI of the GB300 library for the exact one-flavor algorithm
 * (EOFA) with Shamir / Moebius domain-wall fermions.
 *
 * Paper: D. Murphy, "Domain Wall Fermion Simulations with the Exact
 * One-Flavor Algorithm", Lattice 2016.  Equation numbers below are the
 * paper's: Eq. (3) D_DWF = D_EOFA * D-tilde, Eq. (5) the EOFA action,
 * Eq. (6) the heatbath, Eq. (7) the pseudofermion force, Eq. (8) the EOFA
 * linear systems; Sec. 5 the HMC trajectory (gauge action, force-gradient
 * integrators).
 *
 * Conventions shared by every call
 * --------------------------------
 * Lattice dims[4] = {X, Y, Z, T}, every extent even (even-odd
 * decomposition, Sec. 5.1).  Site index i = x + X (y + Y (z + Z t)).
 * Complex numbers are interleaved (re, im) FP64.  Host canonical layouts:
 *   gauge U   [i][mu][a][b]            mu = x, y, z, t -> 0..3     (4 V 9 cplx)
 *   5D field  [s][i][spin][colour]     s = 0..Ls-1                  (12 V Ls cplx)
 *   4D field  [i][spin][colour]                                     (12 V cplx)
 *   force F   [i][mu][a][b]            traceless Hermitian           (4 V 9 cplx)
 * Gamma matrices: Euclidean chiral basis, gamma_5 = diag(1, 1, -1, -1),
 * so P_+ keeps spins 0, 1 and P_- keeps spins 2, 3.
 * D_w = (4 - M5) - 1/2 sum_mu [(1 - g_mu) U_mu(x) psi(x+mu)
 *                              + (1 + g_mu) U_mu(x-mu)^+ psi(x-mu)],
 * periodic in x, y, z; the t-links from T-1 to 0 carry bc_t (+1 or -1).
 * L = P_+ L_+ + P_- L_-, (L_+)_{s,s-1} = 1, (L_+)_{0,Ls-1} = -m_f, L_- = L_+^T.
 * Moebius weights c = alpha/2, d = 1/2 (Shamir: alpha = 1).
 *
 * Ownership and errors
 * --------------------
 * Host pointers are caller-owned and only read or written during the call.
 * "_dev" calls take device pointers (caller-owned, same canonical layout)
 * and a cudaStream_t passed as void*; they are stream-ordered and return once
 * the work is queued unless they must read a scalar back (solves, action).
 * Every call returns EOFA_OK (0) or a negative status and never throws;
 * eofa_last_error() gives a message for the last failure on the context.
 */
#ifndef EOFA_H
#define EOFA_H

#ifdef __cplusplus
extern "C" {
#endif

#define EOFA_OK 0
#define EOFA_EINVAL (-1)    /* bad argument: dims, Ls, masses, pointers, non-unitary U */
#define EOFA_ENOMEM (-2)    /* device allocation failed */
#define EOFA_ENOTCONV (-3)  /* solver hit maxiter; info still filled */
#define EOFA_ENUMERIC (-4)  /* NaN or Inf met */
#define EOFA_ETIMEOUT (-5)  /* a bounded device wait ran out (see eofa_check_device) */
#define EOFA_EDEVICE (-6)   /* CUDA error; message has the CUDA string */

/* storage / arithmetic of the solver's inner iteration */
#define EOFA_PREC_F64 0         /* FP64 storage, FP64 arithmetic */
#define EOFA_PREC_MIXED_F32 1   /* inner FP32 storage + arithmetic, FP64 reliable updates */
#define EOFA_PREC_MIXED_F16 2   /* inner FP16 storage (per-site FP32 scale), FP32 arithmetic */

/* which linear system eofa_solve inverts */
#define EOFA_SYS_DWF 0     /* D_DWF(m_f) x = b                        (Eq. (3)) */
#define EOFA_SYS_EOFA_L 1  /* (H(m1) + shift Delta_- P_-) x = b       (Eq. (8)) */
#define EOFA_SYS_EOFA_R 2  /* (H(m2) + shift Delta_+ P_+) x = b       (Eq. (8)) */

typedef struct eofa_ctx eofa_ctx;

typedef struct {
    int Ls;           /* fifth-dimension extent; must equal the context's */
    double alpha;     /* Moebius scale (c = alpha/2, d = 1/2) */
    double M5;        /* domain-wall height */
    int system;       /* EOFA_SYS_* */
    double mf;        /* mass of EOFA_SYS_DWF */
    double m1, m2;    /* EOFA mass pair (m1 < m2) for EOFA_SYS_EOFA_L/R */
    double shift;     /* a in (H + a Delta P); the action's chi_R uses -1 */
    int precision;    /* EOFA_PREC_* */
    double tol;       /* target true relative residual |b - A x| / |b| */
    int maxiter;      /* cap on inner iterations (all restarts) */
    double delta;     /* mixed precision: largest reduction of |r| between FP64
                         reliable updates; the solver splits the way from the
                         starting residual to the target into the fewest equal
                         reductions no smaller than delta.  <= 0: default (5e-6 for
                         FP32 inner storage, 0.1 for FP16, which is never below
                         0.05) */
    int use_x0;       /* 1: x holds the initial guess on entry */
} eofa_solve_params;

typedef struct {
    int iters;             /* inner CG iterations */
    int reliable_updates;  /* FP64 residual recomputations */
    double true_resid;     /* FP64 |b - A x| / |b| of the full (unpreconditioned) system */
    double seconds;        /* wall time of the solve */
    int status;            /* EOFA_OK or the failure */
    int low_updates;       /* FP32 residual recomputations between the FP64 ones
                              (EOFA_PREC_MIXED_F16 only) */
} eofa_solve_info;

/* Create a context for one lattice.  dims: {X, Y, Z, T}, all even and >= 2;
 * Ls in [1, 64]; bc_t = +1 or -1; flags must be 0.  Picks the current CUDA
 * device.  (Sec. 2 notation: V = X Y Z T, Ls.) */
int eofa_create(eofa_ctx** ctx, const int dims[4], int Ls, int bc_t, int flags);
int eofa_destroy(eofa_ctx* ctx);
const char* eofa_last_error(const eofa_ctx* ctx);

/* Load the gauge field (Sec. 2: U_mu(x) inside D_w).  U: host canonical,
 * copied.  Checks |U^+ U - 1| < 1e-10 on every link (else EOFA_EINVAL). */
int eofa_gauge_load(eofa_ctx* ctx, const double* U);
int eofa_gauge_load_dev(eofa_ctx* ctx, const double* U_dev, void* stream);

/* out = D_DWF in (dagger = 0) or D_DWF^+ in (dagger = 1), full 5D lattice,
 * Eq. (3) first line.  in, out: 5D canonical, 12 V Ls complex each. */
int eofa_dwf_apply(eofa_ctx* ctx, int Ls, double alpha, double M5, double mf, int dagger,
                   const double* in, double* out);
int eofa_dwf_apply_dev(eofa_ctx* ctx, int Ls, double alpha, double M5, double mf, int dagger,
                       const double* in_dev, double* out_dev, void* stream);

/* out = D_EOFA in, Eq. (3) middle line: D_w + (1 - L) D-tilde^{-1} (the
 * 5D-local inverse is applied in O(Ls), never as a dense matrix). */
int eofa_eofa_apply(eofa_ctx* ctx, int Ls, double alpha, double M5, double mf,
                    const double* in, double* out);
int eofa_eofa_apply_dev(eofa_ctx* ctx, int Ls, double alpha, double M5, double mf,
                        const double* in_dev, double* out_dev, void* stream);

/* Even-odd hop on every s-slice, the hopping part of D_w (Sec. 2):
 * out(x, s) = -1/2 sum_mu [...] restricted to output sites of parity
 * out_parity, for a 5D field stored in the library's device layout of the
 * given storage precision (EOFA_PREC_F64 / MIXED_F32 / MIXED_F16 selects
 * FP64 / FP32 / FP16+scale).  For benchmarking and kernel tests: in_dev and
 * out_dev are device buffers of eofa_field_bytes(ctx, precision) bytes. */
long long eofa_field_bytes(const eofa_ctx* ctx, int precision);
int eofa_hop_dev(eofa_ctx* ctx, int precision, int out_parity, int dagger,
                 const void* in_dev, void* out_dev, void* stream);
/* One half of the even-odd preconditioned operator of Eq. (3) in a single
 * fused kernel: out = G^{-1} D_hop in (dagger = 0) or G^{-T} D_hop^+ in
 * (dagger = 1), with D_hop the hop above and G = M D-tilde^{-1} the 5D-local
 * block of D_EOFA = D_hop + G at mass mf (M = (4 - M5) D-tilde + 1 - L).
 * Same buffers and layouts as eofa_hop_dev. */
int eofa_schur_hop_dev(eofa_ctx* ctx, int precision, int out_parity, int dagger, int Ls, double alpha,
                       double M5, double mf, const void* in_dev, void* out_dev, void* stream);
/* Device status of the context: waits for the stream, then returns
 * EOFA_ETIMEOUT (and clears the flag) if a bounded wait inside a staged
 * (bulk-copy) dslash launch on this context ran out since the last check,
 * else EOFA_OK.  Such a launch leaves its output undefined but the context
 * usable.  Solves check this flag themselves when they finish; callers of the
 * asynchronous *_dev kernels above can check it here. */
int eofa_check_device(eofa_ctx* ctx, void* stream);
/* Pack a canonical FP64 5D field (device) into the two half-checkerboard
 * device-layout fields of the given precision, and back. */
int eofa_pack_dev(eofa_ctx* ctx, int precision, const double* canon_dev, void* even_dev,
                  void* odd_dev, void* stream);
int eofa_unpack_dev(eofa_ctx* ctx, int precision, const void* even_dev, const void* odd_dev,
                    double* canon_dev, void* stream);

/* Solve one linear system (Sec. 5.1): even-odd Schur complement, 5D-local
 * inverse through the Cayley factorisation of Eq. (3), CG on the normal
 * equations, optional mixed precision with FP64 reliable updates.
 * b, x: 5D canonical (x is the initial guess when p->use_x0).  Returns
 * EOFA_ENOTCONV with info filled when tol is not reached in maxiter. */
int eofa_solve(eofa_ctx* ctx, const eofa_solve_params* p, const double* b, double* x,
               eofa_solve_info* info);
int eofa_solve_dev(eofa_ctx* ctx, const eofa_solve_params* p, const double* b_dev, double* x_dev,
                   eofa_solve_info* info, void* stream);

/* EOFA action S_f = phi^+ M_EOFA phi, Eq. (5), for a 4D pseudofermion phi.
 * Needs m1 < m2.  Runs the two solves chi_L, chi_R (info[0], info[1]) with
 * the given precision and tol; S is accumulated in FP64. */
int eofa_action(eofa_ctx* ctx, int Ls, double alpha, double M5, double m1, double m2,
                int precision, double tol, const double* phi, double* S, eofa_solve_info info[2]);
int eofa_action_dev(eofa_ctx* ctx, int Ls, double alpha, double M5, double m1, double m2,
                    int precision, double tol, const double* phi_dev, double* S,
                    eofa_solve_info info[2], void* stream);

/* EOFA pseudofermion force, Eq. (7): F_mu(x) = sum_a F^a T^a with
 * F^a = dS_f / dw for U_mu(x) -> exp(i w T^a) U_mu(x), T^a = lambda^a / 2.
 * F: 4 V 3x3 traceless Hermitian, canonical.  S (may be NULL) gets the
 * action from the same solves. */
int eofa_force(eofa_ctx* ctx, int Ls, double alpha, double M5, double m1, double m2,
               int precision, double tol, const double* phi, double* F, double* S,
               eofa_solve_info info[2]);
int eofa_force_dev(eofa_ctx* ctx, int Ls, double alpha, double M5, double m1, double m2,
                   int precision, double tol, const double* phi_dev, double* F_dev, double* S,
                   eofa_solve_info info[2], void* stream);

/* Force from given solutions (Eq. (7) with chi_L, chi_R supplied):
 * F = k T[chi_L] - k T[chi_R], chi: 5D canonical device fields. */
int eofa_force_from_chi_dev(eofa_ctx* ctx, double k, const double* chiL_dev,
                            const double* chiR_dev, double* F_dev, void* stream);

/* The two terms of Eq. (7) separately (asymmetric integration of the L and
 * R parts, Sec. 3.3): FL_dev gets the force of S_L = phi_-^+ M_L phi_- (one
 * solve for chi_L), FR_dev that of S_R = phi_+^+ M_R phi_+ (one solve for
 * chi_R); either may be NULL (its solve is skipped).  Same layout and
 * convention as eofa_force_dev; FL + FR = F.  info[0] / info[1]: the solves
 * (zeroed when skipped). */
int eofa_force_parts_dev(eofa_ctx* ctx, int Ls, double alpha, double M5, double m1, double m2, int precision,
                         double tol, const double* phi_dev, double* FL_dev, double* FR_dev, eofa_solve_info info[2],
                         void* stream);

/* Gradient of S with respect to the real and imaginary parts of every link
 * entry (for automatic differentiation): G has the gauge layout and holds
 * dS/dRe U + i dS/dIm U.  Uses the same chi_L, chi_R as the force. */
int eofa_grad_from_chi_dev(eofa_ctx* ctx, double k, const double* chiL_dev,
                           const double* chiR_dev, double* G_dev, void* stream);

/* EOFA coefficients (Sec. 2): k and Omega_pm with Delta_pm = k Omega Omega^T.
 * Omega_plus, Omega_minus: host arrays of Ls doubles (may be NULL). */
int eofa_coefficients(int Ls, double alpha, double m1, double m2, double* k,
                      double* Omega_plus, double* Omega_minus);

/* The two solves behind Eq. (5) and Eq. (7), into caller buffers:
 * chi_L = H(m1)^{-1} Omega_- P_- phi, chi_R = [H(m2) - Delta_+ P_+]^{-1} Omega_+ P_+ phi
 * (5D canonical, device); S (may be NULL) gets the action. */
int eofa_pseudofermion_solutions_dev(eofa_ctx* ctx, int Ls, double alpha, double M5, double m1, double m2,
                                     int precision, double tol, const double* phi_dev, double* chiL_dev,
                                     double* chiR_dev, double* S, eofa_solve_info info[2], void* stream);

/* Reliable-update reduction delta in [0, 1) (as eofa_solve_params.delta)
 * used by the solves inside eofa_action / eofa_force / eofa_leapfrog_dev and
 * the HMC entry points (0, the default, picks the precision's default). */
int eofa_set_reliable_delta(eofa_ctx* ctx, double delta);

/* CG iteration form of the solves on this context at one precision
 * (EOFA_PREC_*; the form applies to the inner iterations).  Both forms are
 * the same CG on the normal equations of Sec. 5.1 and give the same
 * iterates up to rounding:
 *   EOFA_CG_FORM_FIVE: five fused launches per iteration; the normal
 *     residual s = A^+ r is carried by the update s -= alpha A^+ q;
 *   EOFA_CG_FORM_SIX: six fused launches that stream fewer bytes; s is
 *     formed from r every iteration.
 * EOFA_CG_FORM_AUTO (the default) times both forms, on real iterations of
 * the first solve that runs a chunk of at least six iterations outside
 * stream capture, and keeps the faster for the context's lifetime; until
 * then the five-launch form runs below 2^22 five-dimensional sites per
 * checkerboard and the six-launch form above.  Setting AUTO again forgets
 * the timed choice.  eofa_get_cg_form writes the form in use, or
 * EOFA_CG_FORM_AUTO while it is undecided.  EOFA_EINVAL for a bad
 * precision or form. */
#define EOFA_CG_FORM_AUTO (-1)
#define EOFA_CG_FORM_FIVE 0
#define EOFA_CG_FORM_SIX 1
int eofa_set_cg_form(eofa_ctx* ctx, int precision, int form);
int eofa_get_cg_form(const eofa_ctx* ctx, int precision, int* form);

/* Leapfrog molecular-dynamics trajectory for H = sum_links tr P^2 + S_EOFA
 * (Eq. (5), force Eq. (7)): P <- P - dtau/2 F, then nsteps times
 * {U <- exp(i dtau P) U; P <- P - dtau F} with the last momentum step halved.
 * P_dev (4 V traceless Hermitian 3x3, canonical) is updated in place; the
 * context's gauge field and U_dev (canonical copy, may be NULL) end at the
 * final links.  dH = H(end) - H(start); H0 (may be NULL) = H(start). */
int eofa_leapfrog_dev(eofa_ctx* ctx, int Ls, double alpha, double M5, double m1, double m2, int precision,
                      double tol, int nsteps, double dtau, const double* phi_dev, double* P_dev, double* U_dev,
                      double* dH, double* H0, void* stream);

/* Rational approximation for the heatbath (Sec. 3.2):
 * x^{-1/2} ~ alpha0 + sum_{l<npoles} alpha[l] / (x + beta[l]) on [lmin, lmax]
 * (0 < lmin < lmax), Zolotarev's optimal relative approximation; max_rel_err
 * (may be NULL) gets its maximum relative error.  alpha, beta: host arrays of
 * npoles (1..64) doubles.  Host-only: needs no GPU. */
int eofa_rational_inv_sqrt(int npoles, double lmin, double lmax, double* alpha0, double* alpha, double* beta,
                           double* max_rel_err);

/* EOFA heatbath, Eq. (6): phi = f(M_EOFA) eta with f(x) = alpha0 + sum_l
 * alphas[l] / (x + betas[l]) (betas > 0), from 2 npoles solves of Eq. (8).
 * eta, phi: 4D canonical device fields.  forecast = 1 starts each solve from
 * the minimal-residual combination of up to 6 earlier solutions of the same
 * family (chronological inversion, Sec. 5.2); 0 starts from zero.  info (may
 * be NULL) gets 2 npoles records: pole l, P_- system at 2l, P_+ at 2l + 1. */
int eofa_heatbath_dev(eofa_ctx* ctx, int Ls, double alpha, double M5, double m1, double m2, int precision,
                      double tol, int npoles, double alpha0, const double* alphas, const double* betas,
                      const double* eta_dev, double* phi_dev, int forecast, eofa_solve_info* info, void* stream);

/* Wilson plaquette gauge action (the gauge part of the HMC runs of Sec. 5;
 * the paper's Iwasaki / DSDR actions are not reproduced):
 *   S_g = (beta / 3) sum_{x, mu < nu} Re tr (1 - U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+)
 * on canonical links U_dev (device, 4 V 3x3; NULL = the context's links),
 * periodic in every direction.  S (host) gets the value; synchronous. */
int eofa_gauge_action_dev(eofa_ctx* ctx, double beta, const double* U_dev, double* S, void* stream);

/* Gauge force F_mu(x) = sum_a T^a dS_g/dw^a for U_mu(x) -> exp(i w T^a) U_mu(x)
 * (the convention of eofa_force), traceless Hermitian, canonical 4 V 3x3 on
 * the device; accumulate = 1 adds it to F_dev, 0 overwrites. */
int eofa_gauge_force_dev(eofa_ctx* ctx, double beta, const double* U_dev, double* F_dev, int accumulate,
                         void* stream);

/* HMC molecular-dynamics trajectory (Sec. 5) for
 * H = sum_links tr P^2 + S_g(beta) + S_EOFA(phi) with U <- exp(i h P) U and
 * P <- P - h F.  Integrators: leapfrog; the fourth-order force-gradient
 * schemes PQPQP = P(h/6) Q(h/2) P~(2h/3) Q(h/2) P(h/6) and
 * QPQPQ = Q(lam h) P~(h/2) Q((1-2 lam) h) P~(h/2) Q(lam h), lam = 1/2 - sqrt(3)/6,
 * where P~ kicks with the force at exp(-i z F(U)) U, z = h^2/24 (PQPQP) or
 * (2 - sqrt 3) h^2/12 (QPQPQ).  n_inner > 0 nests the gauge force: the EOFA
 * force sits on the outer level and every outer drift is n_inner steps of
 * the same scheme for S_g.  split_lr = 1 or 2 integrates the two terms of
 * Eq. (5) on separate time scales (Sexton-Weingarten): one EOFA term on the
 * outer level (S_R for 1, S_L for 2), the other with n_middle steps per outer
 * drift, the gauge force with n_inner steps per middle drift (beta = 0: no
 * gauge level); the larger force belongs on the finer level.  phi_dev =
 * NULL integrates the gauge action alone (n_inner must then be 0); beta = 0
 * drops the gauge action. */
#define EOFA_INT_LEAPFROG 0
#define EOFA_INT_FG_PQPQP 1
#define EOFA_INT_FG_QPQPQ 2
typedef struct {
    int Ls;
    double alpha, M5, m1, m2;
    int precision;   /* of the solves, EOFA_PREC_* */
    double tol;
    double beta;     /* Wilson gauge coupling */
    int integrator;  /* EOFA_INT_* */
    int nsteps;      /* outer steps */
    double tau;      /* trajectory length */
    int n_inner;     /* gauge steps per drift of the level above (0: one level) */
    int split_lr;    /* 1: S_R force outermost, S_L in the middle; 2: S_L outermost, S_R in the middle */
    int n_middle;    /* with split_lr: steps of the middle force per outer drift */
} eofa_md_params;
typedef struct {
    double H0, dH;  /* H at the start, H(end) - H(start) */
    double kinetic0, kinetic1, S_gauge0, S_gauge1, S_eofa0, S_eofa1;
    int fermion_forces, gauge_forces, solver_iters;
} eofa_md_info;
/* P_dev (4 V traceless Hermitian 3x3, canonical, device) is updated in place;
 * the context's links end at U(tau) and are copied to U_dev if not NULL.
 * info: energies, force evaluations and total solver iterations. */
int eofa_hmc_trajectory_dev(eofa_ctx* ctx, const eofa_md_params* p, const double* phi_dev, double* P_dev,
                            double* U_dev, eofa_md_info* info, void* stream);

/* HMC Markov chain (Sec. 3 and Sec. 5): ntraj trajectories, each
 *   1. pseudofermion refresh phi = f(M_EOFA) eta_k by the heatbath of
 *      Eq. (6) (eofa_heatbath_dev with alpha0, alphas, betas; forecasting
 *      on), skipped when npoles = 0 (pure gauge chain, md->beta > 0);
 *   2. momenta P_k and one trajectory of eofa_hmc_trajectory_dev (md) from
 *      the current links;
 *   3. Metropolis: accept when u[k] < exp(-dH) (a NaN dH is rejected); a
 *      rejected trajectory restores the links it started from.
 * The context's links are the chain's state: they start as loaded and end
 * at the last accepted configuration (copied to U_dev, canonical, if not
 * NULL).  All random numbers are inputs: P_dev holds ntraj momentum fields
 * (each 4 V traceless Hermitian 3x3, canonical, device) drawn with density
 * exp(-tr P^2) (P = sum_a p_a T^a, p_a ~ N(0, 1)); eta_dev ntraj 4D Gaussian
 * fields with density exp(-eta^+ eta), i.e. real and imaginary parts
 * N(0, 1/2) (device; may be NULL when npoles = 0), so that phi has density
 * exp(-phi^+ M_EOFA phi); u ntraj uniforms in [0, 1) (host).  Draws from
 * other distributions give a chain that does not sample exp(-H).  info[k] gets trajectory k's record.  EOFA_EINVAL for
 * bad arguments; a failed solve or trajectory stops the chain with its
 * status (info holds the records of the trajectories before it). */
typedef struct {
    double H0, dH;        /* H at the trajectory's start, H(end) - H(start) */
    double exp_minus_dH;  /* exp(-dH) (its chain average estimates <exp(-dH)> = 1) */
    int accepted;         /* 1 if the Metropolis step accepted the trajectory */
    double plaquette;     /* average Re tr U_p / 3 after the accept/reject step */
    double S_eofa_start;  /* S_EOFA(phi) at the start: equals eta^+ eta up to the rational error */
    double eta_norm2;     /* eta^+ eta (0 when npoles = 0) */
    int solver_iters;     /* CG iterations of the heatbath and the trajectory */
    double seconds;       /* wall time of the trajectory, heatbath included */
} eofa_hmc_traj_info;
int eofa_hmc_dev(eofa_ctx* ctx, const eofa_md_params* md, int ntraj, double alpha0, int npoles,
                 const double* alphas, const double* betas, const double* P_dev, const double* eta_dev,
                 const double* u, double* U_dev, eofa_hmc_traj_info* info, void* stream);

/* Checkpoint / resume (Sec. 5 production runs restart from saved
 * configurations).  A checkpoint file holds one field in the host
 * canonical layout, the gauge field U or the momenta P (both 4 V 3x3
 * complex = 72 V doubles), after a 64-byte little-endian header: magic
 * "EOFACKPT", version 1, kind, dims {X, Y, Z, T}, the number of doubles,
 * the caller's trajectory number and the FNV-1a 64-bit checksum of the
 * data bytes.  Host-only, no GPU needed.
 *   eofa_checkpoint_write: data (host, 72 V doubles) -> path; EOFA_EINVAL for
 *     bad arguments or an unwritable path, EOFA_EDEVICE for a short write.
 *   eofa_checkpoint_read: path -> data (host, caller-owned, 72 V doubles) and
 *     traj (may be NULL); EOFA_EINVAL when the file is missing, of another
 *     kind or lattice, truncated, longer than its header says or fails the
 *     checksum (data is then left unchanged).
 * eofa_gauge_save writes the context's current links (after an HMC chain,
 * the chain's state); eofa_gauge_restore reads a gauge checkpoint of the
 * context's lattice and loads it as eofa_gauge_load does (unitarity
 * check included). */
#define EOFA_CKPT_GAUGE 0
#define EOFA_CKPT_MOMENTA 1
int eofa_checkpoint_write(const char* path, int kind, const int dims[4], long long traj, const double* data);
int eofa_checkpoint_read(const char* path, int kind, const int dims[4], long long* traj, double* data);
int eofa_gauge_save(eofa_ctx* ctx, const char* path, long long traj);
int eofa_gauge_restore(eofa_ctx* ctx, const char* path, long long* traj);

/* Molecular dynamics link update U <- exp(i eps P) U on the device gauge
 * field of the context and on the canonical copy U_dev (if not NULL);
 * P: 4 V traceless Hermitian 3x3, canonical, device. */
int eofa_link_update_dev(eofa_ctx* ctx, double eps, const double* P_dev, double* U_dev,
                         void* stream);

/* Batched solves: n systems on n contexts (contexts may share a lattice),
 * iterated together in one CUDA-graph-captured loop.  b[i], x[i]: 5D
 * canonical host buffers of context ctxs[i]. */
int eofa_solve_batched(eofa_ctx* const* ctxs, int n, const eofa_solve_params* params,
                       const double* const* b, double* const* x, eofa_solve_info* info);

/* D_DWF in (dagger = 0) or D_DWF^+ in (dagger = 1) on device buffers, with
 * the same arguments and result as eofa_dwf_apply_dev, but without
 * allocating any device memory.  The paper has no counterpart: this is a
 * service for callers that cannot call cudaMalloc when they apply the
 * operator, such as applications that hand all GPU memory to their own pool
 * allocator up front (a fresh cudaMalloc would fail or fragment the pool)
 * and latency-critical loops that cannot afford cudaMalloc's implicit device
 * synchronisation.
 *   - Temporaries live in one 16 MiB static device array per device.  It
 *     is taken, and its device address resolved, when the first context on
 *     that device is created (eofa_create, which allocates anyway), and kept
 *     until the process exits; the calls themselves load no module and do
 *     no set-up.
 *   - Size limit: the four temporaries are FP64 half-checkerboard fields
 *     of 96 V Ls bytes each, each rounded up to a multiple of 256 bytes, so
 *     the lattice must satisfy 4 * round256(96 V Ls) <= 16 MiB, about
 *     384 V Ls bytes (8^4 x 8, 8^4 x 10 and 4^4 x 64 fit; 8^4 x 16 does
 *     not).  Larger lattices are rejected with EOFA_EINVAL and a message
 *     giving both sizes.
 *   - The context must already exist with its gauge field loaded (those
 *     calls allocate) and its device must be current (else EOFA_EINVAL).
 *   - Every call uses the same array: calls that overlap on the GPU (other
 *     streams, threads or contexts at the same time) race and corrupt each
 *     other's results.  Each call writes every temporary before reading it,
 *     so nothing from an earlier call needs clearing. */
int eofa_dwf_apply_noalloc(eofa_ctx* ctx, int Ls, double alpha, double M5, double mf, int dagger,
                           const double* in_dev, double* out_dev, void* stream);

/* Instrumentation.  eofa_kernel_launches: number of CUDA kernels this
 * library has launched since it was loaded (all contexts).
 * eofa_profile_start / _stop: while on, every even-odd hop and 5D-local
 * kernel launch on the context is bracketed by CUDA events recorded on its
 * stream (at most 65536 launches); _stop waits for them and returns per-kind
 * launch counts, summed milliseconds and summed algorithmic bytes (each
 * spinor read or written once per launch, 8 links per 4D output site read
 * once: per output site 2 spinors + 576/Ls (FP32 links) or 1152/Ls (FP64)
 * bytes, plus one spinor for the axpy input y when present).  Kinds: 0..2
 * hop in FP64 / FP32 / FP16 storage, 3..5 5D-local kernel in the same
 * order. */
typedef struct {
    long long launches[6];
    double ms[6];
    double bytes[6];
} eofa_profile;
long long eofa_kernel_launches(void);
/* Measured FP64 fused multiply-add rate of the current device in TFLOP/s
 * (2 flops per FMA; 8 independent chains per thread, best of 3 timed
 * launches): the ALU roofline of the FP64 hop.  Allocates 8 bytes. */
int eofa_probe_fp64_fma(double* tflops);
int eofa_profile_start(eofa_ctx* ctx);
int eofa_profile_stop(eofa_ctx* ctx, eofa_profile* out);

#ifdef __cplusplus
}
#endif
#endif /* EOFA_H */
