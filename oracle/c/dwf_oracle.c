/*
 * Plain FP64 C restatement of the oracle's domain-wall operators and CG
 * (TEST INFRASTRUCTURE ONLY: loaded by the test suite and by the CPU
 * baseline of the benchmark; the product library never uses it and shares
 * no code with it).  It is the same definition as oracle/dwf.py and
 * oracle/solve.py, written as loops over sites so that the host cores can
 * be timed on the large lattices (OpenMP over 4D sites when compiled with
 * -fopenmp).
 *
 * Paper: D. Murphy, "Domain Wall Fermion Simulations with the Exact
 * One-Flavor Algorithm", Lattice 2016, Sec. 2, Eq. (3); the solve is the
 * textbook CG on the normal equations (Sec. 5.1: the cost of a trajectory
 * lies in inverting the Dirac operator).
 *
 * Conventions (the readings the numpy oracle documents and its tests pin):
 *   U    [t][z][y][x][mu][a][b]     complex (re, im interleaved), mu = x, y, z, t
 *   psi  [s][t][z][y][x][spin][c]   complex
 *   Euclidean chiral basis gamma_k = [[0, -i sigma_k], [i sigma_k, 0]],
 *   gamma_4 = [[0, 1], [1, 0]], gamma_5 = diag(1, 1, -1, -1);
 *   D_w = (4 - M5) - 1/2 sum_mu [(1 - g_mu) U_mu(x) psi(x+mu)
 *                               + (1 + g_mu) U_mu(x-mu)^+ psi(x-mu)]
 *   (D_w^+ swaps the two projectors), periodic in x, y, z, the t-hops across
 *   T-1 <-> 0 carry bc_t;  L = P+ L+ + P- L-, (L+)_{s,s-1} = 1,
 *   (L+)_{0,Ls-1} = -mf, L- = L+^T;
 *   D_DWF = ((c+d) D_w + 1) + ((c-d) D_w - 1) L with c = alpha/2, d = 1/2.
 */
#define _POSIX_C_SOURCE 199309L
#include <complex.h>
#include <math.h>
#include <time.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* gamma_mu, mu = x, y, z, t: g[mu][row][col] */
static cplx G[4][4][4];
static int g_ready = 0;

static void init_gammas(void) {
    if (g_ready) return;
    /* Pauli matrices */
    const cplx sig[3][2][2] = {{{0, 1}, {1, 0}}, {{0, -I}, {I, 0}}, {{1, 0}, {0, -1}}};
    memset(G, 0, sizeof(G));
    for (int k = 0; k < 3; k++)
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) {
                G[k][a][2 + b] = -I * sig[k][a][b];
                G[k][2 + a][b] = I * sig[k][a][b];
            }
    for (int a = 0; a < 2; a++) {
        G[3][a][2 + a] = 1;
        G[3][2 + a][a] = 1;
    }
    g_ready = 1;
}

int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* site index of (x, y, z, t) */
static long site(const int d[4], int x, int y, int z, int t) {
    return x + (long)d[0] * (y + (long)d[1] * (z + (long)d[2] * t));
}

/* out = D_w psi (dagger = 0) or D_w^+ psi (dagger = 1) on every s-slice */
void oracle_wilson(const int dims[4], int Ls, const double* Ud, const double* psid, double* outd, double M5,
                   double bc_t, int dagger) {
    init_gammas();
    const cplx* U = (const cplx*)Ud;
    const cplx* psi = (const cplx*)psid;
    cplx* out = (cplx*)outd;
    const long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
    const double sgn = dagger ? -1.0 : 1.0;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < V; i++) {
        int c[4];
        c[0] = (int)(i % dims[0]);
        c[1] = (int)((i / dims[0]) % dims[1]);
        c[2] = (int)((i / ((long)dims[0] * dims[1])) % dims[2]);
        c[3] = (int)(i / ((long)dims[0] * dims[1] * dims[2]));
        for (int s = 0; s < Ls; s++) {
            const cplx* p0 = psi + ((long)s * V + i) * 12;
            cplx acc[4][3];
            for (int sp = 0; sp < 4; sp++)
                for (int a = 0; a < 3; a++) acc[sp][a] = (4.0 - M5) * p0[sp * 3 + a];
            for (int mu = 0; mu < 4; mu++) {
                for (int dir = 0; dir < 2; dir++) {
                    /* dir 0: forward neighbour with U_mu(x); dir 1: backward with U_mu(x-mu)^+ */
                    int n[4] = {c[0], c[1], c[2], c[3]};
                    double phase = 1.0;
                    if (dir == 0) {
                        n[mu] += 1;
                        if (n[mu] == dims[mu]) {
                            n[mu] = 0;
                            if (mu == 3) phase = bc_t;
                        }
                    } else {
                        n[mu] -= 1;
                        if (n[mu] < 0) {
                            n[mu] = dims[mu] - 1;
                            if (mu == 3) phase = bc_t;
                        }
                    }
                    const long j = site(dims, n[0], n[1], n[2], n[3]);
                    const cplx* pn = psi + ((long)s * V + j) * 12;
                    const cplx* L = U + ((dir == 0 ? i : j) * 4 + mu) * 9;
                    /* v = link (or its adjoint) times the colour vector of every spin */
                    cplx v[4][3];
                    for (int sp = 0; sp < 4; sp++)
                        for (int a = 0; a < 3; a++) {
                            cplx t = 0;
                            for (int b = 0; b < 3; b++)
                                t += (dir == 0 ? L[a * 3 + b] : conj(L[b * 3 + a])) * pn[sp * 3 + b];
                            v[sp][a] = phase * t;
                        }
                    /* (1 -+ sgn g_mu) v for the forward term, (1 +- sgn g_mu) v for the backward one */
                    const double pm = dir == 0 ? -sgn : sgn;
                    for (int sp = 0; sp < 4; sp++)
                        for (int a = 0; a < 3; a++) {
                            cplx t = v[sp][a];
                            for (int q = 0; q < 4; q++) t += pm * G[mu][sp][q] * v[q][a];
                            acc[sp][a] -= 0.5 * t;
                        }
                }
            }
            cplx* o = out + ((long)s * V + i) * 12;
            for (int sp = 0; sp < 4; sp++)
                for (int a = 0; a < 3; a++) o[sp * 3 + a] = acc[sp][a];
        }
    }
}

/* out = L psi (transpose = 0) or L^T psi (transpose = 1) */
static void apply_L(long V, int Ls, const cplx* psi, cplx* out, double mf, int transpose) {
#pragma omp parallel for schedule(static)
    for (long i = 0; i < V; i++)
        for (int s = 0; s < Ls; s++)
            for (int sp = 0; sp < 4; sp++) {
                /* P+ (spins 0, 1) with L+ (down-shift), P- (spins 2, 3) with L- (up-shift);
                   the transpose swaps the shifts */
                const int down = (sp < 2) != (transpose != 0);
                int sn;
                double w = 1.0;
                if (down) {
                    sn = s - 1;
                    if (sn < 0) { sn = Ls - 1; w = -mf; }
                } else {
                    sn = s + 1;
                    if (sn == Ls) { sn = 0; w = -mf; }
                }
                for (int a = 0; a < 3; a++)
                    out[((long)s * V + i) * 12 + sp * 3 + a] = w * psi[((long)sn * V + i) * 12 + sp * 3 + a];
            }
}

/* out = D_DWF psi (Eq. (3) first line) */
void oracle_dwf(const int dims[4], int Ls, const double* U, const double* psid, double* outd, double alpha,
                double M5, double mf, double bc_t) {
    const long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
    const long n = V * Ls * 12;
    const double c = 0.5 * alpha, d = 0.5;
    const cplx* psi = (const cplx*)psid;
    cplx* out = (cplx*)outd;
    cplx* Lp = malloc(sizeof(cplx) * n);
    cplx* t = malloc(sizeof(cplx) * n);
    apply_L(V, Ls, psi, Lp, mf, 0);
    oracle_wilson(dims, Ls, U, psid, (double*)out, M5, bc_t, 0);
    oracle_wilson(dims, Ls, U, (const double*)Lp, (double*)t, M5, bc_t, 0);
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; k++) out[k] = ((c + d) * out[k] + psi[k]) + ((c - d) * t[k] - Lp[k]);
    free(Lp);
    free(t);
}

/* out = D_DWF^+ psi = ((c+d) D_w^+ + 1) psi + L^+ ((c-d) D_w^+ - 1) psi */
void oracle_dwf_dag(const int dims[4], int Ls, const double* U, const double* psid, double* outd, double alpha,
                    double M5, double mf, double bc_t) {
    const long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
    const long n = V * Ls * 12;
    const double c = 0.5 * alpha, d = 0.5;
    const cplx* psi = (const cplx*)psid;
    cplx* out = (cplx*)outd;
    cplx* Dd = malloc(sizeof(cplx) * n);
    cplx* t = malloc(sizeof(cplx) * n);
    oracle_wilson(dims, Ls, U, psid, (double*)Dd, M5, bc_t, 1);
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; k++) t[k] = (c - d) * Dd[k] - psi[k];
    apply_L(V, Ls, t, out, mf, 1);
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; k++) out[k] += (c + d) * Dd[k] + psi[k];
    free(Dd);
    free(t);
}

static double norm2(const cplx* a, long n) {
    double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (long k = 0; k < n; k++) s += creal(a[k]) * creal(a[k]) + cimag(a[k]) * cimag(a[k]);
    return s;
}

/* CG on the normal equations for D_DWF x = b (the steps of oracle/solve.py's
   cgnr: r = b - A x, z = A^+ r, p = z; then w = A p, a = |z|^2 / |w|^2,
   x += a p, r -= a w, z = A^+ r, p = z + (|z'|^2 / |z|^2) p), from x as
   given, for at most maxiter iterations or until |r| / |b| <= tol (the
   recursive residual; the caller recomputes the true one).  Returns the
   number of iterations; *rel gets the last |r| / |b|, *loop_s (may be NULL)
   the wall time of the iterations without the set-up. */
static double wall(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return ts.tv_sec + 1e-9 * ts.tv_nsec;
}

int oracle_cgnr_dwf(const int dims[4], int Ls, const double* U, const double* bd, double* xd, double alpha, double M5,
                    double mf, double bc_t, double tol, int maxiter, double* rel, double* loop_s) {
    const long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
    const long n = V * Ls * 12;
    const cplx* b = (const cplx*)bd;
    cplx* x = (cplx*)xd;
    cplx* r = malloc(sizeof(cplx) * n);
    cplx* z = malloc(sizeof(cplx) * n);
    cplx* p = malloc(sizeof(cplx) * n);
    cplx* w = malloc(sizeof(cplx) * n);
    const double bn = sqrt(norm2(b, n));
    oracle_dwf(dims, Ls, U, xd, (double*)w, alpha, M5, mf, bc_t);
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; k++) r[k] = b[k] - w[k];
    oracle_dwf_dag(dims, Ls, U, (const double*)r, (double*)z, alpha, M5, mf, bc_t);
    memcpy(p, z, sizeof(cplx) * n);
    double zz = norm2(z, n);
    double rn = sqrt(norm2(r, n)) / (bn > 0 ? bn : 1.0);
    int it = 0;
    const double t0 = wall();
    while (it < maxiter && rn > tol) {
        oracle_dwf(dims, Ls, U, (const double*)p, (double*)w, alpha, M5, mf, bc_t);
        const double a = zz / norm2(w, n);
#pragma omp parallel for schedule(static)
        for (long k = 0; k < n; k++) {
            x[k] += a * p[k];
            r[k] -= a * w[k];
        }
        it++;
        rn = sqrt(norm2(r, n)) / (bn > 0 ? bn : 1.0);
        if (rn <= tol) break;
        oracle_dwf_dag(dims, Ls, U, (const double*)r, (double*)z, alpha, M5, mf, bc_t);
        const double zn = norm2(z, n);
        const double beta = zn / zz;
        zz = zn;
#pragma omp parallel for schedule(static)
        for (long k = 0; k < n; k++) p[k] = z[k] + beta * p[k];
    }
    if (rel) *rel = rn;
    if (loop_s) *loop_s = wall() - t0;
    free(r);
    free(z);
    free(p);
    free(w);
    return it;
}
