// Even-odd Wilson hop on every s-slice (the hopping part of D_w, Sec. 2).
//
//   out(x, s) = -1/2 sum_mu [ (1 - g_mu) U_mu(x) in(x + mu, s)
//                            + (1 + g_mu) U_mu(x - mu)^+ in(x - mu, s) ]
//
// for the output sites x of one parity; the dagger form swaps the two
// projectors (D_hop^+ = gamma_5 D_hop gamma_5).  In the chiral basis
// gamma_mu = [[0, A_mu], [A_mu^+, 0]] with A = -i sigma_1, -i sigma_2,
// -i sigma_3, 1 for mu = x, y, z, t, so (1 + sg gamma_mu) psi has upper
// half h = psi_u + sg A psi_l and lower half sg A^+ h: each direction
// projects to a half spinor (2 spins x 3 colours), multiplies it by one
// SU(3) link and rebuilds the lower half.  One thread per output 5D site
// (j, s), s fastest, so the Ls threads of a 4D site read the same eight
// links (served by L1 broadcast) and adjacent 16-byte chunks of the
// neighbour spinors.
#include "field.cuh"

namespace {

// A_mu psi_l for the pair (l0, l1) of colour vectors: results (a0, a1)
template <int MU, typename R>
__device__ __forceinline__ void apply_A(const cpx<R>* l0, const cpx<R>* l1, cpx<R>* a0, cpx<R>* a1) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        if (MU == 0) { a0[c] = mitimes(l1[c]); a1[c] = mitimes(l0[c]); }
        if (MU == 1) { a0[c] = mk(-l1[c].re, -l1[c].im); a1[c] = l0[c]; }
        if (MU == 2) { a0[c] = mitimes(l0[c]); a1[c] = itimes(l1[c]); }
        if (MU == 3) { a0[c] = l0[c]; a1[c] = l1[c]; }
    }
}

// A_mu^+ (w0, w1)
template <int MU, typename R>
__device__ __forceinline__ void apply_Adag(const cpx<R>* w0, const cpx<R>* w1, cpx<R>* a0, cpx<R>* a1) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        if (MU == 0) { a0[c] = itimes(w1[c]); a1[c] = itimes(w0[c]); }
        if (MU == 1) { a0[c] = w1[c]; a1[c] = mk(-w0[c].re, -w0[c].im); }
        if (MU == 2) { a0[c] = itimes(w0[c]); a1[c] = mitimes(w1[c]); }
        if (MU == 3) { a0[c] = w0[c]; a1[c] = w1[c]; }
    }
}

template <typename R>
__device__ __forceinline__ void su3_mul(const Link<R>& U, const cpx<R>* h, cpx<R>* w) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
        cpx<R> acc = cmul(U.m[3 * a], h[0]);
        acc = acc + cmul(U.m[3 * a + 1], h[1]);
        acc = acc + cmul(U.m[3 * a + 2], h[2]);
        w[a] = acc;
    }
}

template <typename R>
__device__ __forceinline__ void su3_dag_mul(const Link<R>& U, const cpx<R>* h, cpx<R>* w) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
        cpx<R> acc = cjmul(U.m[a], h[0]);
        acc = acc + cjmul(U.m[3 + a], h[1]);
        acc = acc + cjmul(U.m[6 + a], h[2]);
        w[a] = acc;
    }
}

// one direction: acc += (1 + sg gamma_mu) V psi, V = U or U^+, times phase
template <int MU, int SG, bool DAGLINK, typename R>
__device__ __forceinline__ void hop_dir(const cpx<R>* psi, const Link<R>& U, R phase, cpx<R>* acc) {
    cpx<R> a0[3], a1[3], h0[3], h1[3], w0[3], w1[3];
    apply_A<MU>(psi + 6, psi + 9, a0, a1);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        h0[c] = SG > 0 ? psi[c] + a0[c] : psi[c] - a0[c];
        h1[c] = SG > 0 ? psi[3 + c] + a1[c] : psi[3 + c] - a1[c];
    }
    if (DAGLINK) { su3_dag_mul(U, h0, w0); su3_dag_mul(U, h1, w1); }
    else { su3_mul(U, h0, w0); su3_mul(U, h1, w1); }
#pragma unroll
    for (int c = 0; c < 3; c++) { w0[c] = phase * w0[c]; w1[c] = phase * w1[c]; }
    apply_Adag<MU>(w0, w1, a0, a1);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        acc[c] = acc[c] + w0[c];
        acc[3 + c] = acc[3 + c] + w1[c];
        acc[6 + c] = SG > 0 ? acc[6 + c] + a0[c] : acc[6 + c] - a0[c];
        acc[9 + c] = SG > 0 ? acc[9 + c] + a1[c] : acc[9 + c] - a1[c];
    }
}

template <int P, int DAG, int MU>
__device__ __forceinline__ void hop_mu(const Geom& g, int par, int j, int s, long long n5, const void* in,
                                       const void* gauge, cpx<typename Field<P>::R>* acc) {
    typedef typename Field<P>::R R;
    cpx<R> psi[12];
    Link<R> U;
    // forward neighbour: (1 - g) U_mu(x) psi(x + mu); dagger: (1 + g)
    int e = __ldg(g.nbr[par] + (2 * MU) * g.Vh + j);
    int jn = e & 0x7fffffff;
    R ph = e < 0 ? R(-1) : R(1);
    Field<P>::load(in, jn, s, g.Ls, n5, psi);
    load_link<R>(gauge, ((long long)par * 4 + MU) * g.Vh + j, U);
    hop_dir<MU, DAG ? 1 : -1, false>(psi, U, ph, acc);
    // backward neighbour: (1 + g) U_mu(x - mu)^+ psi(x - mu); dagger: (1 - g)
    e = __ldg(g.nbr[par] + (2 * MU + 1) * g.Vh + j);
    jn = e & 0x7fffffff;
    ph = e < 0 ? R(-1) : R(1);
    Field<P>::load(in, jn, s, g.Ls, n5, psi);
    load_link<R>(gauge, ((long long)(1 - par) * 4 + MU) * g.Vh + jn, U);
    hop_dir<MU, DAG ? -1 : 1, true>(psi, U, ph, acc);
}

template <int P, int DAG>
__global__ void __launch_bounds__(128) hop_kernel(Geom g, int par, const void* __restrict__ in,
                                                  void* __restrict__ out, const void* __restrict__ gauge) {
    typedef typename Field<P>::R R;
    long long n5 = (long long)g.Vh * g.Ls;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= n5) return;
    int j = (int)(t / g.Ls), s = (int)(t - (long long)j * g.Ls);
    cpx<R> acc[12];
#pragma unroll
    for (int c = 0; c < 12; c++) acc[c] = mk(R(0), R(0));
    hop_mu<P, DAG, 0>(g, par, j, s, n5, in, gauge, acc);
    hop_mu<P, DAG, 1>(g, par, j, s, n5, in, gauge, acc);
    hop_mu<P, DAG, 2>(g, par, j, s, n5, in, gauge, acc);
    hop_mu<P, DAG, 3>(g, par, j, s, n5, in, gauge, acc);
#pragma unroll
    for (int c = 0; c < 12; c++) acc[c] = R(-0.5) * acc[c];
    Field<P>::store(out, j, s, g.Ls, n5, acc);
}

}  // namespace

void launch_hop(const eofa_ctx* ctx, int prec, int out_parity, int dagger, const void* in, void* out,
                cudaStream_t st) {
    Geom g = ctx_geom(ctx);
    long long n5 = (long long)g.Vh * g.Ls;
    unsigned nb = (unsigned)((n5 + 127) / 128);
    const void* gauge = ctx->gauge[prec == P64 ? P64 : P32];
    prof_begin(ctx, prec, st);
#define HOP_CASE(PP)                                                                             \
    if (dagger) hop_kernel<PP, 1><<<nb, 128, 0, st>>>(g, out_parity, in, out, gauge);            \
    else hop_kernel<PP, 0><<<nb, 128, 0, st>>>(g, out_parity, in, out, gauge);
    if (prec == P64) { HOP_CASE(P64) }
    else if (prec == P32) { HOP_CASE(P32) }
    else { HOP_CASE(P16) }
#undef HOP_CASE
    EOFA_LAUNCHED();
    prof_end(ctx, st);
}
