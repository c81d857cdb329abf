// 5D-local operators (the s-structure of Eq. (3)): bidiagonal-plus-corner
// matrices p + q L and their inverses, applied per 4D site and spin-colour
// component in O(Ls), plus an optional rank-one term and axpy.
//
// L_+ = down-shift with corner -m_f, L_- = L_+^T.  The inverse of
// B = p + q L_+ follows from L_+^Ls = -m_f: with r = q / p,
//   u_0 = [x_0 - m_f sum_{j>=1} (-r)^(Ls-j) x_j] / (p (1 + m_f (-r)^Ls)),
//   u_s = (x_s - q u_{s-1}) / p                 (s = 1 .. Ls-1),
// and the mirror image for L_-.  The Cayley factorisation of Eq. (3) makes
// every block used here (D-tilde, the even-odd diagonal block
// M = (4 - M5) D-tilde + 1 - L, G = M D-tilde^{-1}, G^{-1} = D-tilde M^{-1},
// their transposes, and the EOFA rank-one corrections by Sherman-Morrison)
// a product of at most one such inverse and one such matrix.
//
// A block of threads stages NS whole 4D sites (12 x Ls complex each) in
// shared memory with coalesced loads, one thread per (site, component) runs
// the recurrences over s, and the result is written back per (site, s).
#include "field.cuh"

namespace {

template <typename R>
__device__ void inv_bidiag(cpx<R>* x, int Ls, R p, R q, int dir, R mass) {
    R r = q / p;
    R mr = -r;
    R pw = 1;
    for (int k = 0; k < Ls; k++) pw *= mr;
    R N = p * (R(1) + mass * pw);
    cpx<R> acc = mk(R(0), R(0));
    if (dir == 0) {
        for (int s = 1; s < Ls; s++) acc = mr * acc + x[s];
        acc = mr * acc;
        x[0] = (R(1) / N) * (x[0] - mass * acc);
        for (int s = 1; s < Ls; s++) x[s] = (R(1) / p) * (x[s] - q * x[s - 1]);
    } else {
        for (int s = Ls - 2; s >= 0; s--) acc = mr * acc + x[s];
        acc = mr * acc;
        x[Ls - 1] = (R(1) / N) * (x[Ls - 1] - mass * acc);
        for (int s = Ls - 2; s >= 0; s--) x[s] = (R(1) / p) * (x[s] - q * x[s + 1]);
    }
}

template <typename R>
__device__ void fwd_bidiag(cpx<R>* x, int Ls, R p, R q, int dir, R mass) {
    if (dir == 0) {
        cpx<R> last = x[Ls - 1];
        for (int s = Ls - 1; s >= 1; s--) x[s] = p * x[s] + q * x[s - 1];
        x[0] = p * x[0] - (q * mass) * last;
    } else {
        cpx<R> first = x[0];
        for (int s = 0; s < Ls - 1; s++) x[s] = p * x[s] + q * x[s + 1];
        x[Ls - 1] = p * x[Ls - 1] - (q * mass) * first;
    }
}

template <int P>
__global__ void op5_kernel(Geom g, Op5 op, int NS, const void* x, const void* y,
                           void* out) {
    typedef typename Field<P>::R R;
    extern __shared__ __align__(128) unsigned char smraw[];
    cpx<R>* sm = reinterpret_cast<cpx<R>*>(smraw);
    const int Ls = g.Ls, LsP = g.Ls + 1;
    long long n5 = (long long)g.Vh * Ls;
    int j0 = blockIdx.x * NS;
    int ns = min(NS, g.Vh - j0);
    // stage: one thread per (site, s)
    for (int idx = threadIdx.x; idx < ns * Ls; idx += blockDim.x) {
        int lj = idx / Ls, s = idx - lj * Ls;
        cpx<R> v[12];
        Field<P>::load(x, j0 + lj, s, Ls, n5, v);
#pragma unroll
        for (int c = 0; c < 12; c++) sm[(lj * 12 + c) * LsP + s] = v[c];
    }
    __syncthreads();
    // columns: one thread per (site, component)
    for (int idx = threadIdx.x; idx < ns * 12; idx += blockDim.x) {
        int c = idx % 12;
        int h = c < 6 ? 0 : 1;
        cpx<R>* col = sm + idx * LsP;
        if (op.inv[h]) inv_bidiag<R>(col, Ls, (R)op.p1[h], (R)op.q1[h], op.dir1[h], (R)op.mass);
        cpx<R> d = mk(R(0), R(0));
        bool r1 = op.sigma[h] != 0.0;
        if (r1) {
            const double* v = op.v[h];
            for (int s = 0; s < Ls; s++) d = d + (R)__ldg(v + s) * col[s];
        }
        if (op.fwd[h]) fwd_bidiag<R>(col, Ls, (R)op.p2[h], (R)op.q2[h], op.dir2[h], (R)op.mass);
        if (r1) {
            const double* w = op.w[h];
            cpx<R> sd = (R)op.sigma[h] * d;
            for (int s = 0; s < Ls; s++) col[s] = col[s] + (R)__ldg(w + s) * sd;
        }
    }
    __syncthreads();
    // write back: one thread per (site, s)
    for (int idx = threadIdx.x; idx < ns * Ls; idx += blockDim.x) {
        int lj = idx / Ls, s = idx - lj * Ls;
        cpx<R> v[12];
#pragma unroll
        for (int c = 0; c < 12; c++) v[c] = (R)op.a_out * sm[(lj * 12 + c) * LsP + s];
        if (y != nullptr && op.b_in != 0.0) {
            cpx<R> yv[12];
            Field<P>::load(y, j0 + lj, s, Ls, n5, yv);
#pragma unroll
            for (int c = 0; c < 12; c++) v[c] = v[c] + (R)op.b_in * yv[c];
        }
        Field<P>::store(out, j0 + lj, s, Ls, n5, v);
    }
}

template <int P>
void run_op5(const eofa_ctx* ctx, const Op5& op, const void* x, const void* y, void* out, cudaStream_t st) {
    typedef typename Field<P>::R R;
    Geom g = ctx_geom(ctx);
    size_t per_site = (size_t)12 * (g.Ls + 1) * sizeof(cpx<R>);
    int NS = (int)(24576 / per_site);
    if (NS < 1) NS = 1;
    if (NS > 32) NS = 32;
    size_t smem = per_site * NS;
    unsigned nb = (unsigned)((g.Vh + NS - 1) / NS);
    if (smem > 40 * 1024) EOFA_CUDA(cudaFuncSetAttribute(op5_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    prof_begin(ctx, 3 + P, st);
    op5_kernel<P><<<nb, 128, smem, st>>>(g, op, NS, x, y, out);
    EOFA_LAUNCHED();
    prof_end(ctx, st);
}

}  // namespace

void launch_op5(const eofa_ctx* ctx, int prec, const Op5& op, const void* x, const void* y, void* out,
                cudaStream_t st) {
    if (prec == P64) run_op5<P64>(ctx, op, x, y, out, st);
    else if (prec == P32) run_op5<P32>(ctx, op, x, y, out, st);
    else run_op5<P16>(ctx, op, x, y, out, st);
}
