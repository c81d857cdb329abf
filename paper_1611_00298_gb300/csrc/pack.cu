// Layout conversion kernels: host-canonical FP64 fields <-> device layouts.
#include "field.cuh"

namespace {

// full lexicographic index of checkerboard site j of parity p
__device__ __forceinline__ int cb_to_lex(const Geom& g, int j, int p) {
    int i0 = 2 * j;
    int x0 = i0 % g.X;
    int rest = i0 / g.X;
    int y = rest % g.Y;
    int z = (rest / g.Y) % g.Z;
    int t = rest / (g.Y * g.Z);
    int x = x0 + ((p + y + z + t) & 1);
    return x + g.X * (y + g.Y * (z + g.Z * t));
}

template <int P>
__global__ void pack_kernel(Geom g, int V, const double* __restrict__ canon, void* even, void* odd) {
    typedef typename Field<P>::R R;
    long long n5 = (long long)g.Vh * g.Ls;
    long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (tid >= 2 * n5) return;
    int p = tid >= n5;
    long long t = tid - p * n5;
    int j = (int)(t / g.Ls), s = (int)(t % g.Ls);
    int i = cb_to_lex(g, j, p);
    const double2* src = (const double2*)canon + ((long long)s * V + i) * 12;
    cpx<R> v[12];
#pragma unroll
    for (int c = 0; c < 12; c++) {
        double2 z = src[c];
        v[c] = mk((R)z.x, (R)z.y);
    }
    Field<P>::store(p ? odd : even, j, s, g.Ls, n5, v);
}

template <int P>
__global__ void unpack_kernel(Geom g, int V, const void* even, const void* odd, double* __restrict__ canon) {
    typedef typename Field<P>::R R;
    long long n5 = (long long)g.Vh * g.Ls;
    long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (tid >= 2 * n5) return;
    int p = tid >= n5;
    long long t = tid - p * n5;
    int j = (int)(t / g.Ls), s = (int)(t % g.Ls);
    int i = cb_to_lex(g, j, p);
    cpx<R> v[12];
    Field<P>::load(p ? odd : even, j, s, g.Ls, n5, v);
    double2* dst = (double2*)canon + ((long long)s * V + i) * 12;
#pragma unroll
    for (int c = 0; c < 12; c++) dst[c] = make_double2((double)v[c].re, (double)v[c].im);
}

// The time-boundary phase bc_t multiplies the packed t-links on the last
// time slice: the forward hop from t = T - 1 and the backward hop from t = 0
// are the only hops that use them, and both cross the boundary.
__global__ void gauge_pack_kernel(Geom g, double bc_t, const double* __restrict__ canon, double2* g64, float2* g32) {
    long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long nl = 2LL * 4 * g.Vh;
    if (tid >= nl) return;
    int j = (int)(tid % g.Vh);
    int mu = (int)((tid / g.Vh) % 4);
    int p = (int)(tid / (4LL * g.Vh));
    int i = cb_to_lex(g, j, p);
    const double2* src = (const double2*)canon + ((long long)i * 4 + mu) * 9;
    const double ph = (mu == 3 && i / (g.X * g.Y * g.Z) == g.T - 1) ? bc_t : 1.0;
    for (int k = 0; k < 9; k++) {
        double2 z = src[k];
        z.x *= ph;
        z.y *= ph;
        g64[tid * 9 + k] = z;
        g32[tid * 10 + k] = make_float2((float)z.x, (float)z.y);
    }
    g32[tid * 10 + 9] = make_float2(0.f, 0.f);  // pad: 80-byte links, five 16-byte loads
}

// max over links of |U^+ U - 1|_max, via atomicMax on the bit pattern (values >= 0)
__global__ void unitarity_kernel(long long nlinks, const double* __restrict__ canon, unsigned long long* out) {
    long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double worst = 0.0;
    if (l < nlinks) {
        const double2* u = (const double2*)canon + l * 9;
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                double re = 0, im = 0;
                for (int k = 0; k < 3; k++) {
                    double2 x = u[k * 3 + a], y = u[k * 3 + b];  // conj(U_ka) U_kb
                    re += x.x * y.x + x.y * y.y;
                    im += x.x * y.y - x.y * y.x;
                }
                if (a == b) re -= 1.0;
                double m = fmax(fabs(re), fabs(im));
                if (!(m <= 1e300)) m = 1e300;  // NaN / Inf -> huge
                worst = fmax(worst, m);
            }
    }
    for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(worst));
}

// R5 gamma5 on a canonical 5D field: out(s) = gamma5 in(Ls-1-s)
__global__ void rs5_kernel(long long V12, int Ls, const double2* __restrict__ in, double2* __restrict__ out) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= V12 * Ls) return;
    int s = (int)(t / V12);
    long long r = t - s * V12;
    int c = (int)(r % 12);
    double2 z = in[(long long)(Ls - 1 - s) * V12 + r];
    if (c >= 6) z = make_double2(-z.x, -z.y);
    out[t] = z;
}

inline unsigned blocks(long long n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

void launch_pack(const eofa_ctx* ctx, int prec, const double* canon, void* even, void* odd, cudaStream_t st) {
    Geom g = ctx_geom(ctx);
    long long n = 2LL * g.Vh * g.Ls;
    if (prec == P64) pack_kernel<P64><<<blocks(n, 256), 256, 0, st>>>(g, ctx->V, canon, even, odd);
    else if (prec == P32) pack_kernel<P32><<<blocks(n, 256), 256, 0, st>>>(g, ctx->V, canon, even, odd);
    else pack_kernel<P16><<<blocks(n, 256), 256, 0, st>>>(g, ctx->V, canon, even, odd);
    EOFA_LAUNCHED();
}

void launch_unpack(const eofa_ctx* ctx, int prec, const void* even, const void* odd, double* canon, cudaStream_t st) {
    Geom g = ctx_geom(ctx);
    long long n = 2LL * g.Vh * g.Ls;
    if (prec == P64) unpack_kernel<P64><<<blocks(n, 256), 256, 0, st>>>(g, ctx->V, even, odd, canon);
    else if (prec == P32) unpack_kernel<P32><<<blocks(n, 256), 256, 0, st>>>(g, ctx->V, even, odd, canon);
    else unpack_kernel<P16><<<blocks(n, 256), 256, 0, st>>>(g, ctx->V, even, odd, canon);
    EOFA_LAUNCHED();
}

void launch_gauge_pack(const eofa_ctx* ctx, const double* canon, cudaStream_t st) {
    Geom g = ctx_geom(ctx);
    long long n = 8LL * g.Vh;
    gauge_pack_kernel<<<blocks(n, 256), 256, 0, st>>>(g, (double)ctx->bc_t, canon, (double2*)ctx->gauge[P64],
                                                      (float2*)ctx->gauge[P32]);
    EOFA_LAUNCHED();
}

void launch_unitarity(const eofa_ctx* ctx, const double* canon, double* out_max, cudaStream_t st) {
    long long nl = 4LL * ctx->V;
    EOFA_CUDA(cudaMemsetAsync(out_max, 0, sizeof(double), st));
    unitarity_kernel<<<blocks(nl, 256), 256, 0, st>>>(nl, canon, (unsigned long long*)out_max);
    EOFA_LAUNCHED();
}

void launch_rs5(const eofa_ctx* ctx, const double* in, double* out, cudaStream_t st) {
    long long V12 = 12LL * ctx->V;
    long long n = V12 * ctx->Ls;
    rs5_kernel<<<blocks(n, 256), 256, 0, st>>>(V12, ctx->Ls, (const double2*)in, (double2*)out);
    EOFA_LAUNCHED();
}
