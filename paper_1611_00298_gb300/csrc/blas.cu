// Vector kernels on half-checkerboard 5D fields: axpby, copies across
// precisions, and deterministic FP64 reductions (norm^2, complex dot).
//
// Reductions: a fixed grid (RED_BLOCKS blocks) strides over the sites; each
// block reduces with warp shuffles into one FP64 partial, and the last block
// to finish (atomic ticket) sums the partials in a fixed order, so results
// are bitwise reproducible and need one launch.  Results land in
// ctx->red[slot] (device) and are read back on demand.
#include "field.cuh"
#include "fused.h"

#define RED_BLOCKS 608  // 4 x 152 SMs
#define RED_THREADS 256
// reduction scratch layout (doubles, see fused.h): [0, 64) results,
// [128, 128 + 2*RED_BLOCKS) partials, then one unsigned ticket counter.
#define RED_PART_OFF 128
#define RED_TICKET_OFF (128 + 2 * RED_BLOCKS)

namespace {

template <int PO, int PI>
__global__ void axpby_kernel(Geom g, double a, const void* x, double b, void* y) {
    typedef typename Field<PO>::R RO;
    typedef typename Field<PI>::R RI;
    long long n5 = (long long)g.Vh * g.Ls;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n5; t += (long long)gridDim.x * blockDim.x) {
        int j = (int)(t / g.Ls), s = (int)(t - (long long)j * g.Ls);
        cpx<RI> xv[12];
        cpx<RO> yv[12];
        Field<PI>::load(x, j, s, g.Ls, n5, xv);
        if (b != 0.0) Field<PO>::load(y, j, s, g.Ls, n5, yv);
#pragma unroll
        for (int c = 0; c < 12; c++) {
            RO re = (RO)(a * (double)xv[c].re), im = (RO)(a * (double)xv[c].im);
            if (b != 0.0) { re += (RO)b * yv[c].re; im += (RO)b * yv[c].im; }
            yv[c] = mk(re, im);
        }
        Field<PO>::store(y, j, s, g.Ls, n5, yv);
    }
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block-reduce (a, b) then last-block finalisation into res[0], res[1]
__device__ void reduce_finish(double a, double b, double* red, int slot) {
    __shared__ double sa[RED_THREADS / 32], sb[RED_THREADS / 32];
    __shared__ bool last;
    a = warp_sum(a);
    b = warp_sum(b);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sa[w] = a; sb[w] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0, tb = 0;
        for (int k = 0; k < RED_THREADS / 32; k++) { ta += sa[k]; tb += sb[k]; }
        red[RED_PART_OFF + 2 * blockIdx.x] = ta;
        red[RED_PART_OFF + 2 * blockIdx.x + 1] = tb;
        __threadfence();
        unsigned* ticket = (unsigned*)(red + RED_TICKET_OFF);
        unsigned v = atomicAdd(ticket, 1u);
        last = (v == gridDim.x - 1);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        double ta = 0, tb = 0;
        for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
            ta += ((volatile double*)red)[RED_PART_OFF + 2 * k];
            tb += ((volatile double*)red)[RED_PART_OFF + 2 * k + 1];
        }
        ta = warp_sum(ta);
        tb = warp_sum(tb);
        __syncthreads();
        if (l == 0) { sa[w] = ta; sb[w] = tb; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double fa = 0, fb = 0;
            for (int k = 0; k < RED_THREADS / 32; k++) { fa += sa[k]; fb += sb[k]; }
            red[slot] = fa;
            red[slot + 1] = fb;
            *(unsigned*)(red + RED_TICKET_OFF) = 0u;
        }
    }
}

template <int P>
__global__ void __launch_bounds__(RED_THREADS) norm2_kernel(Geom g, const void* x, double* red, int slot) {
    typedef typename Field<P>::R R;
    long long n5 = (long long)g.Vh * g.Ls;
    double acc = 0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n5; t += (long long)gridDim.x * blockDim.x) {
        int j = (int)(t / g.Ls), s = (int)(t - (long long)j * g.Ls);
        cpx<R> v[12];
        Field<P>::load(x, j, s, g.Ls, n5, v);
        double loc = 0;
#pragma unroll
        for (int c = 0; c < 12; c++) loc += (double)v[c].re * v[c].re + (double)v[c].im * v[c].im;
        acc += loc;
    }
    reduce_finish(acc, 0.0, red, slot);
}

template <int P>
__global__ void __launch_bounds__(RED_THREADS) dot_kernel(Geom g, const void* x, const void* y, double* red, int slot) {
    typedef typename Field<P>::R R;
    long long n5 = (long long)g.Vh * g.Ls;
    double are = 0, aim = 0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n5; t += (long long)gridDim.x * blockDim.x) {
        int j = (int)(t / g.Ls), s = (int)(t - (long long)j * g.Ls);
        cpx<R> a[12], b[12];
        Field<P>::load(x, j, s, g.Ls, n5, a);
        Field<P>::load(y, j, s, g.Ls, n5, b);
#pragma unroll
        for (int c = 0; c < 12; c++) {
            are += (double)a[c].re * b[c].re + (double)a[c].im * b[c].im;
            aim += (double)a[c].re * b[c].im - (double)a[c].im * b[c].re;
        }
    }
    reduce_finish(are, aim, red, slot);
}

unsigned grid_for(long long n, int b, int sms) {
    long long nb = (n + b - 1) / b;
    long long cap = (long long)sms * 16;
    return (unsigned)(nb < cap ? (nb > 0 ? nb : 1) : cap);
}

}  // namespace

void blas_axpby(const eofa_ctx* ctx, int prec, double a, const void* x, double b, void* y, cudaStream_t st) {
    Geom g = ctx_geom(ctx);
    unsigned nb = grid_for((long long)g.Vh * g.Ls, 256, ctx->sms);
    if (prec == P64) axpby_kernel<P64, P64><<<nb, 256, 0, st>>>(g, a, x, b, y);
    else if (prec == P32) axpby_kernel<P32, P32><<<nb, 256, 0, st>>>(g, a, x, b, y);
    else axpby_kernel<P16, P16><<<nb, 256, 0, st>>>(g, a, x, b, y);
    EOFA_LAUNCHED();
}

void blas_copy(const eofa_ctx* ctx, int po, void* out, int pi, const void* in, cudaStream_t st) {
    Geom g = ctx_geom(ctx);
    unsigned nb = grid_for((long long)g.Vh * g.Ls, 256, ctx->sms);
#define CP(A, B) if (po == A && pi == B) { axpby_kernel<A, B><<<nb, 256, 0, st>>>(g, 1.0, in, 0.0, out); }
    CP(P64, P64) CP(P64, P32) CP(P64, P16) CP(P32, P64) CP(P32, P32) CP(P32, P16) CP(P16, P64) CP(P16, P32) CP(P16, P16)
#undef CP
    EOFA_LAUNCHED();
}

void blas_zero(const eofa_ctx* ctx, int prec, void* x, cudaStream_t st) {
    EOFA_CUDA(cudaMemsetAsync(x, 0, field_bytes(prec, ctx->Vh, ctx->Ls), st));
}

void blas_norm2(const eofa_ctx* ctx, int prec, const void* x, int slot, cudaStream_t st) {
    Geom g = ctx_geom(ctx);
    if (prec == P64) norm2_kernel<P64><<<RED_BLOCKS, RED_THREADS, 0, st>>>(g, x, ctx->red, slot);
    else if (prec == P32) norm2_kernel<P32><<<RED_BLOCKS, RED_THREADS, 0, st>>>(g, x, ctx->red, slot);
    else norm2_kernel<P16><<<RED_BLOCKS, RED_THREADS, 0, st>>>(g, x, ctx->red, slot);
    EOFA_LAUNCHED();
}

void blas_dot(const eofa_ctx* ctx, int prec, const void* x, const void* y, int slot, cudaStream_t st) {
    Geom g = ctx_geom(ctx);
    if (prec == P64) dot_kernel<P64><<<RED_BLOCKS, RED_THREADS, 0, st>>>(g, x, y, ctx->red, slot);
    else if (prec == P32) dot_kernel<P32><<<RED_BLOCKS, RED_THREADS, 0, st>>>(g, x, y, ctx->red, slot);
    else dot_kernel<P16><<<RED_BLOCKS, RED_THREADS, 0, st>>>(g, x, y, ctx->red, slot);
    EOFA_LAUNCHED();
}

double red_fetch(const eofa_ctx* ctx, int slot, cudaStream_t st) {
    double v;
    red_fetch_many(ctx, slot, 1, &v, st);
    return v;
}

void red_fetch_many(const eofa_ctx* ctx, int first, int n, double* out, cudaStream_t st) {
    EOFA_CUDA(cudaMemcpyAsync(ctx->red_host, ctx->red + first, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    EOFA_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k < n; k++) out[k] = ctx->red_host[k];
}

void check_device_error(const eofa_ctx* ctx, cudaStream_t st) {
    int* w = reinterpret_cast<int*>(ctx->red + RED_ERRWORD);
    int v = 0;
    EOFA_CUDA(cudaMemcpyAsync(ctx->red_host, w, sizeof(int), cudaMemcpyDeviceToHost, st));
    EOFA_CUDA(cudaStreamSynchronize(st));
    v = *reinterpret_cast<int*>(ctx->red_host);
    if (v != 0) {
        EOFA_CUDA(cudaMemsetAsync(w, 0, sizeof(int), st));
        throw eofa_error(EOFA_ETIMEOUT, "a device wait ran out of time (staged dslash)");
    }
}

size_t red_scratch_bytes() { return (size_t)RED_TOTAL_DOUBLES * sizeof(double); }
static_assert(RED_TICKET_OFF + 8 <= RED_PART, "reduction scratch regions overlap");

namespace {

// x += alpha p ; r -= alpha q ; |r|^2 -> red[slot]   (p, q, r in precision P, x in PX)
template <int P, int PX>
__global__ void __launch_bounds__(RED_THREADS) cg_update_kernel(Geom g, double alpha, const void* p, const void* q,
                                                                void* x, void* r, double* red, int slot) {
    typedef typename Field<P>::R R;
    typedef typename Field<PX>::R RX;
    long long n5 = (long long)g.Vh * g.Ls;
    double acc = 0;
    R a = (R)alpha;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n5; t += (long long)gridDim.x * blockDim.x) {
        int j = (int)(t / g.Ls), s = (int)(t - (long long)j * g.Ls);
        cpx<R> pv[12], qv[12], rv[12];
        cpx<RX> xv[12];
        Field<P>::load(p, j, s, g.Ls, n5, pv);
        Field<P>::load(q, j, s, g.Ls, n5, qv);
        Field<P>::load(r, j, s, g.Ls, n5, rv);
        Field<PX>::load(x, j, s, g.Ls, n5, xv);
        double loc = 0;
#pragma unroll
        for (int c = 0; c < 12; c++) {
            xv[c] = mk((RX)(xv[c].re + (RX)a * (RX)pv[c].re), (RX)(xv[c].im + (RX)a * (RX)pv[c].im));
            rv[c] = rv[c] - a * qv[c];
            loc += (double)rv[c].re * rv[c].re + (double)rv[c].im * rv[c].im;
        }
        acc += loc;
        Field<PX>::store(x, j, s, g.Ls, n5, xv);
        Field<P>::store(r, j, s, g.Ls, n5, rv);
    }
    reduce_finish(acc, 0.0, red, slot);
}

__global__ void __launch_bounds__(RED_THREADS) flat_dot_kernel(long long n, const double2* a, const double2* b,
                                                               double* red, int slot) {
    double re = 0, im = 0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        double2 x = a[t], y = b[t];
        re += x.x * y.x + x.y * y.y;
        im += x.x * y.y - x.y * y.x;
    }
    reduce_finish(re, im, red, slot);
}

}  // namespace

void blas_cg_update(const eofa_ctx* ctx, int prec, int prec_x, double alpha, const void* p, const void* q, void* x,
                    void* r, int slot, cudaStream_t st) {
    Geom g = ctx_geom(ctx);
#define CGU(A, B) if (prec == A && prec_x == B) cg_update_kernel<A, B><<<RED_BLOCKS, RED_THREADS, 0, st>>>(g, alpha, p, q, x, r, ctx->red, slot);
    CGU(P64, P64) CGU(P32, P32) CGU(P16, P32) CGU(P16, P16)
#undef CGU
    EOFA_LAUNCHED();
}

void blas_flat_dot(const eofa_ctx* ctx, long long ncplx, const double* a, const double* b, int slot, cudaStream_t st) {
    flat_dot_kernel<<<RED_BLOCKS, RED_THREADS, 0, st>>>(ncplx, (const double2*)a, (const double2*)b, ctx->red, slot);
    EOFA_LAUNCHED();
}
