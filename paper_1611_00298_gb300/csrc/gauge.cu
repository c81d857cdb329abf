// Wilson plaquette gauge action and its force on the canonical links
// (U[i][mu][a][b], i = x + X (y + Y (z + Z t)), periodic), the gauge part of
// the HMC Hamiltonian that the paper's EOFA runs integrate beside the
// fermion force (Sec. 5):
//   S_g = (beta / 3) sum_{x, mu < nu} Re tr (1 - U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+),
//   F_mu(x) = sum_a T^a dS_g / dw^a  (U_mu(x) -> exp(i w T^a) U_mu(x))
//           = -i (beta / 12) [(X - X^+) - tr (X - X^+) / 3],  X = U_mu(x) A_mu(x),
// with A_mu(x) the sum of the six staples around U_mu(x).  FP64 throughout;
// one thread per site (action) or per link (force); the action's sum is a
// fixed-order two-pass reduction (bitwise reproducible).
#include "api_util.h"

namespace {

struct M3 {
    double2 e[9];
};

__device__ __forceinline__ double2 cm(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__device__ __forceinline__ double2 cmc(double2 a, double2 b) {
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// conj(a) * b
__device__ __forceinline__ double2 ccm(double2 a, double2 b) {
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

__device__ __forceinline__ M3 ld(const double2* U, long long i, int mu) {
    M3 m;
    const double2* p = U + (i * 4 + mu) * 9;
#pragma unroll
    for (int k = 0; k < 9; k++) m.e[k] = __ldg(p + k);
    return m;
}

// a b
__device__ __forceinline__ M3 mul(const M3& a, const M3& b) {
    M3 c;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            double2 s = cm(a.e[3 * i], b.e[j]);
            s = cadd(s, cm(a.e[3 * i + 1], b.e[3 + j]));
            c.e[3 * i + j] = cadd(s, cm(a.e[3 * i + 2], b.e[6 + j]));
        }
    return c;
}
// a b^+
__device__ __forceinline__ M3 mul_nd(const M3& a, const M3& b) {
    M3 c;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            double2 s = cmc(a.e[3 * i], b.e[3 * j]);
            s = cadd(s, cmc(a.e[3 * i + 1], b.e[3 * j + 1]));
            c.e[3 * i + j] = cadd(s, cmc(a.e[3 * i + 2], b.e[3 * j + 2]));
        }
    return c;
}
// a^+ b
__device__ __forceinline__ M3 mul_dn(const M3& a, const M3& b) {
    M3 c;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            double2 s = ccm(a.e[i], b.e[j]);
            s = cadd(s, ccm(a.e[3 + i], b.e[3 + j]));
            c.e[3 * i + j] = cadd(s, ccm(a.e[6 + i], b.e[6 + j]));
        }
    return c;
}

struct Lat {
    int d[4];
    long long V;
};

__device__ __forceinline__ long long step(const Lat& L, long long i, int mu, int sign) {
    long long stride = 1;
    for (int k = 0; k < mu; k++) stride *= L.d[k];
    const int c = (int)((i / stride) % L.d[mu]);
    int cn = c + sign;
    if (cn < 0) cn += L.d[mu];
    if (cn >= L.d[mu]) cn -= L.d[mu];
    return i + (long long)(cn - c) * stride;
}

// per block: sum over its sites of sum_{mu<nu} (3 - Re tr U_mu,nu(x))
__global__ void __launch_bounds__(256) plaquette_kernel(Lat L, const double2* __restrict__ U, double* part) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double v = 0.0;
    if (i < L.V) {
        for (int mu = 0; mu < 4; mu++) {
            const long long xm = step(L, i, mu, 1);
            const M3 Um = ld(U, i, mu);
            for (int nu = mu + 1; nu < 4; nu++) {
                const M3 A = mul(Um, ld(U, xm, nu));                  // U_mu(x) U_nu(x+mu)
                const M3 B = mul(ld(U, i, nu), ld(U, step(L, i, nu, 1), mu));  // U_nu(x) U_mu(x+nu)
                double tr = 0.0;                                       // Re tr (A B^+)
#pragma unroll
                for (int k = 0; k < 9; k++) tr += A.e[k].x * B.e[k].x + A.e[k].y * B.e[k].y;
                v += 3.0 - tr;
            }
        }
    }
    __shared__ double ws[8];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += ws[w];
        part[blockIdx.x] = t;
    }
}

// fixed-order sum of n partials into out[0], scaled
__global__ void __launch_bounds__(256) sum_kernel(const double* part, int n, double scale, double* out) {
    __shared__ double ws[8];
    double v = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) v += part[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += ws[w];
        out[0] = scale * t;
    }
}

// F_mu(x) (= or +=) the gauge force, one thread per link
__global__ void __launch_bounds__(128) gauge_force_kernel(Lat L, const double2* __restrict__ U, double beta,
                                                          int accumulate, double2* F) {
    const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (l >= 4 * L.V) return;
    const long long i = l >> 2;
    const int mu = (int)(l & 3);
    const long long xpm = step(L, i, mu, 1);
    M3 A;
#pragma unroll
    for (int k = 0; k < 9; k++) A.e[k] = make_double2(0.0, 0.0);
    for (int nu = 0; nu < 4; nu++) {
        if (nu == mu) continue;
        // U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
        const M3 up = mul_nd(mul_nd(ld(U, xpm, nu), ld(U, step(L, i, nu, 1), mu)), ld(U, i, nu));
#pragma unroll
        for (int k = 0; k < 9; k++) A.e[k] = cadd(A.e[k], up.e[k]);
        {
            // U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu) = (U_mu(x-nu) U_nu(x+mu-nu))^+ U_nu(x-nu)
            const long long xmn = step(L, i, nu, -1);
            const M3 w = mul(ld(U, xmn, mu), ld(U, step(L, xpm, nu, -1), nu));
            const M3 d2 = mul_dn(w, ld(U, xmn, nu));
#pragma unroll
            for (int k = 0; k < 9; k++) A.e[k] = cadd(A.e[k], d2.e[k]);
        }
    }
    const M3 X = mul(ld(U, i, mu), A);
    // M = X - X^+ (anti-Hermitian); F = -i (beta / 12) (M - tr M / 3)
    double2 Mv[9];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const double2 x = X.e[3 * a + b], y = X.e[3 * b + a];
            Mv[3 * a + b] = make_double2(x.x - y.x, x.y + y.y);
        }
    const double trim = (Mv[0].y + Mv[4].y + Mv[8].y) / 3.0;  // tr M is imaginary
    const double c = beta / 12.0;
    double2* out = F + l * 9;
#pragma unroll
    for (int k = 0; k < 9; k++) {
        double2 m = Mv[k];
        if (k == 0 || k == 4 || k == 8) m.y -= trim;
        const double2 f = make_double2(c * m.y, -c * m.x);  // -i c m
        out[k] = accumulate ? cadd(out[k], f) : f;
    }
}

inline unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

Lat lat_of(const eofa_ctx* ctx) {
    Lat L;
    for (int k = 0; k < 4; k++) L.d[k] = ctx->dims[k];
    L.V = ctx->V;
    return L;
}

}  // namespace

double gauge_action_now(eofa_ctx* ctx, const double* U, double beta, cudaStream_t st) {
    const Lat L = lat_of(ctx);
    const unsigned nb = nblk(L.V, 256);
    double* part = (double*)ctx_buffer(ctx, "gauge_part", (size_t)(nb + 1) * sizeof(double));
    plaquette_kernel<<<nb, 256, 0, st>>>(L, (const double2*)U, part);
    EOFA_LAUNCHED();
    sum_kernel<<<1, 256, 0, st>>>(part, (int)nb, beta / 3.0, part + nb);
    EOFA_LAUNCHED();
    EOFA_CUDA(cudaMemcpyAsync(ctx->red_host, part + nb, sizeof(double), cudaMemcpyDeviceToHost, st));
    EOFA_CUDA(cudaStreamSynchronize(st));
    return ctx->red_host[0];
}

void gauge_force_launch(eofa_ctx* ctx, const double* U, double beta, int accumulate, double* F, cudaStream_t st) {
    const Lat L = lat_of(ctx);
    gauge_force_kernel<<<nblk(4 * L.V, 128), 128, 0, st>>>(L, (const double2*)U, beta, accumulate, (double2*)F);
    EOFA_LAUNCHED();
}

extern "C" {

int eofa_gauge_action_dev(eofa_ctx* ctx, double beta, const double* U_dev, double* S, void* stream) {
    if (!ctx || !S) return fail(ctx, EOFA_EINVAL, "null argument");
    try {
        const double* U = U_dev;
        if (!U) {
            require_gauge(ctx);
            U = (const double*)ctx_buffer(ctx, "U", 0);
        }
        *S = gauge_action_now(ctx, U, beta, (cudaStream_t)stream);
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return EOFA_OK;
}

int eofa_gauge_force_dev(eofa_ctx* ctx, double beta, const double* U_dev, double* F_dev, int accumulate,
                         void* stream) {
    if (!ctx || !F_dev) return fail(ctx, EOFA_EINVAL, "null argument");
    try {
        const double* U = U_dev;
        if (!U) {
            require_gauge(ctx);
            U = (const double*)ctx_buffer(ctx, "U", 0);
        }
        gauge_force_launch(ctx, U, beta, accumulate ? 1 : 0, F_dev, (cudaStream_t)stream);
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return EOFA_OK;
}

}  // extern "C"
