// Internal declarations shared by the CUDA translation units of libeofa.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <string>
#include <vector>
#include <map>

#include "../../include/eofa.h"

#define EOFA_MAX_LS 64

// ------------------------------------------------------------------ complex

template <typename R>
struct cpx {
    R re, im;
};

template <typename R>
__host__ __device__ __forceinline__ cpx<R> mk(R a, R b) { cpx<R> c; c.re = a; c.im = b; return c; }
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator*(R s, cpx<R> a) { return mk(s * a.re, s * a.im); }
template <typename R>
__host__ __device__ __forceinline__ cpx<R> cmul(cpx<R> a, cpx<R> b) {
    return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// conj(a) * b
template <typename R>
__host__ __device__ __forceinline__ cpx<R> cjmul(cpx<R> a, cpx<R> b) {
    return mk(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> itimes(cpx<R> a) { return mk(-a.im, a.re); }  // i a
template <typename R>
__host__ __device__ __forceinline__ cpx<R> mitimes(cpx<R> a) { return mk(a.im, -a.re); }  // -i a

// ------------------------------------------------------------------ layouts
//
// Half-checkerboard 5D field of N5h = Vh * Ls sites, 12 complex components
// (spin-major: c = 3 * spin + colour).  Site-major with s innermost, stored in
// 16-byte chunks so that threads (j, s), (j, s + 1) read adjacent chunks:
//   FP64: chunk k = component k            -> [j][12][Ls] double2
//   FP32: chunk k = components 2k, 2k + 1  -> [j][6][Ls]  float4
//   FP16: chunk k = components 4k .. 4k+3  -> [j][3][Ls]  8 x half, plus a
//         per-site FP32 scale [j][Ls] stored after the chunks.
// Gauge field (per precision): [parity][mu][j][3x3] complex (row-major),
// forward links U_mu(x) of the sites of that parity; FP64 links take 9
// complex, FP32 links are padded to 10 complex (80 bytes, 16-byte aligned).

enum Prec { P64 = 0, P32 = 1, P16 = 2 };

inline size_t field_bytes(int prec, long long Vh, int Ls) {
    long long n5 = Vh * (long long)Ls;
    if (prec == P64) return (size_t)(n5 * 12 * 16);
    if (prec == P32) return (size_t)(n5 * 12 * 8);
    return (size_t)(n5 * 12 * 4 + n5 * 4);
}

// neighbour table entry: cb index of the neighbour, top bit = boundary phase -1
struct Geom {
    int X, Y, Z, T;
    int Vh, Ls;
    const int* nbr[2];  // [parity of the site][8][Vh]: dir 2*mu = forward, 2*mu+1 = backward
};

// 5D-local operator on each (4D site, component) column over s, per chirality
// h = 0 (P_+, components 0..5) and h = 1 (P_-, components 6..11):
//   u   = B1^{-1} x                   (if inv[h]; else u = x)
//   out = B2 u + sigma[h] w[h] (v[h] . u)   (B2 if fwd[h]; else identity)
//   out = a_out * out + b_in * y      (optional axpy with a second field y)
// with Bk = p I + q L_dir and L_dir the down-shift (dir 0, L_+ shape) or the
// up-shift (dir 1, L_- shape), both with corner -mass.
struct Op5 {
    int inv[2], fwd[2];
    double p1[2], q1[2], p2[2], q2[2];
    int dir1[2], dir2[2];
    double mass;
    double sigma[2];
    const double* w[2];  // device, Ls each
    const double* v[2];
    double a_out, b_in;  // out = a_out * op(x) + b_in * y
    // derived constants of the inverse (filled by op_finalize on the host):
    // mr = -q1/p1, invp = 1/p1, invN = 1/(p1 (1 + mass mr^Ls))
    double mr[2], invp[2], invN[2];
};
Op5 op_finalize(Op5 op, int Ls);

// Kernel launch accounting and optional per-kernel CUDA-event timing.
struct Prof {
    bool on = false;
    int used = 0;
    std::vector<cudaEvent_t> ev;  // pairs (start, stop)
    std::vector<int> kind;        // 0..2 hop per precision, 3..5 op5 per precision
    std::vector<double> bytes;    // algorithmic bytes of each launch
};
// ------------------------------------------------------------------ context

struct eofa_ctx {
    int dims[4];
    int Ls;
    int bc_t;
    int V, Vh;
    int device;
    int sms;
    cudaStream_t stream;  // default stream for host-buffer calls
    std::string err;
    bool gauge_loaded;
    // device
    int* nbr;                 // [2][8][Vh]
    void* gauge[3];           // per precision: [2][4][Vh][9] complex
    double* canon5;           // staging canonical 5D field (FP64)
    double* canon5b;
    double* coef;             // small device buffer for 5D-local vectors (16 * EOFA_MAX_LS)
    double* red;              // reduction scratch (partials + results)
    double* red_host;         // pinned host mirror of reduction results
    std::map<std::string, void*> bufs;  // named workspace fields
    std::map<std::string, size_t> buf_sizes;
    Prof* prof;
    std::map<long long, int>* tuned;  // autotuned dslash configuration (NS * 4 + SPT), by kernel key
    mutable int test_stall;           // EOFA_TEST_STALL=n: the next n staged dslash launches let a wait run out
    int forced_cfg;                   // EOFA_DSLASH_CONFIG="NS,SPT" at context creation (0: autotune)
    double rel_delta;  // reliable-update threshold of the solves inside action / force / MD
};

// ------------------------------------------------------------------ helpers

#define EOFA_CUDA(call)                                                        \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) {                                               \
            throw eofa_error(EOFA_EDEVICE, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        }                                                                      \
    } while (0)

extern long long g_launches;
void prof_begin(const struct eofa_ctx* ctx, int kind, cudaStream_t st, double bytes = 0.0);
void prof_end(const struct eofa_ctx* ctx, cudaStream_t st);

struct eofa_error {
    int code;
    std::string msg;
    eofa_error(int c, const std::string& m) : code(c), msg(m) {}
};

#define EOFA_LAUNCHED()                                                         \
    do {                                                                       \
        __atomic_add_fetch(&g_launches, 1LL, __ATOMIC_RELAXED);                \
        EOFA_CUDA(cudaGetLastError());                                         \
    } while (0)

void* ctx_buffer(eofa_ctx* ctx, const std::string& name, size_t bytes);
Geom ctx_geom(const eofa_ctx* ctx);

// kernels (launchers); all stream-ordered
void launch_pack(const eofa_ctx* ctx, int prec, const double* canon, void* even, void* odd, cudaStream_t st);
void launch_unpack(const eofa_ctx* ctx, int prec, const void* even, const void* odd, double* canon, cudaStream_t st);
void launch_gauge_pack(const eofa_ctx* ctx, const double* canon, cudaStream_t st);
void launch_unitarity(const eofa_ctx* ctx, const double* canon, double* out_max, cudaStream_t st);
void launch_hop(const eofa_ctx* ctx, int prec, int out_parity, int dagger, const void* in, void* out,
                cudaStream_t st);
void launch_op5(const eofa_ctx* ctx, int prec, const Op5& op, const void* x, const void* y, void* out,
                cudaStream_t st);

// BLAS on half-checkerboard fields of precision prec (n5 = Vh * Ls sites)
void blas_axpby(const eofa_ctx* ctx, int prec, double a, const void* x, double b, void* y, cudaStream_t st);
void blas_copy(const eofa_ctx* ctx, int prec_out, void* out, int prec_in, const void* in, cudaStream_t st);
void blas_zero(const eofa_ctx* ctx, int prec, void* x, cudaStream_t st);
// reductions: results written to ctx->red[slot]; returned to host when sync
void blas_norm2(const eofa_ctx* ctx, int prec, const void* x, int slot, cudaStream_t st);
void blas_dot(const eofa_ctx* ctx, int prec, const void* x, const void* y, int slot, cudaStream_t st);
double red_fetch(const eofa_ctx* ctx, int slot, cudaStream_t st);
void red_fetch_many(const eofa_ctx* ctx, int first, int n, double* out, cudaStream_t st);

// CG building blocks (FP64 or FP32/FP16 storage), see solver.cu
void launch_rs5(const eofa_ctx* ctx, const double* in, double* out, cudaStream_t st);  // R5 gamma5 on canonical 5D
void blas_cg_update(const eofa_ctx* ctx, int prec, int prec_x, double alpha, const void* p, const void* q, void* x,
                    void* r, int slot, cudaStream_t st);
void blas_flat_dot(const eofa_ctx* ctx, long long ncplx, const double* a, const double* b, int slot, cudaStream_t st);
size_t red_scratch_bytes();
// resolve the no-allocation entry point's static scratch on device dev (noalloc.cu)
void noalloc_prepare(int dev);
