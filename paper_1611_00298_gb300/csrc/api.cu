// C ABI: context, gauge load, operator applications (Eq. (3)), kernel-level
// entry points.  Solves, action and force live in solver.cu and eofa.cu.
#include "ops.h"
#include "api_util.h"
#include "fused.h"

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

// ------------------------------------------------------------------ context helpers

void* ctx_buffer(eofa_ctx* ctx, const std::string& name, size_t bytes) {
    auto it = ctx->bufs.find(name);
    if (it != ctx->bufs.end()) {
        if (ctx->buf_sizes[name] >= bytes) return it->second;
        cudaFree(it->second);
        ctx->bufs.erase(it);
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes < 256 ? 256 : bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw eofa_error(EOFA_ENOMEM, "cudaMalloc(" + std::to_string(bytes) + " B) for " + name + ": " +
                                          cudaGetErrorString(e));
    }
    ctx->bufs[name] = p;
    ctx->buf_sizes[name] = bytes;
    return p;
}

Geom ctx_geom(const eofa_ctx* ctx) {
    Geom g;
    g.X = ctx->dims[0];
    g.Y = ctx->dims[1];
    g.Z = ctx->dims[2];
    g.T = ctx->dims[3];
    g.Vh = ctx->Vh;
    g.Ls = ctx->Ls;
    g.nbr[0] = ctx->nbr;
    g.nbr[1] = ctx->nbr + 8LL * ctx->Vh;
    return g;
}

int fail(eofa_ctx* ctx, int code, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return code;
}

void check_ls(const eofa_ctx* ctx, int Ls) {
    if (Ls != ctx->Ls) throw eofa_error(EOFA_EINVAL, "Ls " + std::to_string(Ls) + " differs from the context's " +
                                                          std::to_string(ctx->Ls));
}

void require_gauge(const eofa_ctx* ctx) {
    if (!ctx->gauge_loaded) throw eofa_error(EOFA_EINVAL, "no gauge field loaded");
}

static void build_neighbours(eofa_ctx* ctx, std::vector<int>& nb) {
    const int X = ctx->dims[0], Y = ctx->dims[1], Z = ctx->dims[2], T = ctx->dims[3];
    const int Vh = ctx->Vh;
    nb.assign(16LL * Vh, 0);
    int n[4] = {X, Y, Z, T};
    for (int t = 0; t < T; t++)
        for (int z = 0; z < Z; z++)
            for (int y = 0; y < Y; y++)
                for (int x = 0; x < X; x++) {
                    int c[4] = {x, y, z, t};
                    int par = (x + y + z + t) & 1;
                    int i = x + X * (y + Y * (z + Z * t));
                    int j = i / 2;
                    for (int mu = 0; mu < 4; mu++)
                        for (int dirn = 0; dirn < 2; dirn++) {
                            int d[4] = {c[0], c[1], c[2], c[3]};
                            bool wrap = false;
                            if (dirn == 0) {
                                d[mu] += 1;
                                if (d[mu] == n[mu]) { d[mu] = 0; wrap = true; }
                            } else {
                                d[mu] -= 1;
                                if (d[mu] < 0) { d[mu] = n[mu] - 1; wrap = true; }
                            }
                            int in_ = d[0] + X * (d[1] + Y * (d[2] + Z * d[3]));
                            // the t-boundary phase lives in the packed t-links at t = T - 1
                            (void)wrap;
                            int e = in_ / 2;
                            nb[(size_t)par * 8 * Vh + (size_t)(2 * mu + dirn) * Vh + j] = e;
                        }
                }
}

// ------------------------------------------------------------------ operators on fields

// Full-lattice apply of D_DWF (Eq. (3)) on FP64 half-checkerboard fields:
// D_DWF = D_hop D-tilde + M; dagger: D_DWF^+ = D-tilde^T D_hop^+ + M^T.
void apply_dwf_fields(eofa_ctx* ctx, const Coeffs& c, int dagger, const void* in_e, const void* in_o, void* out_e,
                      void* out_o, cudaStream_t st) {
    size_t fb = field_bytes(P64, ctx->Vh, ctx->Ls);
    void* t_e = ctx_buffer(ctx, "dwf_te", fb);
    void* t_o = ctx_buffer(ctx, "dwf_to", fb);
    if (!dagger) {
        Op5 Dt = op_plain(c, 0, 1, 0);
        launch_op5(ctx, P64, Dt, in_e, nullptr, t_e, st);
        launch_op5(ctx, P64, Dt, in_o, nullptr, t_o, st);
        launch_hop(ctx, P64, 0, 0, t_o, out_e, st);
        launch_hop(ctx, P64, 1, 0, t_e, out_o, st);
        Op5 M = op_plain(c, 0, 2, 0);
        M.b_in = 1.0;
        launch_op5(ctx, P64, M, in_e, out_e, out_e, st);
        launch_op5(ctx, P64, M, in_o, out_o, out_o, st);
    } else {
        launch_hop(ctx, P64, 0, 1, in_o, t_e, st);
        launch_hop(ctx, P64, 1, 1, in_e, t_o, st);
        Op5 DtT = op_plain(c, 0, 1, 1);
        launch_op5(ctx, P64, DtT, t_e, nullptr, t_e, st);
        launch_op5(ctx, P64, DtT, t_o, nullptr, t_o, st);
        Op5 MT = op_plain(c, 0, 2, 1);
        MT.b_in = 1.0;
        launch_op5(ctx, P64, MT, in_e, t_e, out_e, st);
        launch_op5(ctx, P64, MT, in_o, t_o, out_o, st);
    }
}

// (D_hop + G') on FP64 half-checkerboard fields (D_EOFA of Eq. (3) plus the
// rank-one EOFA term of the system).
void apply_eofa_fields(eofa_ctx* ctx, const Op5& G, const void* in_e, const void* in_o, void* out_e, void* out_o,
                       cudaStream_t st) {
    launch_hop(ctx, P64, 0, 0, in_o, out_e, st);
    launch_hop(ctx, P64, 1, 0, in_e, out_o, st);
    Op5 g = G;
    g.a_out = 1.0;
    g.b_in = 1.0;
    launch_op5(ctx, P64, g, in_e, out_e, out_e, st);
    launch_op5(ctx, P64, g, in_o, out_o, out_o, st);
}

static void sync_ctx(eofa_ctx* ctx, cudaStream_t st) { EOFA_CUDA(cudaStreamSynchronize(st)); }

// ------------------------------------------------------------------ C ABI

extern "C" {

int eofa_create(eofa_ctx** out, const int dims[4], int Ls, int bc_t, int flags) {
    if (!out || !dims) return EOFA_EINVAL;
    *out = nullptr;
    for (int k = 0; k < 4; k++)
        if (dims[k] < 2 || (dims[k] & 1)) return EOFA_EINVAL;
    if (Ls < 1 || Ls > EOFA_MAX_LS || (bc_t != 1 && bc_t != -1) || flags != 0) return EOFA_EINVAL;
    long long V = (long long)dims[0] * dims[1] * dims[2] * dims[3];
    if (V * Ls * 12 >= (1LL << 40) || V >= (1LL << 30)) return EOFA_EINVAL;
    eofa_ctx* ctx = new eofa_ctx();
    for (int k = 0; k < 4; k++) ctx->dims[k] = dims[k];
    ctx->Ls = Ls;
    ctx->bc_t = bc_t;
    ctx->V = (int)V;
    ctx->Vh = (int)(V / 2);
    ctx->gauge_loaded = false;
    ctx->nbr = nullptr;
    ctx->gauge[0] = ctx->gauge[1] = ctx->gauge[2] = nullptr;
    ctx->canon5 = ctx->canon5b = nullptr;
    ctx->coef = ctx->red = ctx->red_host = nullptr;
    ctx->stream = nullptr;
    ctx->prof = nullptr;
    ctx->tuned = new std::map<long long, int>();
    ctx->forced_cfg = 0;
    // test hook for the bounded waits of the staged dslash: its producer issues
    // nothing, so the consumers' first wait runs out (about 1 s) and the launch
    // reports EOFA_ETIMEOUT through the device error word
    ctx->test_stall = 0;
    if (const char* env = getenv("EOFA_TEST_STALL")) ctx->test_stall = atoi(env) > 0 ? atoi(env) : 0;
    if (const char* env = getenv("EOFA_DSLASH_CONFIG")) {
        // "NS,SPT" selects the direct kernel, "NS,SPT,D" the staged one with ring
        // depth D, "NS,SPT,-K" the pipelined one with K slots per thread
        int ns = 0, spt = 0, depth = 0;
        const int n = sscanf(env, "%d,%d,%d", &ns, &spt, &depth);
        if (n >= 2 && ns >= 1 && ns <= 64 && (spt == 1 || spt == 2)) {
            ctx->forced_cfg = ns * 4 + spt;
            if (n == 3 && depth >= 2 && depth <= 8 && ns <= 32) ctx->forced_cfg = (1 << 20) | depth << 8 | ns;
            if (n == 3 && depth <= -2 && depth >= -3) ctx->forced_cfg = (1 << 21) | (-depth) << 8 | ns;
        }
    }
    ctx->rel_delta = 0.0;  // precision default
    try {
        EOFA_CUDA(cudaGetDevice(&ctx->device));
        EOFA_CUDA(cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device));
        EOFA_CUDA(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
        std::vector<int> nb;
        build_neighbours(ctx, nb);
        ctx->nbr = (int*)ctx_buffer(ctx, "nbr", nb.size() * sizeof(int));
        EOFA_CUDA(cudaMemcpy(ctx->nbr, nb.data(), nb.size() * sizeof(int), cudaMemcpyHostToDevice));
        ctx->gauge[P64] = ctx_buffer(ctx, "gauge64", (size_t)V * 4 * 9 * 16);
        ctx->gauge[P32] = ctx_buffer(ctx, "gauge32", (size_t)V * 4 * 10 * 8);
        ctx->gauge[P16] = ctx->gauge[P32];
        ctx->coef = (double*)ctx_buffer(ctx, "coef", 16 * EOFA_MAX_LS * sizeof(double));
        ctx->red = (double*)ctx_buffer(ctx, "red", red_scratch_bytes());
        EOFA_CUDA(cudaMemset(ctx->red, 0, red_scratch_bytes()));
        EOFA_CUDA(cudaMallocHost((void**)&ctx->red_host, 64 * sizeof(double)));
        noalloc_prepare(ctx->device);
    } catch (const eofa_error& e) {
        int code = e.code;
        eofa_destroy(ctx);
        return code;
    }
    *out = ctx;
    return EOFA_OK;
}

int eofa_destroy(eofa_ctx* ctx) {
    if (!ctx) return EOFA_EINVAL;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (auto& kv : ctx->bufs) cudaFree(kv.second);
    if (ctx->red_host) cudaFreeHost(ctx->red_host);
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    if (ctx->prof) {
        for (auto& e : ctx->prof->ev) cudaEventDestroy(e);
        delete ctx->prof;
    }
    delete ctx->tuned;
    delete ctx;
    return EOFA_OK;
}

const char* eofa_last_error(const eofa_ctx* ctx) {
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

int eofa_check_device(eofa_ctx* ctx, void* stream) {
    if (!ctx) return EOFA_EINVAL;
    try {
        check_device_error(ctx, (cudaStream_t)stream);
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return EOFA_OK;
}

int eofa_gauge_load_dev(eofa_ctx* ctx, const double* U_dev, void* stream) {
    if (!ctx || !U_dev) return fail(ctx, EOFA_EINVAL, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    try {
        double* worst = (double*)ctx_buffer(ctx, "unit_worst", 64);
        launch_unitarity(ctx, U_dev, worst, st);
        double w = 0;
        EOFA_CUDA(cudaMemcpyAsync(ctx->red_host, worst, sizeof(double), cudaMemcpyDeviceToHost, st));
        sync_ctx(ctx, st);
        w = ctx->red_host[0];
        if (!(w < 1e-10)) return fail(ctx, EOFA_EINVAL, "gauge field is not unitary: max |U^+U - 1| = " + std::to_string(w));
        double* canonU = (double*)ctx_buffer(ctx, "U", (size_t)ctx->V * 4 * 9 * 16);
        if (canonU != U_dev)
            EOFA_CUDA(cudaMemcpyAsync(canonU, U_dev, (size_t)ctx->V * 4 * 9 * 16, cudaMemcpyDeviceToDevice, st));
        launch_gauge_pack(ctx, canonU, st);
        sync_ctx(ctx, st);
        ctx->gauge_loaded = true;
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return EOFA_OK;
}

int eofa_gauge_load(eofa_ctx* ctx, const double* U) {
    if (!ctx || !U) return fail(ctx, EOFA_EINVAL, "null argument");
    try {
        double* canonU = (double*)ctx_buffer(ctx, "U", (size_t)ctx->V * 4 * 9 * 16);
        EOFA_CUDA(cudaMemcpyAsync(canonU, U, (size_t)ctx->V * 4 * 9 * 16, cudaMemcpyHostToDevice, ctx->stream));
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return eofa_gauge_load_dev(ctx, (const double*)ctx_buffer(ctx, "U", 0), ctx->stream);
}

long long eofa_field_bytes(const eofa_ctx* ctx, int precision) {
    if (!ctx || precision < 0 || precision > 2) return -1;
    return (long long)field_bytes(precision, ctx->Vh, ctx->Ls);
}

int eofa_hop_dev(eofa_ctx* ctx, int precision, int out_parity, int dagger, const void* in_dev, void* out_dev,
                 void* stream) {
    if (!ctx || !in_dev || !out_dev || precision < 0 || precision > 2 || (out_parity & ~1) || (dagger & ~1))
        return fail(ctx, EOFA_EINVAL, "bad argument");
    try {
        require_gauge(ctx);
        launch_hop(ctx, precision, out_parity, dagger, in_dev, out_dev, (cudaStream_t)stream);
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return EOFA_OK;
}

int eofa_schur_hop_dev(eofa_ctx* ctx, int precision, int out_parity, int dagger, int Ls, double alpha, double M5,
                       double mf, const void* in_dev, void* out_dev, void* stream) {
    if (!ctx || !in_dev || !out_dev || precision < 0 || precision > 2 || (out_parity & ~1) || (dagger & ~1))
        return fail(ctx, EOFA_EINVAL, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    try {
        check_ls(ctx, Ls);
        require_gauge(ctx);
        System5 S = system_dwf(alpha, M5, mf);
        Op5 op = dagger ? op_GinvT(ctx, S, 2, st) : op_Ginv(ctx, S, 0, st);
        fused_dslash(ctx, precision, out_parity, dagger, in_dev, out_dev, op, nullptr, 1.0, 0.0, nullptr, 0, st);
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return EOFA_OK;
}

int eofa_pack_dev(eofa_ctx* ctx, int precision, const double* canon_dev, void* even_dev, void* odd_dev, void* stream) {
    if (!ctx || !canon_dev || !even_dev || !odd_dev || precision < 0 || precision > 2)
        return fail(ctx, EOFA_EINVAL, "bad argument");
    try {
        launch_pack(ctx, precision, canon_dev, even_dev, odd_dev, (cudaStream_t)stream);
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return EOFA_OK;
}

int eofa_unpack_dev(eofa_ctx* ctx, int precision, const void* even_dev, const void* odd_dev, double* canon_dev,
                    void* stream) {
    if (!ctx || !canon_dev || !even_dev || !odd_dev || precision < 0 || precision > 2)
        return fail(ctx, EOFA_EINVAL, "bad argument");
    try {
        launch_unpack(ctx, precision, even_dev, odd_dev, canon_dev, (cudaStream_t)stream);
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return EOFA_OK;
}

int eofa_dwf_apply_dev(eofa_ctx* ctx, int Ls, double alpha, double M5, double mf, int dagger, const double* in_dev,
                       double* out_dev, void* stream) {
    if (!ctx || !in_dev || !out_dev || (dagger & ~1)) return fail(ctx, EOFA_EINVAL, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    try {
        check_ls(ctx, Ls);
        require_gauge(ctx);
        size_t fb = field_bytes(P64, ctx->Vh, ctx->Ls);
        void* ie = ctx_buffer(ctx, "ap_ie", fb);
        void* io = ctx_buffer(ctx, "ap_io", fb);
        void* oe = ctx_buffer(ctx, "ap_oe", fb);
        void* oo = ctx_buffer(ctx, "ap_oo", fb);
        launch_pack(ctx, P64, in_dev, ie, io, st);
        apply_dwf_fields(ctx, make_coeffs(alpha, M5, mf), dagger, ie, io, oe, oo, st);
        launch_unpack(ctx, P64, oe, oo, out_dev, st);
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return EOFA_OK;
}

int eofa_eofa_apply_dev(eofa_ctx* ctx, int Ls, double alpha, double M5, double mf, const double* in_dev,
                        double* out_dev, void* stream) {
    if (!ctx || !in_dev || !out_dev) return fail(ctx, EOFA_EINVAL, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    try {
        check_ls(ctx, Ls);
        require_gauge(ctx);
        size_t fb = field_bytes(P64, ctx->Vh, ctx->Ls);
        void* ie = ctx_buffer(ctx, "ap_ie", fb);
        void* io = ctx_buffer(ctx, "ap_io", fb);
        void* oe = ctx_buffer(ctx, "ap_oe", fb);
        void* oo = ctx_buffer(ctx, "ap_oo", fb);
        launch_pack(ctx, P64, in_dev, ie, io, st);
        System5 S = system_dwf(alpha, M5, mf);
        Op5 G = op_G(ctx, S, 4, st);
        apply_eofa_fields(ctx, G, ie, io, oe, oo, st);
        launch_unpack(ctx, P64, oe, oo, out_dev, st);
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return EOFA_OK;
}

static int host_wrap_5d(eofa_ctx* ctx, const double* in, double* out,
                        int (*fn)(eofa_ctx*, const double*, double*, void*, void*), void* arg) {
    try {
        size_t bytes = (size_t)ctx->V * ctx->Ls * 12 * 16;
        double* din = (double*)ctx_buffer(ctx, "host_in", bytes);
        double* dout = (double*)ctx_buffer(ctx, "host_out", bytes);
        EOFA_CUDA(cudaMemcpyAsync(din, in, bytes, cudaMemcpyHostToDevice, ctx->stream));
        int rc = fn(ctx, din, dout, ctx->stream, arg);
        if (rc != EOFA_OK) return rc;
        EOFA_CUDA(cudaMemcpyAsync(out, dout, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        EOFA_CUDA(cudaStreamSynchronize(ctx->stream));
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return EOFA_OK;
}

struct ApplyArgs {
    int Ls;
    double alpha, M5, mf;
    int dagger;
};

static int dwf_thunk(eofa_ctx* ctx, const double* in, double* out, void* st, void* a) {
    ApplyArgs* p = (ApplyArgs*)a;
    return eofa_dwf_apply_dev(ctx, p->Ls, p->alpha, p->M5, p->mf, p->dagger, in, out, st);
}

static int eofa_thunk(eofa_ctx* ctx, const double* in, double* out, void* st, void* a) {
    ApplyArgs* p = (ApplyArgs*)a;
    return eofa_eofa_apply_dev(ctx, p->Ls, p->alpha, p->M5, p->mf, in, out, st);
}

int eofa_dwf_apply(eofa_ctx* ctx, int Ls, double alpha, double M5, double mf, int dagger, const double* in,
                   double* out) {
    if (!ctx || !in || !out) return fail(ctx, EOFA_EINVAL, "null argument");
    ApplyArgs a = {Ls, alpha, M5, mf, dagger};
    return host_wrap_5d(ctx, in, out, dwf_thunk, &a);
}

int eofa_eofa_apply(eofa_ctx* ctx, int Ls, double alpha, double M5, double mf, const double* in, double* out) {
    if (!ctx || !in || !out) return fail(ctx, EOFA_EINVAL, "null argument");
    ApplyArgs a = {Ls, alpha, M5, mf, 0};
    return host_wrap_5d(ctx, in, out, eofa_thunk, &a);
}

int eofa_set_reliable_delta(eofa_ctx* ctx, double delta) {
    if (!ctx || !(delta >= 0 && delta < 1)) return fail(ctx, EOFA_EINVAL, "delta must lie in [0, 1)");
    ctx->rel_delta = delta;
    return EOFA_OK;
}

int eofa_coefficients(int Ls, double alpha, double m1, double m2, double* k, double* Omega_plus,
                      double* Omega_minus) {
    if (Ls < 1 || Ls > EOFA_MAX_LS || !(alpha > 0)) return EOFA_EINVAL;
    if (k) *k = eofa_k(Ls, alpha, m1, m2);
    eofa_omega(Ls, alpha, Omega_plus, Omega_minus);
    return EOFA_OK;
}

}  // extern "C"
