// D_DWF apply that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they apply the
// operator: an application that has handed all GPU memory to its own pool
// allocator up front (a fresh cudaMalloc fails or fragments that pool), or a
// latency-critical loop where cudaMalloc's implicit device synchronisation is
// not acceptable.  This entry point keeps its four half-checkerboard
// temporaries in one static device array instead of the context's lazily
// allocated work buffers.  The paper has no counterpart; the operator is the
// one of eofa_dwf_apply_dev.
#include "api_util.h"

#include <mutex>

#define NOALLOC_SCRATCH_BYTES (16ull << 20)  // 16 MiB per device, taken when its first context is created
#define NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_addr[NOALLOC_MAX_DEVICES];

// Device address of g_noalloc_scratch on device dev (which must be current).
// In host code the symbol is only a host-side stand-in, so the address is
// looked up once per device with cudaGetSymbolAddress and cached.
void* scratch_on(int dev) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) throw eofa_error(EOFA_EDEVICE, "device ordinal out of range");
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            throw eofa_error(EOFA_EDEVICE, std::string("cudaGetSymbolAddress(no-allocation scratch): ") +
                                               cudaGetErrorString(e));
        g_noalloc_addr[dev] = p;
    }
    return g_noalloc_addr[dev];
}

inline size_t round256(size_t n) { return (n + 255) & ~size_t(255); }

}  // namespace

// Called by eofa_create with the context's device current.  CUDA loads this
// file's module (and with it the 16 MiB array) lazily, on the first use of
// one of its symbols; resolving the address here makes that load, and its
// allocation, happen while the context is created (a call that allocates
// anyway), so that eofa_dwf_apply_noalloc itself never loads a module.
void noalloc_prepare(int dev) { (void)scratch_on(dev); }

extern "C" int eofa_dwf_apply_noalloc(eofa_ctx* ctx, int Ls, double alpha, double M5, double mf, int dagger,
                                      const double* in_dev, double* out_dev, void* stream) {
    if (!ctx || !in_dev || !out_dev || (dagger & ~1)) return fail(ctx, EOFA_EINVAL, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    try {
        check_ls(ctx, Ls);
        require_gauge(ctx);
        int cur = -1;
        EOFA_CUDA(cudaGetDevice(&cur));
        if (cur != ctx->device)
            throw eofa_error(EOFA_EINVAL, "make the context's device current before eofa_dwf_apply_noalloc");
        const size_t fb = round256(field_bytes(P64, ctx->Vh, ctx->Ls));
        if (4 * fb > NOALLOC_SCRATCH_BYTES)
            throw eofa_error(EOFA_EINVAL, "lattice too large for eofa_dwf_apply_noalloc: needs " +
                                              std::to_string(4 * fb) + " bytes of scratch, the static limit is " +
                                              std::to_string(NOALLOC_SCRATCH_BYTES) + " (384 V Ls bytes max)");
        unsigned char* base = (unsigned char*)scratch_on(cur);
        // Every temporary below is fully written before it is read, so nothing
        // left by an earlier call needs clearing.
        void* A = base;
        void* B = base + fb;
        void* C = base + 2 * fb;
        void* D = base + 3 * fb;
        Coeffs c = make_coeffs(alpha, M5, mf);
        launch_pack(ctx, P64, in_dev, A, B, st);  // A = psi_e, B = psi_o
        if (!dagger) {
            // D_DWF = D_hop D-tilde + M
            launch_op5(ctx, P64, op_plain(c, 0, 1, 0), B, nullptr, C, st);  // C = D-tilde psi_o
            launch_hop(ctx, P64, 0, 0, C, D, st);                            // D = D_eo C
            Op5 M = op_plain(c, 0, 2, 0);
            M.b_in = 1.0;
            launch_op5(ctx, P64, M, A, D, D, st);                           // D = M psi_e + D  (out_e)
            launch_op5(ctx, P64, op_plain(c, 0, 1, 0), A, nullptr, C, st);  // C = D-tilde psi_e
            launch_hop(ctx, P64, 1, 0, C, A, st);                            // A = D_oe C
            launch_op5(ctx, P64, M, B, A, A, st);                           // A = M psi_o + A  (out_o)
            launch_unpack(ctx, P64, D, A, out_dev, st);
        } else {
            // D_DWF^+ = D-tilde^T D_hop^+ + M^T
            Op5 DtT = op_plain(c, 0, 1, 1);
            Op5 MT = op_plain(c, 0, 2, 1);
            MT.b_in = 1.0;
            launch_hop(ctx, P64, 0, 1, B, C, st);        // C = D^+_eo psi_o
            launch_op5(ctx, P64, DtT, C, nullptr, C, st);  // C = D-tilde^T C
            launch_op5(ctx, P64, MT, A, C, D, st);        // D = M^T psi_e + C  (out_e)
            launch_hop(ctx, P64, 1, 1, A, C, st);        // C = D^+_oe psi_e
            launch_op5(ctx, P64, DtT, C, nullptr, C, st);
            launch_op5(ctx, P64, MT, B, C, C, st);        // C = M^T psi_o + C  (out_o)
            launch_unpack(ctx, P64, D, C, out_dev, st);
        }
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return EOFA_OK;
}
