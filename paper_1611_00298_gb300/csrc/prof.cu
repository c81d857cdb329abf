// Kernel launch counter and optional CUDA-event timing of the hop and
// 5D-local kernels (events are recorded on the stream each kernel runs on).
#include "api_util.h"

long long g_launches = 0;

#define PROF_PAIRS 65536

void prof_begin(const eofa_ctx* ctx, int kind, cudaStream_t st, double bytes) {
    Prof* p = ctx->prof;
    if (!p || !p->on || p->used >= PROF_PAIRS) return;
    EOFA_CUDA(cudaEventRecord(p->ev[2 * p->used], st));
    p->kind[p->used] = kind;
    p->bytes[p->used] = bytes;
}

void prof_end(const eofa_ctx* ctx, cudaStream_t st) {
    Prof* p = ctx->prof;
    if (!p || !p->on || p->used >= PROF_PAIRS) return;
    EOFA_CUDA(cudaEventRecord(p->ev[2 * p->used + 1], st));
    p->used++;
}

extern "C" {

long long eofa_kernel_launches(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

int eofa_profile_start(eofa_ctx* ctx) {
    if (!ctx) return EOFA_EINVAL;
    try {
        if (!ctx->prof) {
            ctx->prof = new Prof();
            ctx->prof->ev.resize(2 * PROF_PAIRS);
            ctx->prof->kind.resize(PROF_PAIRS);
            ctx->prof->bytes.resize(PROF_PAIRS);
            for (auto& e : ctx->prof->ev) EOFA_CUDA(cudaEventCreate(&e));
        }
        ctx->prof->used = 0;
        ctx->prof->on = true;
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return EOFA_OK;
}

int eofa_profile_stop(eofa_ctx* ctx, eofa_profile* out) {
    if (!ctx || !out) return EOFA_EINVAL;
    for (int k = 0; k < 6; k++) {
        out->launches[k] = 0;
        out->ms[k] = 0.0;
        out->bytes[k] = 0.0;
    }
    Prof* p = ctx->prof;
    if (!p) return EOFA_OK;
    try {
        p->on = false;
        for (int i = 0; i < p->used; i++) {
            EOFA_CUDA(cudaEventSynchronize(p->ev[2 * i + 1]));
            float ms = 0.f;
            EOFA_CUDA(cudaEventElapsedTime(&ms, p->ev[2 * i], p->ev[2 * i + 1]));
            out->launches[p->kind[i]]++;
            out->ms[p->kind[i]] += ms;
            out->bytes[p->kind[i]] += p->bytes[i];
        }
        p->used = 0;
    } catch (const eofa_error& e) {
        return fail(ctx, e.code, e.msg);
    }
    return EOFA_OK;
}

}  // extern "C"
