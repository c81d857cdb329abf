// Pipelined variant of the fused even-odd dslash: each thread copies the
// neighbour spinors of its next PIPE - 1 hop directions into private
// shared-memory slots with asynchronous 16-byte copies (cp.async) while it
// computes the current direction from its slot.  The copies in flight hold
// no registers, so memory-level parallelism is no longer bounded by the
// register file; the hop arithmetic, the 5D-local epilogue and the stores
// are those of the direct kernel.  Each thread reads only what it copied
// itself, so the pipeline needs no barrier (cp.async.wait_group orders a
// thread's own copies before its reads).
#pragma once

// minimum resident blocks of 256 threads per SM requested from the register allocator
#ifndef EOFA_PIPE_MINB
#define EOFA_PIPE_MINB 3
#endif

namespace dsl {
namespace {

__device__ __forceinline__ void cp16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// 16-byte chunks of one spinor per storage precision (FP16 adds a 4-byte scale)
template <int P>
struct PChunks;
template <>
struct PChunks<P64> {
    static constexpr int CH = 12, SC = 0;
};
template <>
struct PChunks<P32> {
    static constexpr int CH = 6, SC = 0;
};
template <>
struct PChunks<P16> {
    static constexpr int CH = 3, SC = 1;
};

// Slot layout: [slot][chunk][thread] 16-byte cells (a warp touches 32
// consecutive cells: conflict-free), then, in FP16, the scales [slot][thread].
template <int P>
__host__ __device__ __forceinline__ int pipe_stage_bytes(int pipe, int nthreads) {
    return pipe * nthreads * (PChunks<P>::CH * 16 + PChunks<P>::SC * 4);
}

// copies of the spinor (site jn, slice s) into slot q
template <int P, int PIPE>
__device__ __forceinline__ void pipe_issue(unsigned char* st, int q, int nt, int tid, const void* in, int jn, int s,
                                           int Ls, long long n5) {
    constexpr int CH = PChunks<P>::CH;
    const uint4* src = (const uint4*)in + (long long)jn * CH * Ls + s;
    uint4* dst = reinterpret_cast<uint4*>(st) + (q * CH) * nt + tid;
#pragma unroll
    for (int k = 0; k < CH; k++) cp16(dst + k * nt, src + k * Ls);
    if (PChunks<P>::SC) {
        const float* ssrc = (const float*)((const char*)in + n5 * 48) + (long long)jn * Ls + s;
        float* sdst = reinterpret_cast<float*>(reinterpret_cast<uint4*>(st) + PIPE * CH * nt) + q * nt + tid;
        cp4(sdst, ssrc);
    }
}

// the spinor in slot q, unpacked as Field<P>::load would
template <int P, int PIPE>
__device__ __forceinline__ void pipe_read(const unsigned char* st, int q, int nt, int tid,
                                          cpx<typename Field<P>::R> v[12]) {
    constexpr int CH = PChunks<P>::CH;
    const uint4* b = reinterpret_cast<const uint4*>(st) + (q * CH) * nt + tid;
    if constexpr (P == P64) {
#pragma unroll
        for (int c = 0; c < 12; c++) {
            const double2 t = *reinterpret_cast<const double2*>(b + c * nt);
            v[c] = mk((typename Field<P>::R)t.x, (typename Field<P>::R)t.y);
        }
    } else if constexpr (P == P32) {
#pragma unroll
        for (int k = 0; k < 6; k++) {
            const float4 t = *reinterpret_cast<const float4*>(b + k * nt);
            v[2 * k] = mk((typename Field<P>::R)t.x, (typename Field<P>::R)t.y);
            v[2 * k + 1] = mk((typename Field<P>::R)t.z, (typename Field<P>::R)t.w);
        }
    } else {
        const float sc = reinterpret_cast<const float*>(reinterpret_cast<const uint4*>(st) + PIPE * CH * nt)[q * nt + tid];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const uint4 t = b[k * nt];
            unsigned w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int e = 0; e < 4; e++) {
                __half2 h = *reinterpret_cast<__half2*>(&w[e]);
                float2 f = __half22float2(h);
                v[4 * k + e] = mk((typename Field<P>::R)(f.x * sc), (typename Field<P>::R)(f.y * sc));
            }
        }
    }
}

// one hop direction d = 2 mu + dirn from slot q
template <int P, int DAG, int D, int PIPE>
__device__ __forceinline__ void pipe_dir(const unsigned char* st, int q, int nt, int tid, const Geom& g, int par, int j,
                                         int jn, const void* gauge, cpx<typename Field<P>::R>* acc) {
    typedef typename Field<P>::R R;
    constexpr int MU = D >> 1, DIRN = D & 1;
    cpx<R> h[6];
    {
        cpx<R> psi[12];
        pipe_read<P, PIPE>(st, q, nt, tid, psi);
        if (DIRN == 0) project<MU, DAG ? 1 : -1>(psi, h);
        else project<MU, DAG ? -1 : 1>(psi, h);
    }
    const long long lidx = DIRN == 0 ? (long long)((par * 4 + MU) * g.Vh + j) : (long long)(((1 - par) * 4 + MU) * g.Vh + jn);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        cpx<R> u[3];
        link_row<R>(gauge, lidx, a, DIRN == 1, u);
        if (DIRN == 0) mac_row<MU, DAG ? 1 : -1>(u, a, h, acc);
        else mac_row<MU, DAG ? -1 : 1>(u, a, h, acc);
    }
}

template <int P, int DAG, int LS, bool HASOP, int PIPE>
__global__ void __launch_bounds__(256, EOFA_PIPE_MINB) dslash_pipe_kernel(
    Geom g, int par, const void* __restrict__ in, void* out, const void* __restrict__ gauge, Op5 op, const void* y,
    double a_out, double b_in, double* red, int slot, int NS) {
    typedef typename Field<P>::R R;
    extern __shared__ __align__(128) unsigned char smraw[];
    const int nt = blockDim.x;
    unsigned char* st = smraw;
    cpx<R>* sm = reinterpret_cast<cpx<R>*>(smraw + pipe_stage_bytes<P>(PIPE, nt));
    const int Ls = LS > 0 ? LS : g.Ls;
    const int LsP = Ls + 1;
    const long long n5 = (long long)g.Vh * Ls;
    const int tid = threadIdx.x;
    const int ls = tid / Ls, s = tid - ls * Ls;
    const bool active_thread = ls < NS;
    const int ntiles = (g.Vh + NS - 1) / NS;
    const R scale = (R)(-0.5 * a_out);
    const int* nb = par ? g.nbr[1] : g.nbr[0];
    __shared__ R wv_s[HASOP ? 4 * EOFA_MAX_LS : 1];
    if (HASOP) {
        stage_wv<R>(op, Ls, wv_s);
        __syncthreads();
    }
    double nacc = 0.0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int j = tile * NS + ls;
        const bool site_ok = active_thread && j < g.Vh;
        int ent[8];
#pragma unroll
        for (int d = 0; d < 8; d++) ent[d] = site_ok ? __ldg(nb + d * g.Vh + j) : 0;
        cpx<R> acc[12];
#pragma unroll
        for (int c = 0; c < 12; c++) acc[c] = mk(R(0), R(0));
#pragma unroll
        for (int d = 0; d < PIPE - 1; d++) {
            if (site_ok) pipe_issue<P, PIPE>(st, d % PIPE, nt, tid, in, ent[d], s, Ls, n5);
            cp_commit();
        }
#define PIPE_STEP(D)                                                                                         \
    {                                                                                                        \
        if (D + PIPE - 1 < 8 && site_ok)                                                                     \
            pipe_issue<P, PIPE>(st, (D + PIPE - 1) % PIPE, nt, tid, in, ent[(D + PIPE - 1) & 7], s, Ls, n5); \
        cp_commit();                                                                                         \
        cp_wait<PIPE - 1>();                                                                                 \
        if (site_ok) pipe_dir<P, DAG, D, PIPE>(st, D % PIPE, nt, tid, g, par, j, ent[D], gauge, acc);        \
    }
        PIPE_STEP(0) PIPE_STEP(1) PIPE_STEP(2) PIPE_STEP(3) PIPE_STEP(4) PIPE_STEP(5) PIPE_STEP(6) PIPE_STEP(7)
#undef PIPE_STEP
        if (HASOP) {
            if (site_ok) {
#pragma unroll
                for (int c = 0; c < 12; c++) sts(sm + (ls * 12 + c) * LsP + s, acc[c]);
            }
            __syncthreads();
            const int nsites = min(NS, g.Vh - tile * NS);
            for (int idx = threadIdx.x; idx < nsites * 12; idx += blockDim.x)
                column_op<R, LS>(op, idx % 12, sm + idx * LsP, Ls, wv_s);
            __syncthreads();
            if (site_ok) {
#pragma unroll
                for (int c = 0; c < 12; c++) acc[c] = lds(sm + (ls * 12 + c) * LsP + s);
            }
        }
        if (site_ok) {
#pragma unroll
            for (int c = 0; c < 12; c++) acc[c] = scale * acc[c];
            if (y != nullptr) {
                cpx<R> yv[12];
                Field<P>::load(y, j, s, Ls, n5, yv);
                const R bb = (R)b_in;
#pragma unroll
                for (int c = 0; c < 12; c++) acc[c] = acc[c] + bb * yv[c];
            }
            Field<P>::store(out, j, s, Ls, n5, acc);
            if (red) nacc += site_norm2<R>(acc);
        }
        if (HASOP) __syncthreads();
    }
    cp_wait<0>();
    if (red) grid_sum(nacc, red, slot);
}

}  // namespace
}  // namespace dsl
