// Multi-right-hand-side solver kernels: the fused even-odd dslash (with the
// multi-output epilogues of the CG iteration) and the CG vector update of
// dslash_impl.cuh, for nr systems on ONE lattice iterated in lock step (the 2 N_p shifted
// systems of the heatbath, the L and R systems of the action and force,
// several mass pairs: Sec. 3.2, 3.3, 5.2, Eq. (8)).
//
// The hop D_hop is the same for every system (it holds only the links); the
// 5D-local blocks differ (mass, Möbius scale, the rank-one term of Eq. (8)).
// A block owns NS sites x RB systems x Ls slices, one thread per
// (site, system, s): all RB x Ls threads of a site read the same neighbour
// indices and link rows, so each of those is fetched from DRAM once per
// launch for every system (L1 serves the rest) instead of once per system.
// Fields stay separate per system (one pointer each), so systems can leave
// the batch without moving any data.  Every system keeps its own reduction
// scratch (the per-solve `red` of solver.h): norms and the CG scalars are
// per system, reduced per block into that system's partials and finished
// by the last block of that system, in fixed order.
#pragma once
#include "dslash_impl.cuh"
#include "mrhs.h"

namespace dsl {
namespace {

template <typename R>
__device__ __forceinline__ void mr_stage(const Op5* ops, int r0, int nr, int RB, int Ls, Op5* ops_s, R* wv_s) {
    for (int i = threadIdx.x; i < RB; i += blockDim.x)
        if (r0 + i < nr) ops_s[i] = ops[r0 + i];
    __syncthreads();
    for (int i = threadIdx.x; i < RB * 4 * Ls; i += blockDim.x) {
        const int rl = i / (4 * Ls), k = i - rl * 4 * Ls;
        R v = R(0);
        if (r0 + rl < nr) {
            const Op5& op = ops_s[rl];
            const int h = k / (2 * Ls), which = (k / Ls) & 1, s = k % Ls;
            const double* src = which ? (h ? op.v[1] : op.v[0]) : (h ? op.w[1] : op.w[0]);
            const double sg = h ? op.sigma[1] : op.sigma[0];
            v = (sg != 0.0 && src) ? (R)src[s] : R(0);
        }
        wv_s[i] = v;
    }
}

// Per-system sums of nv = 1 or 2 values: every thread adds its partials
// into the block's shared slots of its system; thread rl < RB then publishes
// the block partials of system r0 + rl (at RED_PART, RED_PART2) and the last
// block of that system sums all partials in block order into red[r][slot]
// (and red[r][slot2]).
__device__ __noinline__ void mr_grid_sum(double v, double v2, int nv, int rl_mine, bool mine, double* const* reds,
                                         int r0, int nr, int RB, int slot, int slot2, double* part_s,
                                         unsigned* last_s) {
    if (mine) {
        atomicAdd(part_s + rl_mine, v);
        if (nv == 2) atomicAdd(part_s + RB + rl_mine, v2);
    }
    __syncthreads();
    if ((int)threadIdx.x < RB) {
        const int r = r0 + threadIdx.x;
        unsigned lst = 0u;
        if (r < nr) {
            double* red = reds[r];
            red[RED_PART + blockIdx.x] = part_s[threadIdx.x];
            if (nv == 2) red[RED_PART2 + blockIdx.x] = part_s[RB + threadIdx.x];
            __threadfence();
            const unsigned prev = atomicAdd((unsigned*)(red + RED_TICKET), 1u);
            lst = prev == gridDim.x - 1 ? 1u : 0u;
        }
        last_s[threadIdx.x] = lst;
    }
    __syncthreads();
    __shared__ double ws[2][32];
    for (int rl = 0; rl < RB; rl++) {
        if (!last_s[rl]) continue;  // uniform over the block
        __threadfence();
        double* red = reds[r0 + rl];
        double t = 0, t2 = 0;
        for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
            t += ((volatile double*)red)[RED_PART + k];
            if (nv == 2) t2 += ((volatile double*)red)[RED_PART2 + k];
        }
        t = warp_sum(t);
        t2 = warp_sum(t2);
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
        if (l == 0) {
            ws[0][w] = t;
            ws[1][w] = t2;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double f = 0, f2 = 0;
            for (int k = 0; k < nw; k++) {
                f += ws[0][k];
                f2 += ws[1][k];
            }
            red[slot] = f;
            if (nv == 2) red[slot2] = f2;
            *(unsigned*)(red + RED_TICKET) = 0u;
        }
        __syncthreads();
    }
}

// MODE 0: out_r = a (-1/2) B_r[hop(in_r)] + b y_r;  MODE 1: also out2_r = B2_r out_r;
// MODE 2 (B = 1): out_r <- out_r - alpha_r (a (-1/2) hop(in_r) + b y_r) and
// out2_r <- out2_r - alpha_r y_r, |out2_r|^2 -> red_r[slot2].
// |out_r|^2 -> red_r[slot] when slot >= 0.
template <int P, int DAG, int LS, bool HASOP, int MODE>
__global__ void __launch_bounds__(256, HASOP ? EOFA_DSLASH_MINB : EOFA_HOP_MINB)
    mr_dslash_kernel(Geom g, int par, MRPtrs a, const Op5* __restrict__ ops, const Op5* __restrict__ ops2, int nr,
                     int RB, const void* __restrict__ gauge, double a_out, double b_in, int slot, int NS, int it,
                     int slot2) {
    typedef typename Field<P>::R R;
    extern __shared__ __align__(128) unsigned char smraw[];
    const int Ls = LS > 0 ? LS : g.Ls;
    const int LsP = Ls + 1;
    const int r0 = blockIdx.y * RB;
    // shared layout: [Op5 x RB][Op5 x RB][wv: RB x 4 Ls][wv2][part: 2 RB doubles][last: RB][5D columns]
    Op5* ops_s = reinterpret_cast<Op5*>(smraw);
    Op5* ops2_s = reinterpret_cast<Op5*>(smraw + mr_ops_bytes(RB));
    R* wv_s = reinterpret_cast<R*>(smraw + 2 * mr_ops_bytes(RB));
    R* wv2_s = reinterpret_cast<R*>(smraw + 2 * mr_ops_bytes(RB) + mr_wv_bytes(RB, Ls));
    double* part_s = reinterpret_cast<double*>(smraw + 2 * mr_ops_bytes(RB) + 2 * mr_wv_bytes(RB, Ls));
    unsigned* last_s = reinterpret_cast<unsigned*>(part_s + 2 * RB);
    cpx<R>* sm = reinterpret_cast<cpx<R>*>(smraw + mr_head_bytes(RB, Ls));
    if (HASOP) mr_stage<R>(ops, r0, nr, RB, Ls, ops_s, wv_s);
    if (MODE == 1) mr_stage<R>(ops2, r0, nr, RB, Ls, ops2_s, wv2_s);
    for (int i = threadIdx.x; i < 2 * RB; i += blockDim.x) part_s[i] = 0.0;
    __syncthreads();
    const long long n5 = (long long)g.Vh * Ls;
    const int s = threadIdx.x % Ls;
    const int rl = (threadIdx.x / Ls) % RB;
    const int ls = threadIdx.x / (Ls * RB);
    const int r = r0 + rl;
    const bool active_thread = ls < NS && r < nr;
    const void* in = active_thread ? a.in[r] : nullptr;
    void* out = active_thread ? a.out[r] : nullptr;
    void* out2 = (MODE != 0 && active_thread) ? a.out2[r] : nullptr;
    const void* y = active_thread ? a.y[r] : nullptr;
    const R cz = (MODE == 2 && active_thread) ? (R)(-cg_alpha(a.red[r], it)) : R(0);
    const int ntiles = (g.Vh + NS - 1) / NS;
    const R scale = (R)(-0.5 * a_out);
    const int sv[1] = {s};
    const int colbase = (ls * RB + rl) * 12;
    double nacc = 0.0, nacc2 = 0.0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int j = tile * NS + ls;
        const bool site_ok = active_thread && j < g.Vh;
        cpx<R> acc[1][12];
#pragma unroll
        for (int c = 0; c < 12; c++) acc[0][c] = mk(R(0), R(0));
        if (site_ok) {
            const int* nb = par ? g.nbr[1] : g.nbr[0];
            int ent[8];
#pragma unroll
            for (int d = 0; d < 8; d++) ent[d] = __ldg(nb + d * g.Vh + j);
            hop_mu<P, DAG, 0, 1>(g, par, j, ent, sv, Ls, n5, in, gauge, acc);
            hop_mu<P, DAG, 1, 1>(g, par, j, ent, sv, Ls, n5, in, gauge, acc);
            hop_mu<P, DAG, 2, 1>(g, par, j, ent, sv, Ls, n5, in, gauge, acc);
            hop_mu<P, DAG, 3, 1>(g, par, j, ent, sv, Ls, n5, in, gauge, acc);
        }
        const int nsites = min(NS, g.Vh - tile * NS);
        if (HASOP) {
            if (site_ok) {
#pragma unroll
                for (int c = 0; c < 12; c++) sts(sm + (colbase + c) * LsP + s, acc[0][c]);
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < nsites * RB * 12; idx += blockDim.x) {
                const int c = idx % 12, rr = (idx / 12) % RB;
                if (r0 + rr < nr) column_op<R, LS>(ops_s[rr], c, sm + idx * LsP, Ls, wv_s + rr * 4 * Ls);
            }
            __syncthreads();
            if (site_ok) {
#pragma unroll
                for (int c = 0; c < 12; c++) acc[0][c] = lds(sm + (colbase + c) * LsP + s);
            }
        }
        if (site_ok) {
#pragma unroll
            for (int c = 0; c < 12; c++) acc[0][c] = scale * acc[0][c];
            if (y != nullptr) {
                cpx<R> yv[12];
                Field<P>::load_stream(y, j, s, Ls, n5, yv);
                const R bb = (R)b_in;
#pragma unroll
                for (int c = 0; c < 12; c++) acc[0][c] = acc[0][c] + bb * yv[c];
                if (MODE == 2) {
                    // out2 <- out2 - alpha y
                    cpx<R> rv[12];
                    Field<P>::load_stream(out2, j, s, Ls, n5, rv);
#pragma unroll
                    for (int c = 0; c < 12; c++) rv[c] = rv[c] + cz * yv[c];
                    Field<P>::store_stream(out2, j, s, Ls, n5, rv);
                    nacc2 += site_norm2<R>(rv);
                }
            }
            if (MODE == 2) {
                cpx<R> zv[12];
                Field<P>::load_stream(out, j, s, Ls, n5, zv);
#pragma unroll
                for (int c = 0; c < 12; c++) acc[0][c] = zv[c] + cz * acc[0][c];
            }
            Field<P>::store_stream(out, j, s, Ls, n5, acc[0]);
            if (slot >= 0) nacc += site_norm2<R>(acc[0]);
        }
        if (MODE == 1) {
            __syncthreads();
            if (site_ok) {
#pragma unroll
                for (int c = 0; c < 12; c++) sts(sm + (colbase + c) * LsP + s, acc[0][c]);
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < nsites * RB * 12; idx += blockDim.x) {
                const int c = idx % 12, rr = (idx / 12) % RB;
                if (r0 + rr < nr) column_op<R, LS>(ops2_s[rr], c, sm + idx * LsP, Ls, wv2_s + rr * 4 * Ls);
            }
            __syncthreads();
            if (site_ok) {
#pragma unroll
                for (int c = 0; c < 12; c++) acc[0][c] = lds(sm + (colbase + c) * LsP + s);
                Field<P>::store_stream(out2, j, s, Ls, n5, acc[0]);
            }
        }
        if (HASOP) __syncthreads();
    }
    if (slot >= 0)
        mr_grid_sum(nacc, nacc2, MODE == 2 ? 2 : 1, rl, active_thread, a.red, r0, nr, RB, slot, slot2, part_s, last_s);
}

// x_r += alpha_r p_r (x in PX), p_r = s_r + beta_r p_r, system r = blockIdx.y
template <int P, int PX>
__global__ void __launch_bounds__(256) mr_xp_update_kernel(Geom g, MRPtrs a, int it) {
    typedef typename Field<P>::R R;
    typedef typename Field<PX>::R RX;
    const int r = blockIdx.y;
    const long long n5 = (long long)g.Vh * g.Ls;
    const double* sc = a.red[r];
    const R alpha = (R)cg_alpha(sc, it), beta = (R)cg_beta(sc, it);
    void* x = a.out2[r];
    void* p = a.out[r];
    const void* sv_ = a.in[r];
    const unsigned n5u = (unsigned)n5, Lsu = (unsigned)g.Ls;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n5u; t += gridDim.x * blockDim.x) {
        const int j = (int)(t / Lsu);
        const int ss = (int)(t - (unsigned)j * Lsu);
        cpx<R> pv[12], sv[12];
        cpx<RX> xv[12];
        Field<P>::load_stream(p, j, ss, g.Ls, n5, pv);
        Field<P>::load_stream(sv_, j, ss, g.Ls, n5, sv);
        Field<PX>::load_stream(x, j, ss, g.Ls, n5, xv);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            xv[k] = mk((RX)(xv[k].re + (RX)alpha * (RX)pv[k].re), (RX)(xv[k].im + (RX)alpha * (RX)pv[k].im));
            pv[k] = sv[k] + beta * pv[k];
        }
        Field<PX>::store_stream(x, j, ss, g.Ls, n5, xv);
        Field<P>::store_stream(p, j, ss, g.Ls, n5, pv);
    }
}

// ---------------------------------------------------------------- launchers

// systems per block and sites per block: RB x Ls threads per site, at most
// 256 threads; NS sites so that a block has at least 96 threads
inline void mr_shape(int Ls, int nr, int& RB, int& NS) {
    RB = nr;
    while (RB > 1 && RB * Ls > 256) RB = (RB + 1) / 2;
    NS = 1;
    while (NS * 2 * RB * Ls <= 256 && NS * RB * Ls < 96) NS *= 2;
}

template <typename R>
size_t mr_smem(int RB, int NS, int Ls, bool cols) {
    return mr_head_bytes(RB, Ls) + (cols ? (size_t)NS * RB * 12 * (Ls + 1) * sizeof(cpx<R>) : 0);
}

template <int P, int DAG, int LS, bool HASOP, int MODE>
void mr_dslash_launch(const eofa_ctx* ctx, int par, const MRPtrs& a, const Op5* ops, const Op5* ops2, int nr,
                      double a_out, double b_in, int slot, int it, int slot2, cudaStream_t st) {
    typedef typename Field<P>::R R;
    Geom g = ctx_geom(ctx);
    const void* gauge = ctx->gauge[P == P64 ? P64 : P32];
    int RB, NS;
    mr_shape(g.Ls, nr, RB, NS);
    const int threads = (NS * RB * g.Ls + 31) / 32 * 32;
    const size_t smem = mr_smem<R>(RB, NS, g.Ls, HASOP || MODE == 1);
    const int ntiles = (g.Vh + NS - 1) / NS;
    auto k = mr_dslash_kernel<P, DAG, LS, HASOP, MODE>;
    if (smem > 40 * 1024) EOFA_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    unsigned gx = grid_size(k, threads, smem, ntiles, ctx->sms);
    const unsigned gy = (unsigned)((nr + RB - 1) / RB);
    // several systems per grid row: spread the SMs' resident blocks over the rows
    if (gy > 1) gx = (unsigned)std::max<long long>(1, std::min<long long>(ntiles, ((long long)gx + gy - 1) / gy));
    k<<<dim3(gx, gy), threads, smem, st>>>(g, par, a, ops, ops2, nr, RB, gauge, a_out, b_in, slot, NS, it, slot2);
    EOFA_LAUNCHED();
}

template <int P, int DAG, int LS>
void mr_dslash_t(const eofa_ctx* ctx, int par, int mode, const MRPtrs& a, const Op5* ops, const Op5* ops2, int nr,
                 bool hasop, double a_out, double b_in, int slot, int it, int slot2, cudaStream_t st) {
    if (mode == 1)
        mr_dslash_launch<P, DAG, LS, true, 1>(ctx, par, a, ops, ops2, nr, a_out, b_in, slot, it, slot2, st);
    else if (mode == 2)
        mr_dslash_launch<P, DAG, LS, false, 2>(ctx, par, a, ops, ops2, nr, a_out, b_in, slot, it, slot2, st);
    else if (hasop)
        mr_dslash_launch<P, DAG, LS, true, 0>(ctx, par, a, ops, ops2, nr, a_out, b_in, slot, it, slot2, st);
    else
        mr_dslash_launch<P, DAG, LS, false, 0>(ctx, par, a, ops, ops2, nr, a_out, b_in, slot, it, slot2, st);
}

template <int P, int PX>
void mr_xp_t(const eofa_ctx* ctx, const MRPtrs& a, int nr, int it, cudaStream_t st) {
    Geom g = ctx_geom(ctx);
    const long long n5 = (long long)g.Vh * g.Ls;
    const long long nb = (n5 + 255) / 256;
    long long cap = (long long)ctx->sms * 8 / nr;
    if (cap < 1) cap = 1;
    const unsigned gx = (unsigned)(nb < cap ? nb : cap);
    mr_xp_update_kernel<P, PX><<<dim3(gx, nr), 256, 0, st>>>(g, a, it);
    EOFA_LAUNCHED();
}

template <int P>
void mr_dslash_prec(const eofa_ctx* ctx, int par, int dag, int mode, const MRPtrs& a, const Op5* ops,
                    const Op5* ops2, int nr, bool hasop, double a_out, double b_in, int slot, int it, int slot2,
                    cudaStream_t st) {
#define MR_CASE(L)                                                                                            \
    if (dag) mr_dslash_t<P, 1, L>(ctx, par, mode, a, ops, ops2, nr, hasop, a_out, b_in, slot, it, slot2, st); \
    else mr_dslash_t<P, 0, L>(ctx, par, mode, a, ops, ops2, nr, hasop, a_out, b_in, slot, it, slot2, st);
    switch (ctx->Ls) {
        case 8: MR_CASE(8) break;
        case 12: MR_CASE(12) break;
        case 16: MR_CASE(16) break;
        case 24: MR_CASE(24) break;
        default: MR_CASE(0) break;
    }
#undef MR_CASE
}

}  // namespace
}  // namespace dsl

#define MR_DEFINE(NAME, P, PX)                                                                                \
    void mr_dslash_##NAME(const eofa_ctx* ctx, int par, int dag, int mode, const MRPtrs& a, const Op5* ops,  \
                          const Op5* ops2, int nr, bool hasop, double a_out, double b_in, int slot, int it,  \
                          int slot2, cudaStream_t st) {                                                     \
        dsl::mr_dslash_prec<P>(ctx, par, dag, mode, a, ops, ops2, nr, hasop, a_out, b_in, slot, it, slot2,  \
                               st);                                                                          \
    }                                                                                                        \
    void mr_xp_##NAME(const eofa_ctx* ctx, const MRPtrs& a, int nr, int it, cudaStream_t st) {               \
        dsl::mr_xp_t<P, PX>(ctx, a, nr, it, st);                                                             \
    }
