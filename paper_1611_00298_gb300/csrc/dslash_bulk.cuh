// Staged variant of the fused even-odd dslash: the neighbour rows reach
// shared memory through bulk asynchronous copies (cp.async.bulk, completion
// counted in bytes on an mbarrier) instead of per-thread global loads.
//
// Layout facts it relies on: a 4D site's spinors on all Ls slices form one
// contiguous row (chunk-major, s innermost: 96 Ls bytes in FP32), and a link
// is one 80-byte (FP32) or 144-byte (FP64) record.  A block owns NS whole
// 4D sites; per tile the eight hop directions (mu, forward / backward) and,
// for the axpy, the y rows are the stages of a ring of D shared-memory
// buffers.  One producer warp gathers stage by stage: lane i reads the
// neighbour index of site i and copies that neighbour's row and the link
// into the ring slot.  The consumer warps (one thread per (site, s)) wait
// for the slot, project / multiply / accumulate from shared memory, and
// release the slot; the 5D-local epilogue and the stores are those of the
// direct kernel.  Memory in flight is bounded by the ring, not by
// registers, so a few warps per SM keep HBM busy.
//
// Every wait is bounded (about a second of %globaltimer): a wait that runs
// out writes EOFA_DEV_TIMEOUT to the error word, marks the block aborted
// (later waits return at once, later copies are not issued), and the block
// runs to its end through the same barriers, so nothing hangs.  Before
// exiting, the producer waits (bounded) for the copies it issued.
#pragma once

namespace dsl {
namespace {

#define EOFA_DEV_TIMEOUT 1
#define BULK_MAX_THREADS 288

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of the given parity; false (and the block marked
// aborted) after about a second, or at once when the block is aborted.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, volatile int* abort_flag, int* err,
                                          bool honour_abort = true) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 0; it < (1u << 26); it++) {
        if (mbar_try(bar, parity)) return true;
        if (honour_abort && *abort_flag) return false;
        if ((it & 63) == 63 && global_ns() - t0 > 1000000000ull) break;
    }
    *abort_flag = 1;
    if (err) atomicExch(err, EOFA_DEV_TIMEOUT);
    return false;
}

// bulk copy of n bytes (multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned n, unsigned bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(n), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void consumer_sync(int nthreads) {
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// Row geometry of one 4D site: the spinor row as stored in HBM (RB bytes per
// slice) and, in FP16, the row of per-slice scales (SB bytes per slice).
template <int P>
struct SRow;
template <>
struct SRow<P64> {
    static constexpr int RB = 192, SB = 0, LB = 144;
    static __device__ __forceinline__ void load(const unsigned char* row, const float*, int s, int Ls,
                                                cpx<double> v[12]) {
        const double2* b = reinterpret_cast<const double2*>(row) + s;
#pragma unroll
        for (int c = 0; c < 12; c++) {
            const double2 t = b[c * Ls];
            v[c] = mk(t.x, t.y);
        }
    }
};
template <>
struct SRow<P32> {
    static constexpr int RB = 96, SB = 0, LB = 80;
    static __device__ __forceinline__ void load(const unsigned char* row, const float*, int s, int Ls,
                                                cpx<float> v[12]) {
        const float4* b = reinterpret_cast<const float4*>(row) + s;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            const float4 t = b[k * Ls];
            v[2 * k] = mk(t.x, t.y);
            v[2 * k + 1] = mk(t.z, t.w);
        }
    }
};
template <>
struct SRow<P16> {
    static constexpr int RB = 48, SB = 4, LB = 80;
    static __device__ __forceinline__ void load(const unsigned char* row, const float* scale, int s, int Ls,
                                                cpx<float> v[12]) {
        const uint4* b = reinterpret_cast<const uint4*>(row) + s;
        const float sc = scale[s];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const uint4 t = b[k * Ls];
            unsigned w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int e = 0; e < 4; e++) {
                __half2 h = *reinterpret_cast<__half2*>(&w[e]);
                float2 f = __half22float2(h);
                v[4 * k + e] = mk(f.x * sc, f.y * sc);
            }
        }
    }
};

// Shared-memory plan of one block (host and device agree on it).  A ring
// slot holds NS spinor rows, then NS scale rows (FP16), then NS links, each
// group contiguous so that neighbours with consecutive indices arrive in one
// copy.
struct BulkPlan {
    int row_b, sc_off, lk_off, stage_b, col_b, ring_b, total_b;
};

template <int P, typename R>
__host__ __device__ __forceinline__ BulkPlan bulk_plan(int NS, int D, int Ls, bool hasop) {
    BulkPlan b;
    b.row_b = SRow<P>::RB * Ls;
    b.sc_off = NS * b.row_b;
    b.lk_off = b.sc_off + NS * SRow<P>::SB * Ls;
    b.stage_b = (b.lk_off + NS * SRow<P>::LB + 127) / 128 * 128;
    b.ring_b = D * b.stage_b;
    b.col_b = hasop ? (NS * 12 * (Ls + 1) * (int)sizeof(cpx<R>) + 127) / 128 * 128 : 0;
    // + full[D], empty[D] (8 bytes each), abort flag
    b.total_b = b.ring_b + b.col_b + 16 * D + 16;
    return b;
}

// One hop direction from a staged ring slot: neighbour spinor from the row
// of site ls, link from the slot's link records (row of U, or of U^+).
template <int P, int DAG, int MU, int DIRN, typename R>
__device__ __forceinline__ void staged_dir(const unsigned char* stage, const BulkPlan& pl, int ls, int s, int Ls,
                                           cpx<R>* acc) {
    cpx<R> h[6];
    {
        cpx<R> psi[12];
        SRow<P>::load(stage + ls * pl.row_b, reinterpret_cast<const float*>(stage + pl.sc_off) + ls * Ls, s, Ls, psi);
        if (DIRN == 0) project<MU, DAG ? 1 : -1>(psi, h);
        else project<MU, DAG ? -1 : 1>(psi, h);
    }
    const cpx<R>* lk = reinterpret_cast<const cpx<R>*>(stage + pl.lk_off + ls * SRow<P>::LB);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        cpx<R> u[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            if (DIRN == 0) u[k] = lk[3 * a + k];
            else {
                const cpx<R> t = lk[3 * k + a];
                u[k] = mk(t.re, -t.im);
            }
        }
        if (DIRN == 0) mac_row<MU, DAG ? 1 : -1>(u, a, h, acc);
        else mac_row<MU, DAG ? -1 : 1>(u, a, h, acc);
    }
}

// Ring cursor shared by the producer and the consumers (same sequence).
struct Ring {
    int slot, phase, D;
    __device__ __forceinline__ void next() {
        if (++slot == D) { slot = 0; phase ^= 1; }
    }
};

template <int P, int DAG, int LS, bool HASOP>
__global__ void __launch_bounds__(BULK_MAX_THREADS, 2) dslash_bulk_kernel(
    Geom g, int par, const void* __restrict__ in, void* out, const void* __restrict__ gauge, Op5 op, const void* y,
    double a_out, double b_in, double* red, int slot, int NS, int D, int* err, int stall) {
    typedef typename Field<P>::R R;
    extern __shared__ __align__(128) unsigned char smraw[];
    const int Ls = LS > 0 ? LS : g.Ls;
    const BulkPlan pl = bulk_plan<P, R>(NS, D, Ls, HASOP);
    unsigned char* ring = smraw;
    cpx<R>* col = reinterpret_cast<cpx<R>*>(smraw + pl.ring_b);
    unsigned long long* full = reinterpret_cast<unsigned long long*>(smraw + pl.ring_b + pl.col_b);
    unsigned long long* empty = full + D;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + D);
    const int NC = (NS * Ls + 31) / 32 * 32;  // consumer threads
    const int nd = y != nullptr ? 9 : 8;      // stages per tile
    const long long n5 = (long long)g.Vh * Ls;
    const int ntiles = (g.Vh + NS - 1) / NS;
    __shared__ R wv_s[HASOP ? 4 * EOFA_MAX_LS : 1];
    if (HASOP) stage_wv<R>(op, Ls, wv_s);  // the barrier after the mbarrier set-up covers it
    if (threadIdx.x == 0) {
        for (int k = 0; k < D; k++) {
            mbar_init(smem_addr(full + k), 1);
            mbar_init(smem_addr(empty + k), NC / 32);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    double nacc = 0.0;
    if (threadIdx.x >= NC) {
        // ---------------- producer warp
        const int lane = threadIdx.x - NC;
        const int* nb = par ? g.nbr[1] : g.nbr[0];
        const size_t row_b = (size_t)SRow<P>::RB * Ls;
        const unsigned char* inb = static_cast<const unsigned char*>(in);
        const unsigned char* yb = static_cast<const unsigned char*>(y);
        const unsigned char* gb = static_cast<const unsigned char*>(gauge);
        Ring rg{0, 0, D}, after_last{0, 0, D};
        int issued = 0;
        bool ok = !stall;  // stall (test hook): issue nothing, so the consumers' waits run out
        int e[8], en[8];
        int tile = blockIdx.x;
        if (tile < ntiles) {
            const int j = tile * NS + lane;
            const bool act = lane < NS && j < g.Vh;
#pragma unroll
            for (int d = 0; d < 8; d++) e[d] = act ? __ldg(nb + d * g.Vh + j) : 0;
        }
        for (; tile < ntiles; tile += gridDim.x) {
            const int nsites = min(NS, g.Vh - tile * NS);
            const int j = tile * NS + lane;
            const bool act = lane < nsites;
            {  // neighbour entries of the next tile, loaded while this one is issued
                const int jn2 = (tile + gridDim.x) * NS + lane;
                const bool act2 = lane < NS && tile + (int)gridDim.x < ntiles && jn2 < g.Vh;
#pragma unroll
                for (int d = 0; d < 8; d++) en[d] = act2 ? __ldg(nb + d * g.Vh + jn2) : 0;
            }
#pragma unroll
            for (int d = 0; d < 9; d++) {
                if (d == 8 && nd == 8) break;
                if (ok && issued >= D) {
                    ok = mbar_wait(smem_addr(empty + rg.slot), rg.phase ^ 1, abort_flag, err);
                    ok = __all_sync(0xffffffffu, ok);
                }
                if (ok) {
                    unsigned char* stg = ring + rg.slot * pl.stage_b;
                    const unsigned fb = smem_addr(full + rg.slot);
                    const int ed = d < 8 ? e[d] : 0;
                    const int jn = d < 8 ? ed : j;
                    const unsigned bytes =
                        (unsigned)(nsites * ((SRow<P>::RB + SRow<P>::SB) * Ls + (d < 8 ? SRow<P>::LB : 0)));
                    if (lane == 0) mbar_arrive_tx(fb, bytes);
                    __syncwarp();
                    // runs of consecutive neighbour indices travel in one copy each
                    const int prev = __shfl_up_sync(0xffffffffu, jn, 1);
                    const bool start = act && (lane == 0 || jn != prev + 1);
                    const unsigned starts = __ballot_sync(0xffffffffu, start);
                    if (start) {
                        const unsigned later = starts & (0xfffffffeu << lane);
                        const int len = (later ? __ffs(later) - 1 : nsites) - lane;
                        const unsigned char* base = d < 8 ? inb : yb;
                        bulk_g2s(smem_addr(stg + lane * pl.row_b), base + (size_t)jn * row_b,
                                 (unsigned)(len * row_b), fb);
                        if (SRow<P>::SB)
                            bulk_g2s(smem_addr(stg + pl.sc_off + lane * SRow<P>::SB * Ls),
                                     base + n5 * SRow<P>::RB + (size_t)jn * SRow<P>::SB * Ls,
                                     (unsigned)(len * SRow<P>::SB * Ls), fb);
                        if (d < 8) {
                            const int mu = d >> 1;
                            const long long lidx = (d & 1) == 0 ? (long long)(par * 4 + mu) * g.Vh + j
                                                                : (long long)((1 - par) * 4 + mu) * g.Vh + jn;
                            bulk_g2s(smem_addr(stg + pl.lk_off + lane * SRow<P>::LB), gb + lidx * SRow<P>::LB,
                                     (unsigned)(len * SRow<P>::LB), fb);
                        }
                    }
                    issued++;
                }
                rg.next();
                if (ok) after_last = rg;
            }
#pragma unroll
            for (int d = 0; d < 8; d++) e[d] = en[d];
        }
        // wait for the copies still in flight (only after an abort can any be pending)
        if (lane == 0) {
            Ring back = after_last;
            for (int k = 0; k < D && k < issued; k++) {
                back.slot = back.slot == 0 ? D - 1 : back.slot - 1;
                if (back.slot == D - 1) back.phase ^= 1;
                mbar_wait(smem_addr(full + back.slot), back.phase, abort_flag, err, false);
            }
        }
        __syncwarp();
    } else {
        // ---------------- consumers: thread (site ls, slice s)
        const int ls = threadIdx.x / Ls, s = threadIdx.x - ls * Ls;
        const int lane = threadIdx.x & 31;
        const R scale = (R)(-0.5 * a_out);
        const int LsP = Ls + 1;
        Ring rg{0, 0, D};
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const int nsites = min(NS, g.Vh - tile * NS);
            const int j = tile * NS + ls;
            const bool site_ok = ls < nsites;
            cpx<R> acc[12];
#pragma unroll
            for (int c = 0; c < 12; c++) acc[c] = mk(R(0), R(0));
#define STAGED_DIR(MU, DIRN)                                                                                 \
    {                                                                                                       \
        if (ok) ok = mbar_wait(smem_addr(full + rg.slot), rg.phase, abort_flag, err);                      \
        if (ok && site_ok)                                                                                  \
            staged_dir<P, DAG, MU, DIRN, R>(ring + rg.slot * pl.stage_b, pl, ls, s, Ls, acc);                 \
        __syncwarp();                                                                                       \
        if (lane == 0) mbar_arrive(smem_addr(empty + rg.slot));                                             \
        rg.next();                                                                                          \
    }
            STAGED_DIR(0, 0) STAGED_DIR(0, 1) STAGED_DIR(1, 0) STAGED_DIR(1, 1)
            STAGED_DIR(2, 0) STAGED_DIR(2, 1) STAGED_DIR(3, 0) STAGED_DIR(3, 1)
#undef STAGED_DIR
            if (HASOP) {
                if (site_ok) {
#pragma unroll
                    for (int c = 0; c < 12; c++) sts(col + (ls * 12 + c) * LsP + s, acc[c]);
                }
                consumer_sync(NC);
                for (int idx = threadIdx.x; idx < nsites * 12; idx += NC)
                    column_op<R, LS>(op, idx % 12, col + idx * LsP, Ls, wv_s);
                consumer_sync(NC);
                if (site_ok) {
#pragma unroll
                    for (int c = 0; c < 12; c++) acc[c] = lds(col + (ls * 12 + c) * LsP + s);
                }
            }
#pragma unroll
            for (int c = 0; c < 12; c++) acc[c] = scale * acc[c];
            if (y != nullptr) {
                if (ok) ok = mbar_wait(smem_addr(full + rg.slot), rg.phase, abort_flag, err);
                if (ok && site_ok) {
                    cpx<R> yv[12];
                    const unsigned char* stg = ring + rg.slot * pl.stage_b;
                    SRow<P>::load(stg + ls * pl.row_b, reinterpret_cast<const float*>(stg + pl.sc_off) + ls * Ls, s,
                                  Ls, yv);
                    const R bb = (R)b_in;
#pragma unroll
                    for (int c = 0; c < 12; c++) acc[c] = acc[c] + bb * yv[c];
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_addr(empty + rg.slot));
                rg.next();
            }
            if (site_ok) {
                Field<P>::store(out, j, s, Ls, n5, acc);
                if (red) nacc += site_norm2<R>(acc);
            }
            if (HASOP) consumer_sync(NC);
        }
    }
    if (red) grid_sum(nacc, red, slot);
}

}  // namespace
}  // namespace dsl
