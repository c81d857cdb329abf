// Fused even-odd dslash kernels (templates; instantiated per storage
// precision in dslash_p64.cu, dslash_p32.cu, dslash_p16.cu).
//
//   out = a (-1/2) B[ sum_mu hop terms ] + b y,    |out|^2 -> red[slot]
//
// The hop is the Wilson hopping term of Sec. 2 on every s-slice.  B is a
// 5D-local block of Eq. (3) (Op5: per chirality an O(Ls) bidiagonal
// inverse, a bidiagonal matrix and a rank-one term) or the identity.  A
// block owns NS whole 4D sites x Ls slices:
//   phase 1  one thread per (site, s) gathers the 8 neighbours (spin
//            projection, one SU(3) link, reconstruction) into registers;
//   phase 2  (B != 1) the 12 x Ls results go through shared memory and one
//            thread per (site, component) runs the s-recurrences of B on
//            its column held in registers (Ls is a template parameter for
//            the common extents, so the recurrences unroll);
//   phase 3  one thread per (site, s) applies the axpy, stores coalesced
//            16-byte chunks and accumulates the norm.
// The grid strides over tiles of NS sites; reductions have one partial per
// block and a fixed-order final sum (bitwise reproducible).
#pragma once
#include "field.cuh"
#include "fused.h"

#include <cstdio>
#include <cstdlib>
#include <type_traits>

// minimum resident blocks of 256 threads per SM requested from the register
// allocator (3 -> at most 85 registers, 8 blocks of 96 threads per SM)
#ifndef EOFA_DSLASH_MINB
#define EOFA_DSLASH_MINB 3
#endif
#ifndef EOFA_HOP_MINB
#define EOFA_HOP_MINB 3
#endif
// 1: the axpy input y and the output of the fused dslash use streaming
// (evict-first) cache hints, leaving L2 to the neighbour spinors
#ifndef EOFA_STREAM_HINTS
#define EOFA_STREAM_HINTS 1
#endif
// 1: load the eight neighbour entries of a site before its first spinor load
#ifndef EOFA_HOP_PREFETCH
#define EOFA_HOP_PREFETCH 1
#endif

namespace dsl {
namespace {

// ---------------------------------------------------------------- packed FP32 pairs
// (re, im) of one complex number in a 64-bit register; the f32x2 instructions
// do two FP32 multiply-adds each (used by the 5D-local recurrences; the same
// form in the link products of the hop measured slower).
#ifndef EOFA_PACKED_F32
#define EOFA_PACKED_F32 1
#endif
typedef unsigned long long f2p;
__device__ __forceinline__ f2p splat2(float a) {
    f2p r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ f2p fma2(f2p a, f2p b, f2p c) {
    f2p r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f2p mul2(f2p a, f2p b) {
    f2p r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2p ld2(const cpx<float>* p) { return *reinterpret_cast<const f2p*>(p); }
__device__ __forceinline__ void st2(cpx<float>* p, f2p v) { *reinterpret_cast<f2p*>(p) = v; }


// ---------------------------------------------------------------- hop pieces

template <int MU, typename R>
__device__ __forceinline__ void apply_A(const cpx<R>* l0, const cpx<R>* l1, cpx<R>* a0, cpx<R>* a1) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        if (MU == 0) { a0[c] = mitimes(l1[c]); a1[c] = mitimes(l0[c]); }
        if (MU == 1) { a0[c] = mk(-l1[c].re, -l1[c].im); a1[c] = l0[c]; }
        if (MU == 2) { a0[c] = mitimes(l0[c]); a1[c] = itimes(l1[c]); }
        if (MU == 3) { a0[c] = l0[c]; a1[c] = l1[c]; }
    }
}

// One SU(3) row (3 complex) of a link: row a of U, or row a of U^+ (the
// conjugated column a of U).
template <typename R>
__device__ __forceinline__ void link_row(const void* g, long long idx, int a, bool dag, cpx<R>* r);

template <>
__device__ __forceinline__ void link_row<double>(const void* g, long long idx, int a, bool dag, cpx<double>* r) {
    const double2* b = (const double2*)g + idx * 9;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        double2 t = __ldg(b + (dag ? 3 * k + a : 3 * a + k));
        r[k] = dag ? mk(t.x, -t.y) : mk(t.x, t.y);
    }
}

// 1: a forward FP32 link row (three consecutive elements of the 80-byte
// record) is read with one 16-byte and one 8-byte load instead of three
#ifndef EOFA_WIDE_LINK_ROWS
#define EOFA_WIDE_LINK_ROWS 1
#endif

template <>
__device__ __forceinline__ void link_row<float>(const void* g, long long idx, int a, bool dag, cpx<float>* r) {
    const float2* b = (const float2*)g + idx * 10;
    if (EOFA_WIDE_LINK_ROWS && !dag) {
        const float4* b4 = (const float4*)g + idx * 5;
        if (a == 0) {
            const float4 t = __ldg(b4);
            const float2 u = __ldg(b + 2);
            r[0] = mk(t.x, t.y);
            r[1] = mk(t.z, t.w);
            r[2] = mk(u.x, u.y);
        } else if (a == 1) {
            const float2 u = __ldg(b + 3);
            const float4 t = __ldg(b4 + 2);
            r[0] = mk(u.x, u.y);
            r[1] = mk(t.x, t.y);
            r[2] = mk(t.z, t.w);
        } else {
            const float4 t = __ldg(b4 + 3);
            const float2 u = __ldg(b + 8);
            r[0] = mk(t.x, t.y);
            r[1] = mk(t.z, t.w);
            r[2] = mk(u.x, u.y);
        }
        return;
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        float2 t = __ldg(b + (dag ? 3 * k + a : 3 * a + k));
        r[k] = dag ? mk(t.x, -t.y) : mk(t.x, t.y);
    }
}

// (1 + SG gamma_mu) psi has upper half h = psi_u + SG A psi_l (two colour
// vectors h0, h1) and lower half SG A^+ h.  project forms h; mac_row adds
// row a of V h (V = U or U^+, one link row u) to the upper spins and,
// through A^+, to the lower spins.  The time-boundary phase is carried by
// the packed links.
template <int MU, int SG, typename R>
__device__ __forceinline__ void project(const cpx<R>* psi, cpx<R>* h) {
    cpx<R> a0[3], a1[3];
    apply_A<MU>(psi + 6, psi + 9, a0, a1);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        h[c] = SG > 0 ? psi[c] + a0[c] : psi[c] - a0[c];
        h[3 + c] = SG > 0 ? psi[3 + c] + a1[c] : psi[3 + c] - a1[c];
    }
}

template <int MU, int SG, typename R>
__device__ __forceinline__ void mac_row(const cpx<R>* u, int a, const cpx<R>* h, cpx<R>* acc) {
    const cpx<R> w0 = cmul(u[0], h[0]) + cmul(u[1], h[1]) + cmul(u[2], h[2]);
    const cpx<R> w1 = cmul(u[0], h[3]) + cmul(u[1], h[4]) + cmul(u[2], h[5]);
    acc[a] = acc[a] + w0;
    acc[3 + a] = acc[3 + a] + w1;
    cpx<R> l0, l1;
    if (MU == 0) { l0 = itimes(w1); l1 = itimes(w0); }
    else if (MU == 1) { l0 = w1; l1 = mk(-w0.re, -w0.im); }
    else if (MU == 2) { l0 = itimes(w0); l1 = mitimes(w1); }
    else { l0 = w0; l1 = w1; }
    acc[6 + a] = SG > 0 ? acc[6 + a] + l0 : acc[6 + a] - l0;
    acc[9 + a] = SG > 0 ? acc[9 + a] + l1 : acc[9 + a] - l1;
}

// One direction pair for SPT slices s[0..SPT) of site j: the neighbour index
// and every link row are loaded once and used for all SPT slices.
template <int P, int DAG, int MU, int SPT>
__device__ __forceinline__ void hop_mu(const Geom& g, int par, int j, const int* ent, const int* sv, int Ls,
                                       long long n5, const void* in, const void* gauge,
                                       cpx<typename Field<P>::R> (*acc)[12]) {
    typedef typename Field<P>::R R;
#pragma unroll
    for (int dirn = 0; dirn < 2; dirn++) {
        const int e = EOFA_HOP_PREFETCH ? ent[2 * MU + dirn]
                                        : __ldg((par ? g.nbr[1] : g.nbr[0]) + (2 * MU + dirn) * g.Vh + j);
        const int jn = e;
        cpx<R> h[SPT][6];
#pragma unroll
        for (int k = 0; k < SPT; k++) {
            cpx<R> psi[12];
            if constexpr (P == P16) {
                // project the stored unit-scale values, then scale the 6 components of h
                const float sc = Field<P16>::load_unscaled(in, jn, sv[k], Ls, n5, psi);
                if (dirn == 0) project<MU, DAG ? 1 : -1>(psi, h[k]);
                else project<MU, DAG ? -1 : 1>(psi, h[k]);
#pragma unroll
                for (int c = 0; c < 6; c++) h[k][c] = sc * h[k][c];
            } else {
                Field<P>::load(in, jn, sv[k], Ls, n5, psi);
                if (dirn == 0) project<MU, DAG ? 1 : -1>(psi, h[k]);
                else project<MU, DAG ? -1 : 1>(psi, h[k]);
            }
        }
        const long long lidx = dirn == 0 ? (long long)((par * 4 + MU) * g.Vh + j)
                                         : (long long)(((1 - par) * 4 + MU) * g.Vh + jn);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            cpx<R> u[3];
            link_row<R>(gauge, lidx, a, dirn == 1, u);
#pragma unroll
            for (int k = 0; k < SPT; k++) {
                if (dirn == 0) mac_row<MU, DAG ? 1 : -1>(u, a, h[k], acc[k]);
                else mac_row<MU, DAG ? -1 : 1>(u, a, h[k], acc[k]);
            }
        }
    }
}

// ---------------------------------------------------------------- 5D-local column ops
//
// Column x[0..Ls) of one (site, component); B = p + q L_dir with L_dir the
// down-shift (dir 0) or up-shift (dir 1), corner -mass.  The inverse uses
// L^Ls = -mass: u_0 = [x_0 - mass sum_{j>=1} (-r)^(Ls-j) x_j] / (p (1 + mass (-r)^Ls)),
// u_s = (x_s - q u_{s-1}) / p (mirrored for dir 1).

// runtime-Ls versions working in shared memory (fallback for uncommon Ls)
template <typename R>
__device__ void sm_inv(cpx<R>* x, int Ls, R p, R q, int dir, R mass) {
    const R mr = -q / p;
    R pw = 1;
    for (int k = 0; k < Ls; k++) pw *= mr;
    const R invN = R(1) / (p * (R(1) + mass * pw));
    const R invp = R(1) / p;
    cpx<R> acc = mk(R(0), R(0));
    if (dir == 0) {
        for (int s = 1; s < Ls; s++) acc = mr * acc + x[s];
        acc = mr * acc;
        x[0] = invN * (x[0] - mass * acc);
        for (int s = 1; s < Ls; s++) x[s] = invp * (x[s] - q * x[s - 1]);
    } else {
        for (int s = Ls - 2; s >= 0; s--) acc = mr * acc + x[s];
        acc = mr * acc;
        x[Ls - 1] = invN * (x[Ls - 1] - mass * acc);
        for (int s = Ls - 2; s >= 0; s--) x[s] = invp * (x[s] - q * x[s + 1]);
    }
}

template <typename R>
__device__ void sm_fwd(cpx<R>* x, int Ls, R p, R q, int dir, R mass) {
    if (dir == 0) {
        const cpx<R> last = x[Ls - 1];
        for (int s = Ls - 1; s >= 1; s--) x[s] = p * x[s] + q * x[s - 1];
        x[0] = p * x[0] - (q * mass) * last;
    } else {
        const cpx<R> first = x[0];
        for (int s = 0; s < Ls - 1; s++) x[s] = p * x[s] + q * x[s + 1];
        x[Ls - 1] = p * x[Ls - 1] - (q * mass) * first;
    }
}

// per-chirality parameters of an Op5 without dynamic indexing of the struct
template <typename R>
struct Half {
    int inv, fwd, dir1, dir2;
    R p1, q1, p2, q2, sigma, mass, mr, invp, invN;
    const R *w, *v;  // rank-one vectors, staged in shared memory
};

// The rank-one vectors w, v of both chiralities, converted to R once per
// block into shared memory wv[4 * Ls] (layout [h][w, v][s]); callers
// synchronise the block before the first column_op.
template <typename R>
__device__ __forceinline__ void stage_wv(const Op5& op, int Ls, R* wv) {
    for (int i = threadIdx.x; i < 4 * Ls; i += blockDim.x) {
        const int h = i / (2 * Ls), which = (i / Ls) & 1, s = i % Ls;
        const double* src = which ? (h ? op.v[1] : op.v[0]) : (h ? op.w[1] : op.w[0]);
        const double sg = h ? op.sigma[1] : op.sigma[0];
        wv[i] = (sg != 0.0 && src) ? (R)src[s] : R(0);
    }
}

template <typename R>
__device__ __forceinline__ Half<R> half_of(const Op5& op, int h, const R* wv, int Ls) {
    Half<R> H;
    H.inv = h ? op.inv[1] : op.inv[0];
    H.fwd = h ? op.fwd[1] : op.fwd[0];
    H.dir1 = h ? op.dir1[1] : op.dir1[0];
    H.dir2 = h ? op.dir2[1] : op.dir2[0];
    H.p1 = (R)(h ? op.p1[1] : op.p1[0]);
    H.q1 = (R)(h ? op.q1[1] : op.q1[0]);
    H.p2 = (R)(h ? op.p2[1] : op.p2[0]);
    H.q2 = (R)(h ? op.q2[1] : op.q2[0]);
    H.sigma = (R)(h ? op.sigma[1] : op.sigma[0]);
    H.mass = (R)op.mass;
    H.mr = (R)(h ? op.mr[1] : op.mr[0]);
    H.invp = (R)(h ? op.invp[1] : op.invp[0]);
    H.invN = (R)(h ? op.invN[1] : op.invN[0]);
    H.w = wv + (2 * h) * Ls;
    H.v = wv + (2 * h + 1) * Ls;
    return H;
}

// Streaming form of B for a compile-time Ls when the inverse and the matrix
// use the same shift direction (every block built in ops.cu): one pass for
// the Horner sum of the corner term, one pass that runs the inverse
// recurrence u_s = mr u_{s-1} + x_s / p (mr = -q / p; x_s / p does not
// wait for u, so one multiply-add per step is on the dependent chain) and
// emits (p2 + q2 L) u on the fly; two live values per step instead of the
// whole column.
template <typename R>
struct Vec2;
template <>
struct Vec2<float> {
    typedef float2 T;
};
template <>
struct Vec2<double> {
    typedef double2 T;
};

template <typename R>
__device__ __forceinline__ cpx<R> lds(const cpx<R>* p) {
    typename Vec2<R>::T v = *reinterpret_cast<const typename Vec2<R>::T*>(p);
    return mk(v.x, v.y);
}

template <typename R>
__device__ __forceinline__ void sts(cpx<R>* p, cpx<R> a) {
    typename Vec2<R>::T v;
    v.x = a.re;
    v.y = a.im;
    *reinterpret_cast<typename Vec2<R>::T*>(p) = v;
}

template <typename R, int LS, bool R1>
__device__ __forceinline__ void col_stream(const Half<R>& H, cpx<R>* col) {
    const R mass = H.mass, mr = H.mr, invp = H.invp, invN = H.invN;
    const R p2 = H.fwd ? H.p2 : R(1), q2 = H.fwd ? H.q2 : R(0);
    cpx<R> acc = mk(R(0), R(0)), d = mk(R(0), R(0));
    if (H.dir1 == 0) {
#pragma unroll
        for (int s = 1; s < LS; s++) acc = mr * acc + lds(col + s);
        acc = mr * acc;
        const cpx<R> u0 = invN * (lds(col) - mass * acc);
        cpx<R> u = u0;
        if (R1) d = H.v[0] * u0;
#pragma unroll
        for (int s = 1; s < LS; s++) {
            const cpx<R> un = mr * u + invp * lds(col + s);
            if (R1) d = d + H.v[s] * un;
            sts(col + s, p2 * un + q2 * u);
            u = un;
        }
        sts(col, p2 * u0 - (q2 * mass) * u);
    } else {
#pragma unroll
        for (int s = LS - 2; s >= 0; s--) acc = mr * acc + lds(col + s);
        acc = mr * acc;
        const cpx<R> uL = invN * (lds(col + LS - 1) - mass * acc);
        cpx<R> u = uL;
        if (R1) d = H.v[LS - 1] * uL;
#pragma unroll
        for (int s = LS - 2; s >= 0; s--) {
            const cpx<R> un = mr * u + invp * lds(col + s);
            if (R1) d = d + H.v[s] * un;
            sts(col + s, p2 * un + q2 * u);
            u = un;
        }
        sts(col + LS - 1, p2 * uL - (q2 * mass) * u);
    }
    if (R1) {
        // rank-one term: out += sigma w (v . u), u the inverse's result
        const cpx<R> sd = H.sigma * d;
#pragma unroll
        for (int s = 0; s < LS; s++) sts(col + s, lds(col + s) + H.w[s] * sd);
    }
}

// FP32 form of col_stream on packed pairs: every step multiplies a complex
// number by real coefficients, so (re, im) travel as one 64-bit register and
// each complex multiply-add is one f32x2 instruction.
template <int LS, bool R1>
__device__ __forceinline__ void col_stream_f2(const Half<float>& H, cpx<float>* col) {
    const f2p MR = splat2(H.mr), NM = splat2(-H.mass), INVN = splat2(H.invN), INVP = splat2(H.invp);
    const float p2 = H.fwd ? H.p2 : 1.f, q2 = H.fwd ? H.q2 : 0.f;
    const f2p P2 = splat2(p2), Q2 = splat2(q2), Q2M = splat2(-q2 * H.mass);
    f2p acc = 0ull, d = 0ull;
    if (H.dir1 == 0) {
#pragma unroll
        for (int s = 1; s < LS; s++) acc = fma2(MR, acc, ld2(col + s));
        acc = mul2(MR, acc);
        const f2p u0 = mul2(INVN, fma2(NM, acc, ld2(col)));
        f2p u = u0;
        if (R1) d = mul2(splat2(H.v[0]), u0);
#pragma unroll
        for (int s = 1; s < LS; s++) {
            const f2p un = fma2(MR, u, mul2(INVP, ld2(col + s)));
            if (R1) d = fma2(splat2(H.v[s]), un, d);
            st2(col + s, fma2(P2, un, mul2(Q2, u)));
            u = un;
        }
        st2(col, fma2(P2, u0, mul2(Q2M, u)));
    } else {
#pragma unroll
        for (int s = LS - 2; s >= 0; s--) acc = fma2(MR, acc, ld2(col + s));
        acc = mul2(MR, acc);
        const f2p uL = mul2(INVN, fma2(NM, acc, ld2(col + LS - 1)));
        f2p u = uL;
        if (R1) d = mul2(splat2(H.v[LS - 1]), uL);
#pragma unroll
        for (int s = LS - 2; s >= 0; s--) {
            const f2p un = fma2(MR, u, mul2(INVP, ld2(col + s)));
            if (R1) d = fma2(splat2(H.v[s]), un, d);
            st2(col + s, fma2(P2, un, mul2(Q2, u)));
            u = un;
        }
        st2(col + LS - 1, fma2(P2, uL, mul2(Q2M, u)));
    }
    if (R1) {
        const f2p sd = mul2(splat2(H.sigma), d);
#pragma unroll
        for (int s = 0; s < LS; s++) st2(col + s, fma2(splat2(H.w[s]), sd, ld2(col + s)));
    }
}

// apply B to the column at col (shared memory, stride 1, length Ls)
template <typename R, int LS>
__device__ __forceinline__ void column_op(const Op5& op, int c, cpx<R>* col, int Ls, const R* wv) {
    const Half<R> H = half_of<R>(op, c < 6 ? 0 : 1, wv, Ls);
    if (LS > 0 && H.inv && (!H.fwd || H.dir2 == H.dir1)) {
        if constexpr (EOFA_PACKED_F32 && std::is_same<R, float>::value) {
            if (H.sigma == R(0)) col_stream_f2<(LS > 0 ? LS : 1), false>(H, col);
            else col_stream_f2<(LS > 0 ? LS : 1), true>(H, col);
        } else {
            if (H.sigma == R(0)) col_stream<R, (LS > 0 ? LS : 1), false>(H, col);
            else col_stream<R, (LS > 0 ? LS : 1), true>(H, col);
        }
        return;
    }
    if (H.inv) sm_inv<R>(col, Ls, H.p1, H.q1, H.dir1, H.mass);
    cpx<R> d = mk(R(0), R(0));
    if (H.sigma != R(0))
        for (int s = 0; s < Ls; s++) d = d + H.v[s] * col[s];
    if (H.fwd) sm_fwd<R>(col, Ls, H.p2, H.q2, H.dir2, H.mass);
    if (H.sigma != R(0)) {
        const cpx<R> sd = H.sigma * d;
        for (int s = 0; s < Ls; s++) col[s] = col[s] + H.w[s] * sd;
    }
}

// the column phase of a tile: one thread per (site, component) column
template <typename R, int LS>
__device__ __forceinline__ void columns(const Op5& op, cpx<R>* sm, int ncols, int LsP, int Ls, const R* wv) {
    for (int idx = threadIdx.x; idx < ncols; idx += blockDim.x) column_op<R, LS>(op, idx % 12, sm + idx * LsP, Ls, wv);
}

__device__ __forceinline__ bool op_is_identity(const Op5& op) {
    return !op.inv[0] && !op.inv[1] && !op.fwd[0] && !op.fwd[1] && op.sigma[0] == 0.0 && op.sigma[1] == 0.0;
}

// ---------------------------------------------------------------- reductions

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum v over the block, then over the grid (last block, fixed order) into red[slot].
__device__ __noinline__ void grid_sum(double v, double* red, int slot) {
    __shared__ double ws[32];
    __shared__ bool last;
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    if (l == 0) ws[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int k = 0; k < nw; k++) t += ws[k];
        red[RED_PART + blockIdx.x] = t;
        __threadfence();
        unsigned prev = atomicAdd((unsigned*)(red + RED_TICKET), 1u);
        last = prev == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        double t = 0;
        for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) t += ((volatile double*)red)[RED_PART + k];
        t = warp_sum(t);
        __syncthreads();
        if (l == 0) ws[w] = t;
        __syncthreads();
        if (threadIdx.x == 0) {
            double f = 0;
            for (int k = 0; k < nw; k++) f += ws[k];
            red[slot] = f;
            *(unsigned*)(red + RED_TICKET) = 0u;
        }
    }
}

// Two sums at once: v1 -> red[slot1] (partials at RED_PART), v2 -> red[slot2]
// (partials at RED_PART2); one ticket, fixed-order final sums.
__device__ __noinline__ void grid_sum2(double v1, double v2, double* red, int slot1, int slot2) {
    __shared__ double ws[2][32];
    __shared__ bool last;
    v1 = warp_sum(v1);
    v2 = warp_sum(v2);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    if (l == 0) {
        ws[0][w] = v1;
        ws[1][w] = v2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0, t2 = 0;
        for (int k = 0; k < nw; k++) {
            t1 += ws[0][k];
            t2 += ws[1][k];
        }
        red[RED_PART + blockIdx.x] = t1;
        red[RED_PART2 + blockIdx.x] = t2;
        __threadfence();
        unsigned prev = atomicAdd((unsigned*)(red + RED_TICKET), 1u);
        last = prev == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        double t1 = 0, t2 = 0;
        for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
            t1 += ((volatile double*)red)[RED_PART + k];
            t2 += ((volatile double*)red)[RED_PART2 + k];
        }
        t1 = warp_sum(t1);
        t2 = warp_sum(t2);
        __syncthreads();
        if (l == 0) {
            ws[0][w] = t1;
            ws[1][w] = t2;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double f1 = 0, f2 = 0;
            for (int k = 0; k < nw; k++) {
                f1 += ws[0][k];
                f2 += ws[1][k];
            }
            red[slot1] = f1;
            red[slot2] = f2;
            *(unsigned*)(red + RED_TICKET) = 0u;
        }
    }
}

template <typename R>
__device__ __forceinline__ double site_norm2(const cpx<R>* v) {
    R a = 0;
#pragma unroll
    for (int c = 0; c < 12; c++) a += v[c].re * v[c].re + v[c].im * v[c].im;
    return (double)a;
}

__device__ __forceinline__ double cg_alpha(const double* sc, int it) {
    const double gam = sc[SC_GAMMA + (it & 1)], del = sc[SC_DELTA];
    return (del > 0.0 && gam > 0.0) ? gam / del : 0.0;
}

__device__ __forceinline__ double cg_beta(const double* sc, int it) {
    const double gold = sc[SC_GAMMA + (it & 1)], gnew = sc[SC_GAMMA + ((it + 1) & 1)];
    return gold > 0.0 ? gnew / gold : 0.0;
}

// ---------------------------------------------------------------- fused dslash

// Extra epilogue of the CG launches with more than one output (MODE 1, 2).
struct Epi {
    Op5 op2;           // MODE 1: block of the second output
    void* out2;        // MODE 1: out2 = B2 out;  MODE 2: r (may be null), updated in place (r -= alpha y);
                       // MODE 3: x, updated in place (x += alpha aux)
    const void* aux;   // MODE 3: p
    void* out3;        // MODE 3: r, updated in place (r -= alpha aux2)
    const void* aux2;  // MODE 3: q
    int it, slot2;     // MODE 2, 3: iteration of the CG scalars and the slot of |r|^2
};

// HASOP = false: B is the identity (plain hop), compiled separately so that
// the register budget of the hop is not set by the 5D-local recurrences.
// MODE 0: out = value.  MODE 1: also out2 = B2 out (a second 5D-local pass
// through shared memory).  MODE 2: out is updated in place,
// out <- out - alpha(red, it) value, and so is out2 <- out2 - alpha y, with
// |out|^2 -> red[slot] and |out2|^2 -> red[ep.slot2] (out2 may be null).
// MODE 3: out = value, and the CG updates x <- x + alpha(red, it) p and
// (when r = out3 is not null) r <- r - alpha q at the same (j, s),
// |r|^2 -> red[ep.slot2] (x = out2 in the solution's precision, p = aux,
// q = aux2): elementwise updates ride in this latency-bound launch instead
// of streaming kernels.
// SPT slices per thread: thread (site, sh) handles s = sh + k Ls/SPT,
// k < SPT, so neighbour indices and link rows are loaded once for SPT output
// sites (Ls/SPT threads per site; SPT = 2 needs an even Ls).
// the two-pass epilogue of MODE 1 gets up to 128 registers (its 80-register
// build spilled 224 bytes)
#ifndef EOFA_MODE1_MINB
#define EOFA_MODE1_MINB 2
#endif
// (The FP64 builds spill at this cap but are bound by the FP64 FMA rate:
// 244 registers without spills measured 5% slower at 24^3x64.)
template <int P, int DAG, int LS, bool HASOP, int SPT, int MODE = 0>
__global__ void __launch_bounds__(256, SPT == 2 ? 2 : (MODE == 1 ? EOFA_MODE1_MINB : (HASOP ? EOFA_DSLASH_MINB : EOFA_HOP_MINB))) dslash_kernel(
    Geom g, int par, const void* __restrict__ in, void* out, const void* __restrict__ gauge, Op5 op, const void* y,
    double a_out, double b_in, double* red, int slot, int NS, Epi ep) {
    typedef typename Field<P>::R R;
    extern __shared__ __align__(128) unsigned char smraw[];
    cpx<R>* sm = reinterpret_cast<cpx<R>*>(smraw);
    const int Ls = LS > 0 ? LS : g.Ls;
    const int LsP = Ls + 1;
    const int Lt = Ls / SPT;  // threads per site
    __shared__ R wv_s[HASOP ? 4 * EOFA_MAX_LS : 1];
    __shared__ R wv2_s[MODE == 1 ? 4 * EOFA_MAX_LS : 1];
    if (HASOP) stage_wv<R>(op, Ls, wv_s);
    if (MODE == 1) stage_wv<R>(ep.op2, Ls, wv2_s);
    if (HASOP || MODE == 1) __syncthreads();
    const R cz = MODE == 2 ? (R)(-cg_alpha(red, ep.it)) : R(0);
    // MODE 3: x is stored in FP32 when the field is FP16, else in the field's precision
    constexpr int PX = P == P16 ? P32 : P;
    typedef typename Field<PX>::R RX;
    const RX ax = MODE == 3 ? (RX)cg_alpha(red, ep.it) : RX(0);
    const long long n5 = (long long)g.Vh * Ls;
    const int ls = threadIdx.x / Lt, sh = threadIdx.x - ls * Lt;
    int sv[SPT];
#pragma unroll
    for (int k = 0; k < SPT; k++) sv[k] = sh + k * Lt;
    const bool active_thread = ls < NS;
    const int ntiles = (g.Vh + NS - 1) / NS;
    const R scale = (R)(-0.5 * a_out);
    double nacc = 0.0, nacc2 = 0.0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int j = tile * NS + ls;
        const bool site_ok = active_thread && j < g.Vh;
        cpx<R> acc[SPT][12];
#pragma unroll
        for (int k = 0; k < SPT; k++)
#pragma unroll
            for (int c = 0; c < 12; c++) acc[k][c] = mk(R(0), R(0));
        if (site_ok) {
            // the eight neighbour entries are loaded up front, so that no
            // spinor load waits behind the load of its own index
            const int* nb = par ? g.nbr[1] : g.nbr[0];
            int ent[8];
            if (EOFA_HOP_PREFETCH) {
#pragma unroll
                for (int d = 0; d < 8; d++) ent[d] = __ldg(nb + d * g.Vh + j);
            }
            hop_mu<P, DAG, 0, SPT>(g, par, j, ent, sv, Ls, n5, in, gauge, acc);
            hop_mu<P, DAG, 1, SPT>(g, par, j, ent, sv, Ls, n5, in, gauge, acc);
            hop_mu<P, DAG, 2, SPT>(g, par, j, ent, sv, Ls, n5, in, gauge, acc);
            hop_mu<P, DAG, 3, SPT>(g, par, j, ent, sv, Ls, n5, in, gauge, acc);
        }
        if (HASOP) {
            if (site_ok) {
#pragma unroll
                for (int k = 0; k < SPT; k++)
#pragma unroll
                    for (int c = 0; c < 12; c++) sts(sm + (ls * 12 + c) * LsP + sv[k], acc[k][c]);
            }
            __syncthreads();
            const int nsites = min(NS, g.Vh - tile * NS);
            columns<R, LS>(op, sm, nsites * 12, LsP, Ls, wv_s);
            __syncthreads();
            if (site_ok) {
#pragma unroll
                for (int k = 0; k < SPT; k++)
#pragma unroll
                    for (int c = 0; c < 12; c++) acc[k][c] = lds(sm + (ls * 12 + c) * LsP + sv[k]);
            }
        }
        if (site_ok) {
#pragma unroll
            for (int k = 0; k < SPT; k++) {
#pragma unroll
                for (int c = 0; c < 12; c++) acc[k][c] = scale * acc[k][c];
                if (y != nullptr) {
                    cpx<R> yv[12];
                    if (EOFA_STREAM_HINTS) Field<P>::load_stream(y, j, sv[k], Ls, n5, yv);
                    else Field<P>::load(y, j, sv[k], Ls, n5, yv);
                    const R bb = (R)b_in;
#pragma unroll
                    for (int c = 0; c < 12; c++) acc[k][c] = acc[k][c] + bb * yv[c];
                    if (MODE == 2 && ep.out2 != nullptr) {
                        // r <- r - alpha y
                        cpx<R> rv[12];
                        Field<P>::load_stream(ep.out2, j, sv[k], Ls, n5, rv);
#pragma unroll
                        for (int c = 0; c < 12; c++) rv[c] = rv[c] + cz * yv[c];
                        Field<P>::store_stream(ep.out2, j, sv[k], Ls, n5, rv);
                        nacc2 += site_norm2<R>(rv);
                    }
                }
                if (MODE == 2) {
                    cpx<R> zv[12];
                    Field<P>::load_stream(out, j, sv[k], Ls, n5, zv);
#pragma unroll
                    for (int c = 0; c < 12; c++) acc[k][c] = zv[c] + cz * acc[k][c];
                }
                if (EOFA_STREAM_HINTS) Field<P>::store_stream(out, j, sv[k], Ls, n5, acc[k]);
                else Field<P>::store(out, j, sv[k], Ls, n5, acc[k]);
                if (red && slot >= 0) nacc += site_norm2<R>(acc[k]);
                if (MODE == 3) {
                    // x += alpha p at this (j, s); x and p belong to the other checkerboard,
                    // the update is elementwise
                    cpx<R> pv[12];
                    cpx<RX> xv[12];
                    Field<P>::load_stream(ep.aux, j, sv[k], Ls, n5, pv);
                    Field<PX>::load_stream(ep.out2, j, sv[k], Ls, n5, xv);
#pragma unroll
                    for (int c = 0; c < 12; c++)
                        xv[c] = mk((RX)(xv[c].re + ax * (RX)pv[c].re), (RX)(xv[c].im + ax * (RX)pv[c].im));
                    Field<PX>::store_stream(ep.out2, j, sv[k], Ls, n5, xv);
                    if (ep.out3 != nullptr) {
                        // r -= alpha q
                        cpx<R> qv[12], rv[12];
                        Field<P>::load_stream(ep.aux2, j, sv[k], Ls, n5, qv);
                        Field<P>::load_stream(ep.out3, j, sv[k], Ls, n5, rv);
#pragma unroll
                        for (int c = 0; c < 12; c++) rv[c] = rv[c] - (R)ax * qv[c];
                        Field<P>::store_stream(ep.out3, j, sv[k], Ls, n5, rv);
                        nacc2 += site_norm2<R>(rv);
                    }
                }
            }
        }
        if (MODE == 1) {
            // out2 = B2 out: the block's outputs go through shared memory once more
            __syncthreads();
            if (site_ok) {
#pragma unroll
                for (int c = 0; c < 12; c++) sts(sm + (ls * 12 + c) * LsP + sv[0], acc[0][c]);
            }
            __syncthreads();
            const int nsites = min(NS, g.Vh - tile * NS);
            columns<R, LS>(ep.op2, sm, nsites * 12, LsP, Ls, wv2_s);
            __syncthreads();
            if (site_ok) {
#pragma unroll
                for (int c = 0; c < 12; c++) acc[0][c] = lds(sm + (ls * 12 + c) * LsP + sv[0]);
                Field<P>::store_stream(ep.out2, j, sv[0], Ls, n5, acc[0]);
            }
        }
        if (HASOP) __syncthreads();
    }
    if (MODE == 3) {
        if (ep.out3 != nullptr) grid_sum(nacc2, red, ep.slot2);
    } else if (red && slot >= 0) {
        if (MODE == 2 && ep.out2 != nullptr) grid_sum2(nacc, nacc2, red, slot, ep.slot2);
        else grid_sum(nacc, red, slot);
    }
}

// x' = x + c z (c = -alpha from the device scalars when use_alpha, else c0);
// xw <- x' (if xw), |x'|^2 -> red[slot] (if red), out = a B x' (if out).
#ifndef EOFA_LOCAL5_MINB
#define EOFA_LOCAL5_MINB 2
#endif
// Up to 128 registers: at 80 the FP32 Ls = 24 build spilled 256 bytes and
// streamed 4.9 TB/s at 24^3x64 instead of 6.4.
template <int P, int LS>
__global__ void __launch_bounds__(256, EOFA_LOCAL5_MINB) local5_kernel(Geom g, Op5 op, const void* x, const void* z, double c0,
                                                     const double* sc, int it, int use_alpha, void* xw, void* out,
                                                     double a_out, double* red, int slot, int NS) {
    typedef typename Field<P>::R R;
    extern __shared__ __align__(128) unsigned char smraw[];
    cpx<R>* sm = reinterpret_cast<cpx<R>*>(smraw);
    const int Ls = LS > 0 ? LS : g.Ls;
    const int LsP = Ls + 1;
    const long long n5 = (long long)g.Vh * Ls;
    const int ls = threadIdx.x / Ls, s = threadIdx.x - ls * Ls;
    const bool active_thread = ls < NS;
    const bool ident = op_is_identity(op);
    const int ntiles = (g.Vh + NS - 1) / NS;
    const R c = (R)(use_alpha ? -cg_alpha(sc, it) : c0);
    __shared__ R wv_s[4 * EOFA_MAX_LS];
    if (out && !ident) {
        stage_wv<R>(op, Ls, wv_s);
        __syncthreads();
    }
    double nacc = 0.0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int j = tile * NS + ls;
        const bool site_ok = active_thread && j < g.Vh;
        cpx<R> v[12];
        if (site_ok) {
            if (EOFA_STREAM_HINTS) Field<P>::load_stream(x, j, s, Ls, n5, v);
            else Field<P>::load(x, j, s, Ls, n5, v);
            if (z != nullptr) {
                cpx<R> zv[12];
                if (EOFA_STREAM_HINTS) Field<P>::load_stream(z, j, s, Ls, n5, zv);
                else Field<P>::load(z, j, s, Ls, n5, zv);
#pragma unroll
                for (int k = 0; k < 12; k++) v[k] = v[k] + c * zv[k];
            }
            if (xw) {
                if (EOFA_STREAM_HINTS) Field<P>::store_stream(xw, j, s, Ls, n5, v);
                else Field<P>::store(xw, j, s, Ls, n5, v);
            }
            if (red) nacc += site_norm2<R>(v);
        }
        if (out) {
            if (!ident) {
                if (site_ok) {
#pragma unroll
                    for (int k = 0; k < 12; k++) sts(sm + (ls * 12 + k) * LsP + s, v[k]);
                }
                __syncthreads();
                const int nsites = min(NS, g.Vh - tile * NS);
                for (int idx = threadIdx.x; idx < nsites * 12; idx += blockDim.x)
                    column_op<R, LS>(op, idx % 12, sm + idx * LsP, Ls, wv_s);
                __syncthreads();
                if (site_ok) {
#pragma unroll
                    for (int k = 0; k < 12; k++) v[k] = lds(sm + (ls * 12 + k) * LsP + s);
                }
            }
            if (site_ok) {
#pragma unroll
                for (int k = 0; k < 12; k++) v[k] = (R)a_out * v[k];
                if (EOFA_STREAM_HINTS) Field<P>::store_stream(out, j, s, Ls, n5, v);
                else Field<P>::store(out, j, s, Ls, n5, v);
            }
            if (!ident) __syncthreads();
        }
    }
    if (red) grid_sum(nacc, red, slot);
}

// x += alpha p (x in PX; skipped when x is null), p = s + beta p
template <int P, int PX>
__global__ void __launch_bounds__(256) xp_update_kernel(Geom g, const double* sc, int it, void* x, void* p,
                                                        const void* s) {
    typedef typename Field<P>::R R;
    typedef typename Field<PX>::R RX;
    const long long n5 = (long long)g.Vh * g.Ls;
    const R alpha = (R)cg_alpha(sc, it), beta = (R)cg_beta(sc, it);
    const unsigned n5u = (unsigned)n5, Lsu = (unsigned)g.Ls;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n5u; t += gridDim.x * blockDim.x) {
        const int j = (int)(t / Lsu);
        const int ss = (int)(t - (unsigned)j * Lsu);
        cpx<R> pv[12], sv[12];
        Field<P>::load(p, j, ss, g.Ls, n5, pv);
        Field<P>::load(s, j, ss, g.Ls, n5, sv);
        if (x != nullptr) {
            cpx<RX> xv[12];
            Field<PX>::load(x, j, ss, g.Ls, n5, xv);
#pragma unroll
            for (int k = 0; k < 12; k++)
                xv[k] = mk((RX)(xv[k].re + (RX)alpha * (RX)pv[k].re), (RX)(xv[k].im + (RX)alpha * (RX)pv[k].im));
            Field<PX>::store(x, j, ss, g.Ls, n5, xv);
        }
#pragma unroll
        for (int k = 0; k < 12; k++) pv[k] = sv[k] + beta * pv[k];
        Field<P>::store(p, j, ss, g.Ls, n5, pv);
    }
}

// ---------------------------------------------------------------- launch helpers

// sites per tile: NS * Ls a multiple of 32 where possible, 96..256 threads,
// at most 32 KB of shared memory
}  // namespace
}  // namespace dsl

#include "dslash_bulk.cuh"
#include "dslash_pipe.cuh"

namespace dsl {
namespace {

inline int pick_ns(int Ls, size_t elem) {
    int gg = 1;
    for (int k = 32; k >= 1; k >>= 1)
        if (Ls % k == 0) { gg = k; break; }
    int ns = 32 / gg;
    while (ns * Ls < 96) ns *= 2;
    while (ns * Ls > 256 && ns > 1) ns /= 2;
    while ((size_t)ns * 12 * (Ls + 1) * elem > 32768 && ns > 1) ns /= 2;
    if (ns < 1) ns = 1;
    return ns;
}

template <typename K>
unsigned grid_size(K kernel, int threads, size_t smem, int ntiles, int sms) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (per_sm < 1) per_sm = 1;
    long long cap = (long long)per_sm * sms;
    if (cap > RED_MAX_BLOCKS) cap = RED_MAX_BLOCKS;
    return (unsigned)(ntiles < cap ? (ntiles > 0 ? ntiles : 1) : cap);
}

// Autotuner: the sites per tile (NS) of the fused dslash are timed once per
// context and kernel variant, with CUDA events on the launching stream, over
// the heuristic choice and its halving / doubling.  The kernel is
// idempotent (it only writes out and the reduction scratch), so the trial
// launches are harmless.  Small lattices, and launches during stream capture,
// use the heuristic.
template <typename K>
void launch_with(K k, const eofa_ctx* ctx, const Geom& g, int NS, int spt, size_t elem, bool hasop, int par,
                 const void* in, void* out, const void* gauge, const Op5& op, const void* y, double a_out, double b_in,
                 double* red, int slot, cudaStream_t st) {
    const int threads = (NS * (g.Ls / spt) + 31) / 32 * 32;
    const size_t smem = hasop ? (size_t)NS * 12 * (g.Ls + 1) * elem : 0;
    const int ntiles = (g.Vh + NS - 1) / NS;
    if (smem > 40 * 1024) EOFA_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    unsigned grid = grid_size(k, threads, smem, ntiles, ctx->sms);
    Epi ep;
    ep.op2 = op;
    ep.out2 = nullptr;
    ep.aux = nullptr;
    ep.out3 = nullptr;
    ep.aux2 = nullptr;
    ep.it = 0;
    ep.slot2 = 0;
    k<<<grid, threads, smem, st>>>(g, par, in, out, gauge, op, y, a_out, b_in, red, slot, NS, ep);
}

// direct kernel with a multi-output epilogue (MODE 1, 2) at NS sites per tile
template <typename K>
void launch_epi(K k, const eofa_ctx* ctx, const Geom& g, int NS, size_t elem, bool hasop, int par, const void* in,
                void* out, const void* gauge, const Op5& op, const void* y, double a_out, double b_in, double* red,
                int slot, const Epi& ep, cudaStream_t st) {
    const int threads = (NS * g.Ls + 31) / 32 * 32;
    const size_t smem = hasop ? (size_t)NS * 12 * (g.Ls + 1) * elem : 0;
    const int ntiles = (g.Vh + NS - 1) / NS;
    if (smem > 40 * 1024) EOFA_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    unsigned grid = grid_size(k, threads, smem, ntiles, ctx->sms);
    k<<<grid, threads, smem, st>>>(g, par, in, out, gauge, op, y, a_out, b_in, red, slot, NS, ep);
}

// Staged (bulk-copy) configurations are encoded as CFG_BULK | D << 8 | NS,
// pipelined (cp.async) ones as CFG_PIPE | PIPE << 8 | NS, direct ones as
// NS * 4 + SPT.
#define CFG_BULK (1 << 20)
#define CFG_PIPE (1 << 21)

// the EOFA_DSLASH_CONFIG spelling of a configuration
inline std::string cfg_str(int cfg) {
    if (cfg & CFG_BULK) return std::to_string(cfg & 0xff) + ",1," + std::to_string((cfg >> 8) & 0xf);
    if (cfg & CFG_PIPE) return std::to_string(cfg & 0xff) + ",1,-" + std::to_string((cfg >> 8) & 0xf);
    return std::to_string(cfg / 4) + "," + std::to_string(cfg % 4);
}

template <int P>
bool bulk_fits(const Geom& g, int NS, int D, bool hasop, const void* in, const void* y) {
    typedef typename Field<P>::R R;
    if (NS < 1 || NS > 32 || D < 2 || D > 8) return false;
    if ((NS * g.Ls + 31) / 32 * 32 + 32 > BULK_MAX_THREADS) return false;
    if (P == P16 && g.Ls % 4 != 0) return false;  // scale rows must be 16-byte multiples
    if (((uintptr_t)in & 15) || (y && ((uintptr_t)y & 15))) return false;
    return bulk_plan<P, R>(NS, D, g.Ls, hasop).total_b <= 200 * 1024;
}

template <int P>
bool pipe_fits(const Geom& g, int NS, int pipe, bool hasop, const void* in, size_t elem) {
    if (NS < 1 || pipe < 2 || pipe > 3) return false;
    const int threads = (NS * g.Ls + 31) / 32 * 32;
    if (threads > 256 || ((uintptr_t)in & 15)) return false;
    const size_t smem = (size_t)pipe_stage_bytes<P>(pipe, threads) + (hasop ? (size_t)NS * 12 * (g.Ls + 1) * elem : 0);
    return smem <= 96 * 1024;
}

template <int P, typename K>
void launch_pipe(K k, const eofa_ctx* ctx, const Geom& g, int NS, int pipe, size_t elem, bool hasop, int par,
                 const void* in, void* out, const void* gauge, const Op5& op, const void* y, double a_out, double b_in,
                 double* red, int slot, cudaStream_t st) {
    const int threads = (NS * g.Ls + 31) / 32 * 32;
    const size_t smem =
        (size_t)pipe_stage_bytes<P>(pipe, threads) + (hasop ? (size_t)NS * 12 * (g.Ls + 1) * elem : 0);
    const int ntiles = (g.Vh + NS - 1) / NS;
    if (smem > 40 * 1024) EOFA_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    unsigned grid = grid_size(k, threads, smem, ntiles, ctx->sms);
    k<<<grid, threads, smem, st>>>(g, par, in, out, gauge, op, y, a_out, b_in, red, slot, NS);
}

template <int P, typename K>
void launch_bulk(K k, const eofa_ctx* ctx, const Geom& g, int NS, int D, bool hasop, int par, const void* in,
                 void* out, const void* gauge, const Op5& op, const void* y, double a_out, double b_in, double* red,
                 int slot, cudaStream_t st) {
    typedef typename Field<P>::R R;
    const BulkPlan pl = bulk_plan<P, R>(NS, D, g.Ls, hasop);
    const int threads = (NS * g.Ls + 31) / 32 * 32 + 32;
    const int ntiles = (g.Vh + NS - 1) / NS;
    if (pl.total_b > 40 * 1024)
        EOFA_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, pl.total_b));
    unsigned grid = grid_size(k, threads, pl.total_b, ntiles, ctx->sms);
    int* err = reinterpret_cast<int*>(ctx->red + RED_ERRWORD);
    int stall = 0;
    if (ctx->test_stall > 0) {
        ctx->test_stall--;
        stall = 1;
    }
    k<<<grid, threads, pl.total_b, st>>>(g, par, in, out, gauge, op, y, a_out, b_in, red, slot, NS, D, err, stall);
}

template <int P, typename KP2, typename KP3>
void launch_pipe_cfg(KP2 kp2, KP3 kp3, const eofa_ctx* ctx, const Geom& g, int cfg, size_t elem, bool hasop, int par,
                     const void* in, void* out, const void* gauge, const Op5& op, const void* y, double a_out,
                     double b_in, double* red, int slot, cudaStream_t st) {
    const int NS = cfg & 0xff, pipe = (cfg >> 8) & 0xf;
    if (pipe == 2)
        launch_pipe<P>(kp2, ctx, g, NS, 2, elem, hasop, par, in, out, gauge, op, y, a_out, b_in, red, slot, st);
    else
        launch_pipe<P>(kp3, ctx, g, NS, 3, elem, hasop, par, in, out, gauge, op, y, a_out, b_in, red, slot, st);
}

// Autotuned configuration, timed once per context and kernel variant with
// CUDA events on the launching stream: the direct kernel at the heuristic
// sites per tile NS and its halving / doubling, and the staged kernel at
// the same NS with ring depths 2 to 4.  The kernels are idempotent (they
// only write out and the reduction scratch), so the trial launches are
// harmless.  Small lattices, and launches during stream capture, use the
// heuristic direct configuration.
template <int P, typename K1, typename KB, typename KP2, typename KP3>
int tuned_cfg(K1 k1, KB kb, KP2 kp2, KP3 kp3, const eofa_ctx* ctx, const Geom& g, long long key, int ns0, size_t elem, bool hasop,
              int par, const void* in, void* out, const void* gauge, const Op5& op, const void* y, double a_out,
              double b_in, double* red, int slot, cudaStream_t st) {
    auto direct_ok = [&](int c) {
        return c >= 1 && (c * g.Ls + 31) / 32 * 32 <= 256 && (!hasop || (size_t)c * 12 * (g.Ls + 1) * elem <= 64 * 1024);
    };
    if (ctx->forced_cfg) {
        const int f = ctx->forced_cfg;
        if (f & CFG_BULK) {
            if (bulk_fits<P>(g, f & 0xff, (f >> 8) & 0xf, hasop, in, y)) return f;
        } else if (f & CFG_PIPE) {
            if (pipe_fits<P>(g, f & 0xff, (f >> 8) & 0xf, hasop, in, elem)) return f;
        } else if (direct_ok(f / 4)) {
            return (f / 4) * 4 + 1;
        }
    }
    auto it = ctx->tuned->find(key);
    if (it != ctx->tuned->end()) return it->second;
    const int def = ns0 * 4 + 1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    EOFA_CUDA(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone || (long long)g.Vh * g.Ls < (1LL << 20)) return def;
    // FP64 storage is bound by the FP64 pipe: every configuration was measured
    // within 1% (22.8-22.9 ms at 24^3 x 64 x 24), while trying them all costs
    // ~2 s of FP64 launches per context, so FP64 keeps the heuristic tile
    if (P == P64) return def;
    std::vector<int> cands;
    for (int c : {ns0 / 2, ns0, ns0 * 2, ns0 * 4})
        if (direct_ok(c)) cands.push_back(c * 4 + 1);
    for (int c : {ns0 / 2, ns0, ns0 * 2, ns0 * 4})
        for (int d = 2; d <= 4; d++)
            if (bulk_fits<P>(g, c, d, hasop, in, y)) cands.push_back(CFG_BULK | d << 8 | c);
    for (int c : {ns0 / 2, ns0, ns0 * 2})
        for (int d = 2; d <= 3; d++)
            if (pipe_fits<P>(g, c, d, hasop, in, elem)) cands.push_back(CFG_PIPE | d << 8 | c);
    int best = def;
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    EOFA_CUDA(cudaEventCreate(&e0));
    EOFA_CUDA(cudaEventCreate(&e1));
    for (int cfg : cands) {
        auto run = [&]() {
            if (cfg & CFG_BULK)
                launch_bulk<P>(kb, ctx, g, cfg & 0xff, (cfg >> 8) & 0xf, hasop, par, in, out, gauge, op, y, a_out,
                               b_in, red, slot, st);
            else if (cfg & CFG_PIPE)
                launch_pipe_cfg<P>(kp2, kp3, ctx, g, cfg, elem, hasop, par, in, out, gauge, op, y, a_out, b_in, red,
                                   slot, st);
            else
                launch_with(k1, ctx, g, cfg / 4, 1, elem, hasop, par, in, out, gauge, op, y, a_out, b_in, red, slot,
                            st);
        };
        run();  // warm
        EOFA_CUDA(cudaEventRecord(e0, st));
        for (int r = 0; r < 3; r++) run();
        EOFA_CUDA(cudaEventRecord(e1, st));
        EOFA_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        EOFA_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (getenv("EOFA_TUNE_LOG")) fprintf(stderr, "dslash tune key %lld: %s %.4f ms\n", key, cfg_str(cfg).c_str(), ms / 3);
        if (ms < best_ms) {
            best_ms = ms;
            best = cfg;
        }
    }
    EOFA_CUDA(cudaEventDestroy(e0));
    EOFA_CUDA(cudaEventDestroy(e1));
    EOFA_CUDA(cudaGetLastError());
    if (getenv("EOFA_TUNE_LOG")) fprintf(stderr, "dslash tune key %lld: best %s\n", key, cfg_str(best).c_str());
    (*ctx->tuned)[key] = best;
    return best;
}

// Two slices per thread (SPT = 2) was measured slower than one in every tile
// shape at 24^3 x 64 x 24 (0.79 vs 0.69 ms, FP32 hop), so only SPT = 1 is built.
template <int P, int DAG, int LS>
void launch_dslash_t(const eofa_ctx* ctx, int par, const void* in, void* out, const Op5& op, const void* y,
                     double a_out, double b_in, double* red, int slot, cudaStream_t st) {
    typedef typename Field<P>::R R;
    Geom g = ctx_geom(ctx);
    const void* gauge = ctx->gauge[P == P64 ? P64 : P32];
    const bool hasop = op.inv[0] || op.inv[1] || op.fwd[0] || op.fwd[1] || op.sigma[0] != 0.0 || op.sigma[1] != 0.0;
    auto k1 = hasop ? dslash_kernel<P, DAG, LS, true, 1> : dslash_kernel<P, DAG, LS, false, 1>;
    auto kb = hasop ? dslash_bulk_kernel<P, DAG, LS, true> : dslash_bulk_kernel<P, DAG, LS, false>;
    auto kp2 = hasop ? dslash_pipe_kernel<P, DAG, LS, true, 2> : dslash_pipe_kernel<P, DAG, LS, false, 2>;
    auto kp3 = hasop ? dslash_pipe_kernel<P, DAG, LS, true, 3> : dslash_pipe_kernel<P, DAG, LS, false, 3>;
    const long long key = ((((long long)P * 2 + DAG) * 128 + g.Ls) * 2 + (hasop ? 1 : 0)) * 2 + (y ? 1 : 0);
    const int ns0 = pick_ns(g.Ls, sizeof(cpx<R>));
    int cfg = tuned_cfg<P>(k1, kb, kp2, kp3, ctx, g, key, ns0, sizeof(cpx<R>), hasop, par, in, out, gauge, op, y, a_out, b_in,
                           red, slot, st);
    if ((cfg & CFG_BULK) && !bulk_fits<P>(g, cfg & 0xff, (cfg >> 8) & 0xf, hasop, in, y)) cfg = ns0 * 4 + 1;
    if ((cfg & CFG_PIPE) && !pipe_fits<P>(g, cfg & 0xff, (cfg >> 8) & 0xf, hasop, in, sizeof(cpx<R>)))
        cfg = ns0 * 4 + 1;
    if (cfg & CFG_PIPE)
        launch_pipe_cfg<P>(kp2, kp3, ctx, g, cfg, sizeof(cpx<R>), hasop, par, in, out, gauge, op, y, a_out, b_in, red,
                           slot, st);
    else if (cfg & CFG_BULK)
        launch_bulk<P>(kb, ctx, g, cfg & 0xff, (cfg >> 8) & 0xf, hasop, par, in, out, gauge, op, y, a_out, b_in, red,
                       slot, st);
    else
        launch_with(k1, ctx, g, cfg / 4, 1, sizeof(cpx<R>), hasop, par, in, out, gauge, op, y, a_out, b_in, red, slot,
                    st);
    EOFA_LAUNCHED();
}

// MODE 1 (second output, B = op) and MODE 2 (in-place update, B = identity)
// use the direct kernel at the sites per tile that the autotuner picked for
// the same hop shape (or the heuristic).
template <int P, int DAG, int LS, int MODE>
void launch_dslash_epi_t(const eofa_ctx* ctx, int par, const void* in, void* out, const Op5& op, const void* y,
                         double a_out, double b_in, double* red, int slot, const Epi& ep, cudaStream_t st) {
    typedef typename Field<P>::R R;
    Geom g = ctx_geom(ctx);
    const void* gauge = ctx->gauge[P == P64 ? P64 : P32];
    constexpr bool HASOP = MODE == 1 || MODE == 3;
    const long long key = ((((long long)P * 2 + DAG) * 128 + g.Ls) * 2 + (HASOP ? 1 : 0)) * 2 + (y ? 1 : 0);
    int NS = pick_ns(g.Ls, sizeof(cpx<R>));
    auto it = ctx->tuned->find(key);
    if (it != ctx->tuned->end() && !(it->second & (CFG_BULK | CFG_PIPE))) NS = it->second / 4;
    if (ctx->forced_cfg && !(ctx->forced_cfg & (CFG_BULK | CFG_PIPE))) NS = ctx->forced_cfg / 4;
    if ((NS * g.Ls + 31) / 32 * 32 > 256) NS = pick_ns(g.Ls, sizeof(cpx<R>));
    launch_epi(dslash_kernel<P, DAG, LS, HASOP, 1, MODE>, ctx, g, NS, sizeof(cpx<R>), HASOP, par, in, out, gauge, op,
               y, a_out, b_in, red, slot, ep, st);
    EOFA_LAUNCHED();
}

template <int P, int MODE>
void dslash_epi_prec(const eofa_ctx* ctx, int par, int dag, const void* in, void* out, const Op5& op, const void* y,
                     double a_out, double b_in, double* red, int slot, const Epi& ep, cudaStream_t st) {
#define EPI_CASE(L)                                                                                      \
    if (dag) launch_dslash_epi_t<P, 1, L, MODE>(ctx, par, in, out, op, y, a_out, b_in, red, slot, ep, st); \
    else launch_dslash_epi_t<P, 0, L, MODE>(ctx, par, in, out, op, y, a_out, b_in, red, slot, ep, st);
    switch (ctx->Ls) {
        case 8: EPI_CASE(8) break;
        case 12: EPI_CASE(12) break;
        case 16: EPI_CASE(16) break;
        case 24: EPI_CASE(24) break;
        default: EPI_CASE(0) break;
    }
#undef EPI_CASE
}

template <int P, int LS>
void launch_local5_t(const eofa_ctx* ctx, const Op5& op, const void* x, const void* z, double c0, const double* sc,
                     int it, int use_alpha, void* xw, void* out, double a_out, double* red, int slot, cudaStream_t st) {
    typedef typename Field<P>::R R;
    Geom g = ctx_geom(ctx);
    const int NS = pick_ns(g.Ls, sizeof(cpx<R>));
    const int threads = (NS * g.Ls + 31) / 32 * 32;
    const size_t smem = (size_t)NS * 12 * (g.Ls + 1) * sizeof(cpx<R>);
    const int ntiles = (g.Vh + NS - 1) / NS;
    auto k = local5_kernel<P, LS>;
    if (smem > 40 * 1024) EOFA_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    unsigned grid = grid_size(k, threads, smem, ntiles, ctx->sms);
    k<<<grid, threads, smem, st>>>(g, op, x, z, c0, sc, it, use_alpha, xw, out, a_out, red, slot, NS);
    EOFA_LAUNCHED();
}

// dispatch on Ls: unrolled columns for the common extents, shared-memory loops otherwise
template <int P>
void dslash_prec(const eofa_ctx* ctx, int par, int dag, const void* in, void* out, const Op5& op, const void* y,
                 double a_out, double b_in, double* red, int slot, cudaStream_t st) {
#define DSL_CASE(L)                                                                             \
    if (dag) launch_dslash_t<P, 1, L>(ctx, par, in, out, op, y, a_out, b_in, red, slot, st);   \
    else launch_dslash_t<P, 0, L>(ctx, par, in, out, op, y, a_out, b_in, red, slot, st);
    switch (ctx->Ls) {
        case 8: DSL_CASE(8) break;
        case 12: DSL_CASE(12) break;
        case 16: DSL_CASE(16) break;
        case 24: DSL_CASE(24) break;
        default: DSL_CASE(0) break;
    }
#undef DSL_CASE
}

template <int P>
void local5_prec(const eofa_ctx* ctx, const Op5& op, const void* x, const void* z, double c0, const double* sc,
                 int it, int use_alpha, void* xw, void* out, double a_out, double* red, int slot, cudaStream_t st) {
    switch (ctx->Ls) {
        case 8: launch_local5_t<P, 8>(ctx, op, x, z, c0, sc, it, use_alpha, xw, out, a_out, red, slot, st); break;
        case 12: launch_local5_t<P, 12>(ctx, op, x, z, c0, sc, it, use_alpha, xw, out, a_out, red, slot, st); break;
        case 16: launch_local5_t<P, 16>(ctx, op, x, z, c0, sc, it, use_alpha, xw, out, a_out, red, slot, st); break;
        case 24: launch_local5_t<P, 24>(ctx, op, x, z, c0, sc, it, use_alpha, xw, out, a_out, red, slot, st); break;
        default: launch_local5_t<P, 0>(ctx, op, x, z, c0, sc, it, use_alpha, xw, out, a_out, red, slot, st); break;
    }
}

template <int P, int PX>
void xp_update_prec(const eofa_ctx* ctx, const double* sc, int it, void* x, void* p, const void* s, cudaStream_t st) {
    Geom g = ctx_geom(ctx);
    long long n5 = (long long)g.Vh * g.Ls;
    long long nb = (n5 + 255) / 256;
    long long cap = (long long)ctx->sms * 8;
    unsigned grid = (unsigned)(nb < cap ? nb : cap);
    xp_update_kernel<P, PX><<<grid, 256, 0, st>>>(g, sc, it, x, p, s);
    EOFA_LAUNCHED();
}

}  // namespace
}  // namespace dsl

// per-precision entry points (dslash_p64.cu, dslash_p32.cu, dslash_p16.cu)
#define DSL_DECLARE(NAME)                                                                                        \
    void dslash_##NAME(const eofa_ctx* ctx, int par, int dag, const void* in, void* out, const Op5& op,         \
                       const void* y, double a_out, double b_in, double* red, int slot, cudaStream_t st);       \
    void local5_##NAME(const eofa_ctx* ctx, const Op5& op, const void* x, const void* z, double c0,            \
                       const double* sc, int it, int use_alpha, void* xw, void* out, double a_out, double* red, \
                       int slot, cudaStream_t st);                                                              \
    void xp_update_##NAME(const eofa_ctx* ctx, const double* sc, int it, void* x, void* p, const void* s,      \
                          cudaStream_t st);                                                                     \
    void dslash_to_##NAME(const eofa_ctx* ctx, int par, int dag, const void* in, void* out, const Op5& op,      \
                          const void* y, double a_out, double b_in, double* red, int slot, const Op5& op2,      \
                          void* out2, cudaStream_t st);                                                         \
    void dslash_z_##NAME(const eofa_ctx* ctx, int par, int dag, const void* in, void* z, const Op5& op,         \
                         const void* y, double a_out, double b_in, double* red, int slot, int it, void* r,      \
                         int rslot, cudaStream_t st);                                                           \
    void dslash_x_##NAME(const eofa_ctx* ctx, int par, int dag, const void* in, void* out, const Op5& op,       \
                         double* red, int it, void* x, const void* p, void* r, const void* q, int rslot,        \
                         cudaStream_t st);
DSL_DECLARE(p64)
DSL_DECLARE(p32)
DSL_DECLARE(p16)

#define DSL_DEFINE(NAME, P, PX)                                                                                  \
    void dslash_##NAME(const eofa_ctx* ctx, int par, int dag, const void* in, void* out, const Op5& op,         \
                       const void* y, double a_out, double b_in, double* red, int slot, cudaStream_t st) {      \
        dsl::dslash_prec<P>(ctx, par, dag, in, out, op, y, a_out, b_in, red, slot, st);                        \
    }                                                                                                           \
    void local5_##NAME(const eofa_ctx* ctx, const Op5& op, const void* x, const void* z, double c0,            \
                       const double* sc, int it, int use_alpha, void* xw, void* out, double a_out, double* red, \
                       int slot, cudaStream_t st) {                                                             \
        dsl::local5_prec<P>(ctx, op, x, z, c0, sc, it, use_alpha, xw, out, a_out, red, slot, st);               \
    }                                                                                                           \
    void xp_update_##NAME(const eofa_ctx* ctx, const double* sc, int it, void* x, void* p, const void* s,      \
                          cudaStream_t st) {                                                                    \
        dsl::xp_update_prec<P, PX>(ctx, sc, it, x, p, s, st);                                                   \
    }                                                                                                           \
    void dslash_to_##NAME(const eofa_ctx* ctx, int par, int dag, const void* in, void* out, const Op5& op,      \
                          const void* y, double a_out, double b_in, double* red, int slot, const Op5& op2,      \
                          void* out2, cudaStream_t st) {                                                        \
        dsl::Epi ep;                                                                                            \
        ep.op2 = op2;                                                                                           \
        ep.out2 = out2;                                                                                         \
        ep.aux = nullptr;                                                                                       \
        ep.out3 = nullptr;                                                                                      \
        ep.aux2 = nullptr;                                                                                      \
        ep.it = 0;                                                                                              \
        ep.slot2 = 0;                                                                                           \
        dsl::dslash_epi_prec<P, 1>(ctx, par, dag, in, out, op, y, a_out, b_in, red, slot, ep, st);              \
    }                                                                                                           \
    void dslash_z_##NAME(const eofa_ctx* ctx, int par, int dag, const void* in, void* z, const Op5& op,         \
                         const void* y, double a_out, double b_in, double* red, int slot, int it, void* r,      \
                         int rslot, cudaStream_t st) {                                                          \
        dsl::Epi ep;                                                                                            \
        ep.op2 = op;                                                                                            \
        ep.out2 = r;                                                                                            \
        ep.aux = nullptr;                                                                                       \
        ep.out3 = nullptr;                                                                                      \
        ep.aux2 = nullptr;                                                                                      \
        ep.it = it;                                                                                             \
        ep.slot2 = rslot;                                                                                       \
        dsl::dslash_epi_prec<P, 2>(ctx, par, dag, in, z, op, y, a_out, b_in, red, slot, ep, st);                \
    }                                                                                                           \
    void dslash_x_##NAME(const eofa_ctx* ctx, int par, int dag, const void* in, void* out, const Op5& op,       \
                         double* red, int it, void* x, const void* p, void* r, const void* q, int rslot,        \
                         cudaStream_t st) {                                                                     \
        dsl::Epi ep;                                                                                            \
        ep.op2 = op;                                                                                            \
        ep.out2 = x;                                                                                            \
        ep.aux = p;                                                                                             \
        ep.out3 = r;                                                                                            \
        ep.aux2 = q;                                                                                            \
        ep.it = it;                                                                                             \
        ep.slot2 = rslot;                                                                                       \
        dsl::dslash_epi_prec<P, 3>(ctx, par, dag, in, out, op, nullptr, 1.0, 0.0, red, -1, ep, st);             \
    }
