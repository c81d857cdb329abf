// Device-side access to half-checkerboard 5D fields in the three storage
// precisions (layouts are described in internal.h).
#pragma once
#include "internal.h"

template <int P>
struct Field;

template <>
struct Field<P64> {
    typedef double R;  // arithmetic type
    static __device__ __forceinline__ void load(const void* base, int j, int s, int Ls, long long n5,
                                                cpx<double> v[12]) {
        const double2* b = (const double2*)base + (long long)j * 12 * Ls + s;
#pragma unroll
        for (int c = 0; c < 12; c++) {
            double2 t = __ldg(b + c * Ls);
            v[c] = mk(t.x, t.y);
        }
    }
    static __device__ __forceinline__ void store(void* base, int j, int s, int Ls, long long n5,
                                                 const cpx<double> v[12]) {
        double2* b = (double2*)base + (long long)j * 12 * Ls + s;
#pragma unroll
        for (int c = 0; c < 12; c++) b[c * Ls] = make_double2(v[c].re, v[c].im);
    }
    // read-once / write-once forms with the streaming cache hint (evict first)
    static __device__ __forceinline__ void load_stream(const void* base, int j, int s, int Ls, long long n5,
                                                       cpx<double> v[12]) {
        const double2* b = (const double2*)base + (long long)j * 12 * Ls + s;
#pragma unroll
        for (int c = 0; c < 12; c++) {
            double2 t = __ldcs(b + c * Ls);
            v[c] = mk(t.x, t.y);
        }
    }
    static __device__ __forceinline__ void store_stream(void* base, int j, int s, int Ls, long long n5,
                                                        const cpx<double> v[12]) {
        double2* b = (double2*)base + (long long)j * 12 * Ls + s;
#pragma unroll
        for (int c = 0; c < 12; c++) __stcs(b + c * Ls, make_double2(v[c].re, v[c].im));
    }
};

template <>
struct Field<P32> {
    typedef float R;
    static __device__ __forceinline__ void load(const void* base, int j, int s, int Ls, long long n5,
                                                cpx<float> v[12]) {
        const float4* b = (const float4*)base + (long long)j * 6 * Ls + s;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            float4 t = __ldg(b + k * Ls);
            v[2 * k] = mk(t.x, t.y);
            v[2 * k + 1] = mk(t.z, t.w);
        }
    }
    static __device__ __forceinline__ void store(void* base, int j, int s, int Ls, long long n5,
                                                 const cpx<float> v[12]) {
        float4* b = (float4*)base + (long long)j * 6 * Ls + s;
#pragma unroll
        for (int k = 0; k < 6; k++)
            b[k * Ls] = make_float4(v[2 * k].re, v[2 * k].im, v[2 * k + 1].re, v[2 * k + 1].im);
    }
    static __device__ __forceinline__ void load_stream(const void* base, int j, int s, int Ls, long long n5,
                                                       cpx<float> v[12]) {
        const float4* b = (const float4*)base + (long long)j * 6 * Ls + s;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            float4 t = __ldcs(b + k * Ls);
            v[2 * k] = mk(t.x, t.y);
            v[2 * k + 1] = mk(t.z, t.w);
        }
    }
    static __device__ __forceinline__ void store_stream(void* base, int j, int s, int Ls, long long n5,
                                                        const cpx<float> v[12]) {
        float4* b = (float4*)base + (long long)j * 6 * Ls + s;
#pragma unroll
        for (int k = 0; k < 6; k++)
            __stcs(b + k * Ls, make_float4(v[2 * k].re, v[2 * k].im, v[2 * k + 1].re, v[2 * k + 1].im));
    }
};

// FP16 storage: 12 complex as 24 halves in three 16-byte chunks; value =
// half * scale, scale = max |real component| of the site, so the stored
// halves lie in [-1, 1].
template <>
struct Field<P16> {
    typedef float R;
    static __device__ __forceinline__ const float* scales(const void* base, long long n5) {
        return (const float*)((const char*)base + n5 * 48);
    }
    static __device__ __forceinline__ void load(const void* base, int j, int s, int Ls, long long n5,
                                                cpx<float> v[12]) {
        const uint4* b = (const uint4*)base + (long long)j * 3 * Ls + s;
        float sc = __ldg(scales(base, n5) + (long long)j * Ls + s);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            uint4 t = __ldg(b + k * Ls);
            unsigned w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int e = 0; e < 4; e++) {
                __half2 h = *reinterpret_cast<__half2*>(&w[e]);
                float2 f = __half22float2(h);
                v[4 * k + e] = mk(f.x * sc, f.y * sc);
            }
        }
    }
    // the stored (unit-scale) values and the site's scale, for callers that
    // apply the scale after a linear step (the hop scales its half spinors)
    static __device__ __forceinline__ float load_unscaled(const void* base, int j, int s, int Ls, long long n5,
                                                          cpx<float> v[12]) {
        const uint4* b = (const uint4*)base + (long long)j * 3 * Ls + s;
        const float sc = __ldg(scales(base, n5) + (long long)j * Ls + s);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            uint4 t = __ldg(b + k * Ls);
            unsigned w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int e = 0; e < 4; e++) {
                __half2 h = *reinterpret_cast<__half2*>(&w[e]);
                float2 f = __half22float2(h);
                v[4 * k + e] = mk(f.x, f.y);
            }
        }
        return sc;
    }
    static __device__ __forceinline__ void store(void* base, int j, int s, int Ls, long long n5,
                                                 const cpx<float> v[12]) {
        float m = 0.f;
#pragma unroll
        for (int c = 0; c < 12; c++) m = fmaxf(m, fmaxf(fabsf(v[c].re), fabsf(v[c].im)));
        float sc = m;                       // stored values in [-1, 1]
        float inv = m > 0.f ? 1.f / m : 0.f;
        uint4* b = (uint4*)base + (long long)j * 3 * Ls + s;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            unsigned w[4];
#pragma unroll
            for (int e = 0; e < 4; e++) {
                __half2 h = __floats2half2_rn(v[4 * k + e].re * inv, v[4 * k + e].im * inv);
                w[e] = *reinterpret_cast<unsigned*>(&h);
            }
            b[k * Ls] = make_uint4(w[0], w[1], w[2], w[3]);
        }
        ((float*)((char*)base + n5 * 48))[(long long)j * Ls + s] = sc;
    }
    static __device__ __forceinline__ void load_stream(const void* base, int j, int s, int Ls, long long n5,
                                                       cpx<float> v[12]) {
        load(base, j, s, Ls, n5, v);
    }
    static __device__ __forceinline__ void store_stream(void* base, int j, int s, int Ls, long long n5,
                                                        const cpx<float> v[12]) {
        store(base, j, s, Ls, n5, v);
    }
};

// gauge link access: 9 complex per link, row-major
template <typename R>
struct Link {
    cpx<R> m[9];
};

template <typename R>
__device__ __forceinline__ void load_link(const void* g, long long idx, Link<R>& L);

template <>
__device__ __forceinline__ void load_link<double>(const void* g, long long idx, Link<double>& L) {
    const double2* b = (const double2*)g + idx * 9;
#pragma unroll
    for (int k = 0; k < 9; k++) {
        double2 t = __ldg(b + k);
        L.m[k] = mk(t.x, t.y);
    }
}

// FP32 links are padded to 10 complex (80 bytes) and read as five float4
template <>
__device__ __forceinline__ void load_link<float>(const void* g, long long idx, Link<float>& L) {
    const float4* b = (const float4*)g + idx * 5;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        float4 t = __ldg(b + k);
        L.m[2 * k] = mk(t.x, t.y);
        L.m[2 * k + 1] = mk(t.z, t.w);
    }
    float4 t = __ldg(b + 4);
    L.m[8] = mk(t.x, t.y);
}
