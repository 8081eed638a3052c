// qc_jones.cuh -- float32 complex and 2x2 Jones-matrix algebra for the solver kernels.
//
// A Jones matrix is stored row-major, [[a, b], [c, d]], matching the
// correlation order XX XY YX YY of the paper's row-major vectorisation
// (Eq. gvec, Eq. jones).
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

namespace qc {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * b
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// acc + conj(a) * b
__device__ __forceinline__ float2 cfma_conj(float2 a, float2 b, float2 acc)
{
    acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
    return acc;
}
__device__ __forceinline__ float cnorm2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// a b + c d  (fused: one multiply and three FMAs per component)
__device__ __forceinline__ float2 cdot(float2 a, float2 b, float2 c, float2 d)
{
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, fmaf(c.x, d.x, -c.y * d.y))),
                       fmaf(a.x, b.y, fmaf(a.y, b.x, fmaf(c.x, d.y, c.y * d.x))));
}
// a conj(b) + c conj(d)
__device__ __forceinline__ float2 cdotc(float2 a, float2 b, float2 c, float2 d)
{
    return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(c.x, d.x, c.y * d.y))),
                       fmaf(a.y, b.x, fmaf(-a.x, b.y, fmaf(c.y, d.x, -c.x * d.y))));
}

struct J2 {
    float2 a, b, c, d;
};

__device__ __forceinline__ J2 j_identity()
{
    J2 r;
    r.a = make_float2(1.f, 0.f); r.b = make_float2(0.f, 0.f);
    r.c = make_float2(0.f, 0.f); r.d = make_float2(1.f, 0.f);
    return r;
}

// A B
__device__ __forceinline__ J2 j_mul(const J2 &A, const J2 &B)
{
    J2 r;
    r.a = cdot(A.a, B.a, A.b, B.c);
    r.b = cdot(A.a, B.b, A.b, B.d);
    r.c = cdot(A.c, B.a, A.d, B.c);
    r.d = cdot(A.c, B.b, A.d, B.d);
    return r;
}

// A B^H
__device__ __forceinline__ J2 j_mul_h(const J2 &A, const J2 &B)
{
    J2 r;
    r.a = cdotc(A.a, B.a, A.b, B.b);
    r.b = cdotc(A.a, B.c, A.b, B.d);
    r.c = cdotc(A.c, B.a, A.d, B.b);
    r.d = cdotc(A.c, B.c, A.d, B.d);
    return r;
}

// A^H
__device__ __forceinline__ J2 j_herm(const J2 &A)
{
    J2 r;
    r.a = cconj(A.a); r.b = cconj(A.c);
    r.c = cconj(A.b); r.d = cconj(A.d);
    return r;
}

// diag(x, y) A   (left multiply by a diagonal Jones)
__device__ __forceinline__ J2 j_dmul(float2 x, float2 y, const J2 &A)
{
    J2 r;
    r.a = cmul(x, A.a); r.b = cmul(x, A.b);
    r.c = cmul(y, A.c); r.d = cmul(y, A.d);
    return r;
}

// A diag(x, y)
__device__ __forceinline__ J2 j_muld(const J2 &A, float2 x, float2 y)
{
    J2 r;
    r.a = cmul(A.a, x); r.b = cmul(A.b, y);
    r.c = cmul(A.c, x); r.d = cmul(A.d, y);
    return r;
}

__device__ __forceinline__ J2 j_from(float4 lo, float4 hi)
{
    J2 r;
    r.a = make_float2(lo.x, lo.y); r.b = make_float2(lo.z, lo.w);
    r.c = make_float2(hi.x, hi.y); r.d = make_float2(hi.z, hi.w);
    return r;
}

__device__ __forceinline__ J2 j_diag(float4 v)
{
    J2 r;
    r.a = make_float2(v.x, v.y); r.b = make_float2(0.f, 0.f);
    r.c = make_float2(0.f, 0.f); r.d = make_float2(v.z, v.w);
    return r;
}

__device__ __forceinline__ float2 h2f(__half2 h) { return __half22float2(h); }

// Two-sum (Knuth): s + c accumulates x with the rounding error of s carried in c.
__device__ __forceinline__ void two_sum_add(float &s, float &c, float x)
{
    float t = s + x;
    float z = t - s;
    c += (s - (t - z)) + (x - z);
    s = t;
}

} // namespace qc
