// Packed FP32 arithmetic on two right-hand sides at once.
//
// FP32 spinor fields store two RHS interleaved: for pair q (RHS 2q and 2q+1)
// and complex component k of site s the float4 at index (k*Vh + s)*P + q
// (P = n/2 pairs) holds (re_2q, re_2q+1, im_2q, im_2q+1).  A 64-bit register
// then carries the real (or imaginary) parts of both RHS, and every
// arithmetic step is one packed f32x2 instruction (fma/add/sub/mul .rn.f32x2,
// IEEE round-to-nearest per lane) for both RHS.  Quantities shared by the two
// RHS (links, hop factors, clover entries) are broadcast into both lanes.
#pragma once

#include <cuda_runtime.h>

namespace dp {

typedef unsigned long long f2;  // two packed floats (lane 0 in the low half)

__device__ __forceinline__ f2 bc(float s)
{
    f2 r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(s));
    return r;
}
__device__ __forceinline__ f2 pk(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 ffma2(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 fadd2(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fsub2(f2 a, f2 b)
{
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fmul2(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// exact negation of both lanes (sign bits)
__device__ __forceinline__ f2 fneg2(f2 a) { return a ^ 0x8000000080000000ull; }

// a complex number for two RHS
struct C2 {
    f2 re, im;
};

__device__ __forceinline__ C2 c2_add(C2 a, C2 b) { return {fadd2(a.re, b.re), fadd2(a.im, b.im)}; }
__device__ __forceinline__ C2 c2_sub(C2 a, C2 b) { return {fsub2(a.re, b.re), fsub2(a.im, b.im)}; }
// a + i b and a - i b
__device__ __forceinline__ C2 c2_addi(C2 a, C2 b) { return {fsub2(a.re, b.im), fadd2(a.im, b.re)}; }
__device__ __forceinline__ C2 c2_subi(C2 a, C2 b) { return {fadd2(a.re, b.im), fsub2(a.im, b.re)}; }

// a complex scalar shared by both lanes, broadcast: (re, im, -im)
struct B2 {
    f2 re, im, mim;
};
__device__ __forceinline__ B2 bcast(float re, float im)
{
    const f2 i = bc(im);
    return {bc(re), i, fneg2(i)};
}

// acc + u x (u shared), acc + conj(u) x
__device__ __forceinline__ C2 c2_fma(const B2 &u, C2 x, C2 acc)
{
    acc.re = ffma2(u.re, x.re, acc.re);
    acc.re = ffma2(u.mim, x.im, acc.re);
    acc.im = ffma2(u.re, x.im, acc.im);
    acc.im = ffma2(u.im, x.re, acc.im);
    return acc;
}
__device__ __forceinline__ C2 c2_mul(const B2 &u, C2 x)
{
    C2 r;
    r.re = fmul2(u.re, x.re);
    r.re = ffma2(u.mim, x.im, r.re);
    r.im = fmul2(u.re, x.im);
    r.im = ffma2(u.im, x.re, r.im);
    return r;
}
__device__ __forceinline__ C2 c2_cjfma(const B2 &u, C2 x, C2 acc)
{
    acc.re = ffma2(u.re, x.re, acc.re);
    acc.re = ffma2(u.im, x.im, acc.re);
    acc.im = ffma2(u.re, x.im, acc.im);
    acc.im = ffma2(u.mim, x.re, acc.im);
    return acc;
}
__device__ __forceinline__ C2 c2_cjmul(const B2 &u, C2 x)
{
    C2 r;
    r.re = fmul2(u.re, x.re);
    r.re = ffma2(u.im, x.im, r.re);
    r.im = fmul2(u.re, x.im);
    r.im = ffma2(u.mim, x.re, r.im);
    return r;
}

// per-lane complex scalars (different for the two RHS, e.g. BiCGStab's alpha)
__device__ __forceinline__ C2 c2_lanefma(C2 a, C2 x, C2 acc)
{
    acc.re = ffma2(a.re, x.re, acc.re);
    acc.re = ffma2(fneg2(a.im), x.im, acc.re);
    acc.im = ffma2(a.re, x.im, acc.im);
    acc.im = ffma2(a.im, x.re, acc.im);
    return acc;
}

// 12 complex components of a pair spinor; b points at component 0, cs is the
// stride between components (in float4 units)
__device__ __forceinline__ void load_pair(const float4 *__restrict__ b, long long cs, C2 s[12])
{
    const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(b);
#pragma unroll
    for (int k = 0; k < 12; k++) {
        const ulonglong2 v = __ldg(p + k * cs);
        s[k] = {v.x, v.y};
    }
}
__device__ __forceinline__ void store_pair(float4 *b, long long cs, const C2 s[12])
{
    ulonglong2 *p = reinterpret_cast<ulonglong2 *>(b);
#pragma unroll
    for (int k = 0; k < 12; k++) p[k * cs] = make_ulonglong2(s[k].re, s[k].im);
}

// y = H x for a packed Hermitian 6x6 block (scalar, shared by both lanes)
__device__ __forceinline__ void herm6_pair(const float m[36], const C2 *x, C2 *y)
{
#pragma unroll
    for (int i = 0; i < 6; i++) {
        const f2 d = bc(m[i]);
        y[i] = {fmul2(d, x[i].re), fmul2(d, x[i].im)};
    }
    int k = 6;
#pragma unroll
    for (int i = 0; i < 6; i++) {
#pragma unroll
        for (int j = i + 1; j < 6; j++) {
            const B2 a = bcast(m[k], m[k + 1]);
            k += 2;
            y[i] = c2_fma(a, x[j], y[i]);
            y[j] = c2_cjfma(a, x[i], y[j]);
        }
    }
}

}  // namespace dp
