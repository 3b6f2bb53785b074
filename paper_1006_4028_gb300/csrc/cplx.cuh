// Small complex-arithmetic helpers and spinor/link/clover loaders used by the
// kernels.  Layouts are described in dp_internal.h.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "dp_internal.h"

namespace dp {

template <typename R>
struct Cx {
    R re, im;
};

__device__ __forceinline__ float fmx(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmx(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename R>
__device__ __forceinline__ Cx<R> cx(R a, R b) { return Cx<R>{a, b}; }
template <typename R>
__device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R>
__device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R>
__device__ __forceinline__ Cx<R> operator-(Cx<R> a) { return {-a.re, -a.im}; }
// a * b
template <typename R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// conj(a) * b
template <typename R>
__device__ __forceinline__ Cx<R> cjmul(Cx<R> a, Cx<R> b)
{
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// acc + a * b
template <typename R>
__device__ __forceinline__ Cx<R> cfma(Cx<R> a, Cx<R> b, Cx<R> acc)
{
    acc.re = fmx(a.re, b.re, acc.re);
    acc.re = fmx(-a.im, b.im, acc.re);
    acc.im = fmx(a.re, b.im, acc.im);
    acc.im = fmx(a.im, b.re, acc.im);
    return acc;
}
// acc + conj(a) * b
template <typename R>
__device__ __forceinline__ Cx<R> cjfma(Cx<R> a, Cx<R> b, Cx<R> acc)
{
    acc.re = fmx(a.re, b.re, acc.re);
    acc.re = fmx(a.im, b.im, acc.re);
    acc.im = fmx(a.re, b.im, acc.im);
    acc.im = fmx(-a.im, b.re, acc.im);
    return acc;
}
// i * a and -i * a
template <typename R>
__device__ __forceinline__ Cx<R> mul_i(Cx<R> a) { return {-a.im, a.re}; }
template <typename R>
__device__ __forceinline__ Cx<R> mul_mi(Cx<R> a) { return {a.im, -a.re}; }
template <typename R>
__device__ __forceinline__ Cx<R> scale(R c, Cx<R> a) { return {c * a.re, c * a.im}; }

// ---- spinor chunks -------------------------------------------------------
template <typename R>
struct Chunk;
template <>
struct Chunk<float> {
    using T = float4;
    static constexpr int kPerSpinor = 6;
};
template <>
struct Chunk<double> {
    using T = double2;
    static constexpr int kPerSpinor = 12;
};

// load the 12 complex components of one spinor; b points at chunk 0, cs is
// the stride between chunks (in chunks)
__device__ __forceinline__ void load_spinor(const float4 *__restrict__ b, long long cs,
                                            Cx<float> s[12])
{
#pragma unroll
    for (int c = 0; c < 6; c++) {
        float4 v = __ldg(b + c * cs);
        s[2 * c] = {v.x, v.y};
        s[2 * c + 1] = {v.z, v.w};
    }
}
__device__ __forceinline__ void load_spinor(const double2 *__restrict__ b, long long cs,
                                            Cx<double> s[12])
{
#pragma unroll
    for (int c = 0; c < 12; c++) {
        double2 v = __ldg(b + c * cs);
        s[c] = {v.x, v.y};
    }
}
__device__ __forceinline__ void store_spinor(float4 *b, long long cs, const Cx<float> s[12])
{
#pragma unroll
    for (int c = 0; c < 6; c++)
        b[c * cs] = make_float4(s[2 * c].re, s[2 * c].im, s[2 * c + 1].re, s[2 * c + 1].im);
}
__device__ __forceinline__ void store_spinor(double2 *b, long long cs, const Cx<double> s[12])
{
#pragma unroll
    for (int c = 0; c < 12; c++) b[c * cs] = make_double2(s[c].re, s[c].im);
}

// ---- links -----------------------------------------------------------------
// full 3x3 link U_mu at half-site `site` of the given parity array
template <int LF, typename R>
__device__ __forceinline__ void load_link(const void *base, long long Vh, long long site, int mu,
                                          Cx<R> u[9]);

template <>
__device__ __forceinline__ void load_link<LINK_F64_18, double>(const void *base, long long Vh,
                                                              long long site, int mu,
                                                              Cx<double> u[9])
{
    const double2 *l = static_cast<const double2 *>(base) + (long long)mu * 9 * Vh + site;
#pragma unroll
    for (int k = 0; k < 9; k++) {
        double2 v = __ldg(l + k * Vh);
        u[k] = {v.x, v.y};
    }
}

// 18-real FP32 storage: entries 0-7 as four float4 [mu][k][s] (two complex
// entries each), entry 8 as a float2 [mu][s] after them (72 bytes a link)
template <>
__device__ __forceinline__ void load_link<LINK_F32_18, float>(const void *base, long long Vh,
                                                             long long site, int mu,
                                                             Cx<float> u[9])
{
    const float4 *l = static_cast<const float4 *>(base) + (long long)mu * 4 * Vh + site;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const float4 v = __ldg(l + k * Vh);
        u[2 * k] = {v.x, v.y};
        u[2 * k + 1] = {v.z, v.w};
    }
    const float2 w = __ldg(reinterpret_cast<const float2 *>(static_cast<const float4 *>(base) + 16 * Vh) +
                           (long long)mu * Vh + site);
    u[8] = {w.x, w.y};
}

// 12-real storage: rows 0 and 1; row 2 = conj(row0 x row1) (unitary, det 1)
template <>
__device__ __forceinline__ void load_link<LINK_F32_12, float>(const void *base, long long Vh,
                                                             long long site, int mu,
                                                             Cx<float> u[9])
{
    const float4 *l = static_cast<const float4 *>(base) + (long long)mu * 3 * Vh + site;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        float4 v = __ldg(l + k * Vh);
        u[2 * k] = {v.x, v.y};
        u[2 * k + 1] = {v.z, v.w};
    }
    // u20 = conj(u01 u12 - u02 u11), u21 = conj(u02 u10 - u00 u12), u22 = conj(u00 u11 - u01 u10)
    Cx<float> a = cmul(u[1], u[5]) - cmul(u[2], u[4]);
    Cx<float> b = cmul(u[2], u[3]) - cmul(u[0], u[5]);
    Cx<float> c = cmul(u[0], u[4]) - cmul(u[1], u[3]);
    u[6] = {a.re, -a.im};
    u[7] = {b.re, -b.im};
    u[8] = {c.re, -c.im};
}

// 16-bit storage: rows 0 and 1 in FP16 / BF16 times one FP32 scale per link,
// row 2 rebuilt as above
template <typename H2>
__device__ __forceinline__ float2 h2f(unsigned v);
template <>
__device__ __forceinline__ float2 h2f<__half2>(unsigned v)
{
    __half2 h;
    memcpy(&h, &v, 4);
    return __half22float2(h);
}
template <>
__device__ __forceinline__ float2 h2f<__nv_bfloat162>(unsigned v)
{
    __nv_bfloat162 h;
    memcpy(&h, &v, 4);
    return __bfloat1622float2(h);
}

template <typename H2>
__device__ __forceinline__ void load_link16(const void *base, long long Vh, long long site, int mu,
                                            Cx<float> u[9])
{
    const uint2 *l = static_cast<const uint2 *>(base) + (long long)mu * 3 * Vh + site;
    const float sc = __ldg(reinterpret_cast<const float *>(static_cast<const uint2 *>(base) + 12 * Vh) +
                           (long long)mu * Vh + site);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const uint2 v = __ldg(l + k * Vh);
        const float2 a = h2f<H2>(v.x), b = h2f<H2>(v.y);
        u[2 * k] = {sc * a.x, sc * a.y};
        u[2 * k + 1] = {sc * b.x, sc * b.y};
    }
    Cx<float> a = cmul(u[1], u[5]) - cmul(u[2], u[4]);
    Cx<float> b = cmul(u[2], u[3]) - cmul(u[0], u[5]);
    Cx<float> c = cmul(u[0], u[4]) - cmul(u[1], u[3]);
    u[6] = {a.re, -a.im};
    u[7] = {b.re, -b.im};
    u[8] = {c.re, -c.im};
}

template <>
__device__ __forceinline__ void load_link<LINK_H16_12, float>(const void *base, long long Vh,
                                                             long long site, int mu,
                                                             Cx<float> u[9])
{
    load_link16<__half2>(base, Vh, site, mu, u);
}
template <>
__device__ __forceinline__ void load_link<LINK_B16_12, float>(const void *base, long long Vh,
                                                             long long site, int mu,
                                                             Cx<float> u[9])
{
    load_link16<__nv_bfloat162>(base, Vh, site, mu, u);
}

// ---- clover blocks ------------------------------------------------------------
// the 36 reals of chiral block `blk` (0: spins 0,1; 1: spins 2,3) of a site
__device__ __forceinline__ void load_clover_block(const float4 *__restrict__ base, long long Vh,
                                                  long long site, int blk, float m[36])
{
    const float4 *c = base + (long long)blk * 9 * Vh + site;
#pragma unroll
    for (int k = 0; k < 9; k++) {
        float4 v = __ldg(c + k * Vh);
        m[4 * k] = v.x;
        m[4 * k + 1] = v.y;
        m[4 * k + 2] = v.z;
        m[4 * k + 3] = v.w;
    }
}
__device__ __forceinline__ void load_clover_block(const double2 *__restrict__ base, long long Vh,
                                                  long long site, int blk, double m[36])
{
    const double2 *c = base + (long long)blk * 18 * Vh + site;
#pragma unroll
    for (int k = 0; k < 18; k++) {
        double2 v = __ldg(c + k * Vh);
        m[2 * k] = v.x;
        m[2 * k + 1] = v.y;
    }
}

// y = H x for a packed Hermitian 6x6 block (6 real diagonal, then (re, im) of
// the upper triangle i<j in row-major order)
template <typename R>
__device__ __forceinline__ void herm6_apply(const R m[36], const Cx<R> *x, Cx<R> *y)
{
#pragma unroll
    for (int i = 0; i < 6; i++) y[i] = scale(m[i], x[i]);
    int k = 6;
#pragma unroll
    for (int i = 0; i < 6; i++) {
#pragma unroll
        for (int j = i + 1; j < 6; j++) {
            Cx<R> a = {m[k], m[k + 1]};
            k += 2;
            y[i] = cfma(a, x[j], y[i]);
            y[j] = cjfma(a, x[i], y[j]);
        }
    }
}

}  // namespace dp
