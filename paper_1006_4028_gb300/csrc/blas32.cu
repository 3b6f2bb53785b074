// FP32 inner-solver BLAS-1 kernels on the paired layout of pair.cuh: one
// thread per (site, RHS pair), every update one packed f32x2 instruction for
// the two RHS, per-RHS scalars (alpha, omega, beta) held per lane.  Dot
// products are summed in FP32 over the sites one thread visits (24 terms a
// site, a few tens of sites: one packed f32x2 add per site and value, where
// an FP64 add per site would run on GB300's 1/64-rate FP64 pipe) and across
// threads and blocks in FP64 per RHS; the reductions and the scalar
// recurrences (those the FP64 kernels share, and the shadow-form BiCGStab's
// own) are in reduce.cuh, so every decision stays per RHS.
//
// A pair is processed while either of its RHS is active; an inactive lane's
// solution x is never changed (lane blend), and its terms are excluded from
// every reduction.  Other vectors of an inactive lane are scratch.
#include "cplx.cuh"
#include "dp_internal.h"
#include "pair.cuh"
#include "reduce.cuh"

namespace dp {
namespace {

struct P12 {
    C2 c[12];
};

__device__ __forceinline__ P12 ldp(const void *base, long long cs, long long me)
{
    P12 v;
    load_pair(static_cast<const float4 *>(base) + me, cs, v.c);
    return v;
}
__device__ __forceinline__ void stp(void *base, long long cs, long long me, const P12 &v)
{
    store_pair(static_cast<float4 *>(base) + me, cs, v.c);
}

// component k of one pair
__device__ __forceinline__ C2 ld1(const void *base, long long cs, long long me, int k)
{
    const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(base) + me + k * cs);
    return {v.x, v.y};
}
__device__ __forceinline__ void st1(void *base, long long cs, long long me, int k, C2 v)
{
    reinterpret_cast<ulonglong2 *>(base)[me + k * cs] = make_ulonglong2(v.re, v.im);
}

// per-lane complex scalar from the two RHS states
__device__ __forceinline__ C2 lanes(double2 a0, double2 a1)
{
    return {pk((float)a0.x, (float)a1.x), pk((float)a0.y, (float)a1.y)};
}
__device__ __forceinline__ C2 neg(C2 a) { return {fneg2(a.re), fneg2(a.im)}; }

// <a, b> per lane over one site, FP32
__device__ __forceinline__ C2 pdot(const P12 &a, const P12 &b)
{
    f2 re = 0ull, im = 0ull;
#pragma unroll
    for (int k = 0; k < 12; k++) {
        re = ffma2(a.c[k].re, b.c[k].re, re);
        re = ffma2(a.c[k].im, b.c[k].im, re);
        im = ffma2(a.c[k].re, b.c[k].im, im);
        im = ffma2(fneg2(a.c[k].im), b.c[k].re, im);
    }
    return {re, im};
}
__device__ __forceinline__ f2 pnorm(const P12 &a)
{
    f2 s = 0ull;
#pragma unroll
    for (int k = 0; k < 12; k++) {
        s = ffma2(a.c[k].re, a.c[k].re, s);
        s = ffma2(a.c[k].im, a.c[k].im, s);
    }
    return s;
}

// add the two lanes of an f2 into FP64 accumulators, only for active lanes
__device__ __forceinline__ void add_lanes(double &d0, double &d1, f2 v, bool a0, bool a1)
{
    float l0, l1;
    upk(v, l0, l1);
    if (a0) d0 += (double)l0;
    if (a1) d1 += (double)l1;
}

#define PAIR_LOOP                                                              \
    const int P = nrhs / 2;                                                    \
    const int q = threadIdx.x % P, lane = threadIdx.x / P;                     \
    const long long cs = Vh * P;                                               \
    const bool a0 = st[2 * q].active != 0, a1 = st[2 * q + 1].active != 0;     \
    for (long long s = (long long)blockIdx.x * c.lanes + lane; (a0 || a1) && s < Vh; \
         s += (long long)gridDim.x * c.lanes)

__global__ void __launch_bounds__(kMaxBlock) k32_alpha(Cfg c, const void *rh, const void *vv, long long Vh, int nrhs,
                          RhsState *st, double *partials, unsigned int *counter)
{
    double acc[4] = {0, 0, 0, 0};  // lane 0: re, im; lane 1: re, im
    {
        f2 sum0 = 0ull, sum1 = 0ull;
        PAIR_LOOP
        {
            const long long me = s * P + q;
            const C2 d = pdot(ldp(rh, cs, me), ldp(vv, cs, me));
            sum0 = fadd2(sum0, d.re);
            sum1 = fadd2(sum1, d.im);
        }
        add_lanes(acc[0], acc[2], sum0, a0, a1);
        add_lanes(acc[1], acc[3], sum1, a0, a1);
    }
    const int q = threadIdx.x % (nrhs / 2);
    if (!reduce_last<2, 2>(acc, c, partials, counter, nrhs / 2)) return;
    finish_alpha(st[2 * q], acc[0], acc[1]);
    finish_alpha(st[2 * q + 1], acc[2], acc[3]);
}

// keep the lanes of `old` whose RHS is inactive
__device__ __forceinline__ f2 blend(f2 nw, f2 old, f2 m) { return (nw & m) | (old & ~m); }

__global__ void __launch_bounds__(kMaxBlock) k32_init(Cfg c, const void *bv, void *rv, void *rh, void *pv,
                                                      long long Vh, int nrhs, RhsState *st,
                                                      double *partials, unsigned int *counter)
{
    double acc[2] = {0, 0};
    {
        f2 sum0 = 0ull;
        PAIR_LOOP
        {
            const long long me = s * P + q;
            const P12 b = ldp(bv, cs, me);
            stp(rv, cs, me, b);
            stp(rh, cs, me, b);
            if (pv) stp(pv, cs, me, b);
            sum0 = fadd2(sum0, pnorm(b));
        }
        add_lanes(acc[0], acc[1], sum0, a0, a1);
    }
    const int q = threadIdx.x % (nrhs / 2);
    if (!reduce_last<1, 2>(acc, c, partials, counter, nrhs / 2)) return;
    finish_init(st[2 * q], acc[0]);
    finish_init(st[2 * q + 1], acc[1]);
}

// ---- BiCGStab with the shadow image rhat' = Mhat^dag rhat ----
//
// <rhat, v> = <rhat', p> is formed where p is written (update_pa), <rhat, t>
// = <rhat', s> where s is written (s_dots), <t, s> and |t|^2 in the
// x - A^-1 D launch that forms t (per-site sums, totalled by omega_dots):
// 14 vector streams per iteration (s_dots: r, v, rhat, rhat' -> s; update:
// x, p, s, t, v, rhat' -> x, r, p) and no separate alpha or omega pass.

__global__ void __launch_bounds__(kMaxBlock) k32_s_dots(Cfg c, const void *rv, const void *vv,
                                                        void *sv, const void *rh, const void *rh2,
                                                        long long Vh, int nrhs, RhsState *st,
                                                        double *partials, unsigned int *counter)
{
    double acc[8];
#pragma unroll
    for (int k = 0; k < 8; k++) acc[k] = 0;
    {
        const int qq = threadIdx.x % (nrhs / 2);
        const C2 mal = neg(lanes(st[2 * qq].alpha, st[2 * qq + 1].alpha));
        f2 sum0 = 0ull, sum1 = 0ull, sum2 = 0ull, sum3 = 0ull;
        PAIR_LOOP
        {
            const long long me = s * P + q;
            f2 rsr = 0ull, rsi = 0ull, rtr = 0ull, rti = 0ull;
#pragma unroll 4
            for (int k = 0; k < 12; k++) {
                // every load ahead of the store (the pointers may alias, so a
                // later load could not be moved above it)
                const C2 r = ld1(rv, cs, me, k), v = ld1(vv, cs, me, k);
                const C2 h = ld1(rh, cs, me, k), h2 = ld1(rh2, cs, me, k);
                const C2 sx = c2_lanefma(mal, v, r);
                st1(sv, cs, me, k, sx);
                rsr = ffma2(h.re, sx.re, rsr);
                rsr = ffma2(h.im, sx.im, rsr);
                rsi = ffma2(h.re, sx.im, rsi);
                rsi = ffma2(fneg2(h.im), sx.re, rsi);
                rtr = ffma2(h2.re, sx.re, rtr);
                rtr = ffma2(h2.im, sx.im, rtr);
                rti = ffma2(h2.re, sx.im, rti);
                rti = ffma2(fneg2(h2.im), sx.re, rti);
            }
            sum0 = fadd2(sum0, rsr);
            sum1 = fadd2(sum1, rsi);
            sum2 = fadd2(sum2, rtr);
            sum3 = fadd2(sum3, rti);
        }
        add_lanes(acc[0], acc[4], sum0, a0, a1);
        add_lanes(acc[1], acc[5], sum1, a0, a1);
        add_lanes(acc[2], acc[6], sum2, a0, a1);
        add_lanes(acc[3], acc[7], sum3, a0, a1);
    }
    const int q = threadIdx.x % (nrhs / 2);
    if (!reduce_last<4, 2>(acc, c, partials, counter, nrhs / 2)) return;
    finish_s_dots(st[2 * q], acc[0], acc[1], acc[2], acc[3]);
    finish_s_dots(st[2 * q + 1], acc[4], acc[5], acc[6], acc[7]);
}

__global__ void __launch_bounds__(kMaxBlock) k32_omega_dots(Cfg c, const void *dots, long long Vh,
                                                            int nrhs, RhsState *st,
                                                            double *partials, unsigned int *counter)
{
    double acc[6] = {0, 0, 0, 0, 0, 0};
    {
        const f2 *d = static_cast<const f2 *>(dots);
        f2 sum0 = 0ull, sum1 = 0ull, sum2 = 0ull;
        PAIR_LOOP
        {
            const long long me = s * P + q;
            sum0 = fadd2(sum0, __ldg(d + me));
            sum1 = fadd2(sum1, __ldg(d + cs + me));
            sum2 = fadd2(sum2, __ldg(d + 2 * cs + me));
        }
        add_lanes(acc[0], acc[3], sum0, a0, a1);
        add_lanes(acc[1], acc[4], sum1, a0, a1);
        add_lanes(acc[2], acc[5], sum2, a0, a1);
    }
    const int q = threadIdx.x % (nrhs / 2);
    if (!reduce_last<3, 2>(acc, c, partials, counter, nrhs / 2)) return;
    finish_omega_shadow(st[2 * q], acc[0], acc[1], acc[2]);
    finish_omega_shadow(st[2 * q + 1], acc[3], acc[4], acc[5]);
}

__global__ void __launch_bounds__(kMaxBlock)
k32_update_pa(Cfg c, void *xv, void *rv, void *pv, const void *sv, const void *tv, const void *vv,
              const void *rh2, long long Vh, int nrhs, RhsState *st, int max_iter,
              double *partials, unsigned int *counter)
{
    double acc[6] = {0, 0, 0, 0, 0, 0};
    {
        const int qq = threadIdx.x % (nrhs / 2);
        const C2 al = lanes(st[2 * qq].alpha, st[2 * qq + 1].alpha);
        const C2 om = lanes(st[2 * qq].omega, st[2 * qq + 1].omega);
        const C2 be = lanes(st[2 * qq].beta, st[2 * qq + 1].beta);
        const C2 mom = neg(om);
        f2 sum0 = 0ull, sum1 = 0ull, sum2 = 0ull;
        PAIR_LOOP
        {
            const long long me = s * P + q;
            const f2 m = (a0 ? 0x00000000ffffffffull : 0ull) | (a1 ? 0xffffffff00000000ull : 0ull);
            f2 nn = 0ull, rpr = 0ull, rpi = 0ull;
#pragma unroll 4
            for (int k = 0; k < 12; k++) {
                const C2 x = ld1(xv, cs, me, k), p = ld1(pv, cs, me, k), sx = ld1(sv, cs, me, k);
                const C2 t = ld1(tv, cs, me, k), v = ld1(vv, cs, me, k);
                const C2 h2 = ld1(rh2, cs, me, k);  // with the others, ahead of the stores
                C2 xn = c2_lanefma(om, sx, c2_lanefma(al, p, x));
                xn.re = blend(xn.re, x.re, m);
                xn.im = blend(xn.im, x.im, m);
                st1(xv, cs, me, k, xn);
                const C2 r = c2_lanefma(mom, t, sx);
                st1(rv, cs, me, k, r);
                const C2 pn = c2_lanefma(be, c2_lanefma(mom, v, p), r);
                st1(pv, cs, me, k, pn);
                nn = ffma2(r.re, r.re, nn);
                nn = ffma2(r.im, r.im, nn);
                rpr = ffma2(h2.re, pn.re, rpr);
                rpr = ffma2(h2.im, pn.im, rpr);
                rpi = ffma2(h2.re, pn.im, rpi);
                rpi = ffma2(fneg2(h2.im), pn.re, rpi);
            }
            sum0 = fadd2(sum0, nn);
            sum1 = fadd2(sum1, rpr);
            sum2 = fadd2(sum2, rpi);
        }
        add_lanes(acc[0], acc[3], sum0, a0, a1);
        add_lanes(acc[1], acc[4], sum1, a0, a1);
        add_lanes(acc[2], acc[5], sum2, a0, a1);
    }
    const int q = threadIdx.x % (nrhs / 2);
    if (!reduce_last<3, 2>(acc, c, partials, counter, nrhs / 2)) return;
    // convergence on |r|^2, then the next alpha = rho' / <rhat', p> for the
    // RHS still iterating
    finish_update_rr(st[2 * q], acc[0], max_iter);
    finish_alpha(st[2 * q], acc[1], acc[2]);
    finish_update_rr(st[2 * q + 1], acc[3], max_iter);
    finish_alpha(st[2 * q + 1], acc[4], acc[5]);
}

// ---- CGNE on the normal equations: real per-RHS scalars, per lane ----

__device__ __forceinline__ f2 lanes_re(double a0, double a1) { return pk((float)a0, (float)a1); }

__global__ void __launch_bounds__(kMaxBlock)
k32_cg_gamma(Cfg c, const void *zv, long long Vh, int nrhs, RhsState *st, int first,
             double *partials, unsigned int *counter)
{
    double acc[2] = {0, 0};
    {
        f2 sum0 = 0ull;
        PAIR_LOOP
        {
            const long long me = s * P + q;
            f2 nn = 0ull;
#pragma unroll
            for (int k = 0; k < 12; k++) {
                const C2 z = ld1(zv, cs, me, k);
                nn = ffma2(z.re, z.re, nn);
                nn = ffma2(z.im, z.im, nn);
            }
            sum0 = fadd2(sum0, nn);
        }
        add_lanes(acc[0], acc[1], sum0, a0, a1);
    }
    const int q = threadIdx.x % (nrhs / 2);
    if (!reduce_last<1, 2>(acc, c, partials, counter, nrhs / 2)) return;
    finish_cg_gamma(st[2 * q], acc[0], first);
    finish_cg_gamma(st[2 * q + 1], acc[1], first);
}

// p = z + beta p
__global__ void __launch_bounds__(kMaxBlock)
k32_cg_p(Cfg c, const void *zv, void *pv, long long Vh, int nrhs, const RhsState *st)
{
    const int qq = threadIdx.x % (nrhs / 2);
    const f2 be = lanes_re(st[2 * qq].beta.x, st[2 * qq + 1].beta.x);
    PAIR_LOOP
    {
        const long long me = s * P + q;
#pragma unroll
        for (int k = 0; k < 12; k++) {
            const C2 z = ld1(zv, cs, me, k);
            C2 p = ld1(pv, cs, me, k);
            p.re = ffma2(be, p.re, z.re);
            p.im = ffma2(be, p.im, z.im);
            st1(pv, cs, me, k, p);
        }
    }
}

// alpha = rho / |w|^2
__global__ void __launch_bounds__(kMaxBlock)
k32_cg_alpha(Cfg c, const void *wv, long long Vh, int nrhs, RhsState *st, double *partials,
             unsigned int *counter)
{
    double acc[2] = {0, 0};
    {
        f2 sum0 = 0ull;
        PAIR_LOOP
        {
            const long long me = s * P + q;
            f2 nn = 0ull;
#pragma unroll
            for (int k = 0; k < 12; k++) {
                const C2 w = ld1(wv, cs, me, k);
                nn = ffma2(w.re, w.re, nn);
                nn = ffma2(w.im, w.im, nn);
            }
            sum0 = fadd2(sum0, nn);
        }
        add_lanes(acc[0], acc[1], sum0, a0, a1);
    }
    const int q = threadIdx.x % (nrhs / 2);
    if (!reduce_last<1, 2>(acc, c, partials, counter, nrhs / 2)) return;
    finish_cg_alpha(st[2 * q], acc[0]);
    finish_cg_alpha(st[2 * q + 1], acc[1]);
}

// x += alpha p (active lanes only), r -= alpha w, |r|^2
__global__ void __launch_bounds__(kMaxBlock)
k32_cg_update(Cfg c, void *xv, void *rv, const void *pv, const void *wv, long long Vh, int nrhs,
              RhsState *st, int max_iter, double *partials, unsigned int *counter)
{
    double acc[2] = {0, 0};
    {
        const int qq = threadIdx.x % (nrhs / 2);
        const f2 al = lanes_re(st[2 * qq].alpha.x, st[2 * qq + 1].alpha.x);
        const f2 mal = fneg2(al);
        f2 sum0 = 0ull;
        PAIR_LOOP
        {
            const long long me = s * P + q;
            const f2 m = (a0 ? 0x00000000ffffffffull : 0ull) | (a1 ? 0xffffffff00000000ull : 0ull);
            f2 nn = 0ull;
#pragma unroll
            for (int k = 0; k < 12; k++) {
                const C2 x = ld1(xv, cs, me, k), p = ld1(pv, cs, me, k);
                C2 xn = {ffma2(al, p.re, x.re), ffma2(al, p.im, x.im)};
                xn.re = blend(xn.re, x.re, m);
                xn.im = blend(xn.im, x.im, m);
                st1(xv, cs, me, k, xn);
                C2 r = ld1(rv, cs, me, k);
                const C2 w = ld1(wv, cs, me, k);
                r.re = ffma2(mal, w.re, r.re);
                r.im = ffma2(mal, w.im, r.im);
                st1(rv, cs, me, k, r);
                nn = ffma2(r.re, r.re, nn);
                nn = ffma2(r.im, r.im, nn);
            }
            sum0 = fadd2(sum0, nn);
        }
        add_lanes(acc[0], acc[1], sum0, a0, a1);
    }
    const int q = threadIdx.x % (nrhs / 2);
    if (!reduce_last<1, 2>(acc, c, partials, counter, nrhs / 2)) return;
    finish_cg_update(st[2 * q], acc[0], max_iter);
    finish_cg_update(st[2 * q + 1], acc[1], max_iter);
}

// ---- GCR (the Krylov part of SAP+GCR): per-RHS dot products into device
// arrays, and updates with per-RHS coefficients read from them ----

// out[r] = <a, b> = sum conj(a) b (complex) per RHS
__global__ void __launch_bounds__(kMaxBlock)
k32_dotv(Cfg c, const void *av, const void *bv, long long Vh, int nrhs, const RhsState *st,
         double2 *out, double *partials, unsigned int *counter)
{
    double acc[4] = {0, 0, 0, 0};
    {
        f2 sum0 = 0ull, sum1 = 0ull;
        PAIR_LOOP
        {
            const long long me = s * P + q;
            f2 re = 0ull, im = 0ull;
#pragma unroll
            for (int k = 0; k < 12; k++) {
                const C2 x = ld1(av, cs, me, k), y = ld1(bv, cs, me, k);
                re = ffma2(x.re, y.re, re);
                re = ffma2(x.im, y.im, re);
                im = ffma2(x.re, y.im, im);
                im = ffma2(fneg2(x.im), y.re, im);
            }
            sum0 = fadd2(sum0, re);
            sum1 = fadd2(sum1, im);
        }
        add_lanes(acc[0], acc[2], sum0, a0, a1);
        add_lanes(acc[1], acc[3], sum1, a0, a1);
    }
    const int q = threadIdx.x % (nrhs / 2);
    if (!reduce_last<2, 2>(acc, c, partials, counter, nrhs / 2)) return;
    out[2 * q] = make_double2(acc[0], acc[1]);
    out[2 * q + 1] = make_double2(acc[2], acc[3]);
}

// out[r] = |a|^2 per RHS
__global__ void __launch_bounds__(kMaxBlock)
k32_norm2v(Cfg c, const void *av, long long Vh, int nrhs, const RhsState *st, double *out,
           double *partials, unsigned int *counter)
{
    double acc[2] = {0, 0};
    {
        f2 sum0 = 0ull;
        PAIR_LOOP
        {
            const long long me = s * P + q;
            f2 nn = 0ull;
#pragma unroll
            for (int k = 0; k < 12; k++) {
                const C2 x = ld1(av, cs, me, k);
                nn = ffma2(x.re, x.re, nn);
                nn = ffma2(x.im, x.im, nn);
            }
            sum0 = fadd2(sum0, nn);
        }
        add_lanes(acc[0], acc[1], sum0, a0, a1);
    }
    const int q = threadIdx.x % (nrhs / 2);
    if (!reduce_last<1, 2>(acc, c, partials, counter, nrhs / 2)) return;
    out[2 * q] = acc[0];
    out[2 * q + 1] = acc[1];
}

__device__ __forceinline__ C2 coef_lanes(const double2 *cf, int q, double sign)
{
    const double2 c0 = cf[2 * q], c1 = cf[2 * q + 1];
    return {pk((float)(sign * c0.x), (float)(sign * c1.x)), pk((float)(sign * c0.y), (float)(sign * c1.y))};
}

// w -= c wi, z -= c zi (modified Gram-Schmidt step, c per RHS)
__global__ void __launch_bounds__(kMaxBlock)
k32_mgs(Cfg c, void *wv, void *zv, const void *wiv, const void *ziv, long long Vh, int nrhs,
        const RhsState *st, const double2 *cf)
{
    const int qq = threadIdx.x % (nrhs / 2);
    const C2 mc = coef_lanes(cf, qq, -1.0);
    PAIR_LOOP
    {
        const long long me = s * P + q;
#pragma unroll
        for (int k = 0; k < 12; k++) {
            st1(wv, cs, me, k, c2_lanefma(mc, ld1(wiv, cs, me, k), ld1(wv, cs, me, k)));
            st1(zv, cs, me, k, c2_lanefma(mc, ld1(ziv, cs, me, k), ld1(zv, cs, me, k)));
        }
    }
}

// w /= |w|, z /= |w| (nrm = |w|^2 per RHS)
__global__ void __launch_bounds__(kMaxBlock)
k32_normalise(Cfg c, void *wv, void *zv, long long Vh, int nrhs, const RhsState *st,
              const double *nrm)
{
    const int qq = threadIdx.x % (nrhs / 2);
    const double n0 = nrm[2 * qq], n1 = nrm[2 * qq + 1];
    // a vanishing direction (|w|^2 below FP32 range) is dropped rather than
    // scaled to overflow
    const f2 sc = pk(n0 > 1e-60 ? (float)(1.0 / sqrt(n0)) : 0.f, n1 > 1e-60 ? (float)(1.0 / sqrt(n1)) : 0.f);
    PAIR_LOOP
    {
        const long long me = s * P + q;
#pragma unroll
        for (int k = 0; k < 12; k++) {
            const C2 w = ld1(wv, cs, me, k), z = ld1(zv, cs, me, k);
            st1(wv, cs, me, k, {fmul2(sc, w.re), fmul2(sc, w.im)});
            st1(zv, cs, me, k, {fmul2(sc, z.re), fmul2(sc, z.im)});
        }
    }
}

// x += a z (active lanes), r -= a w, |r|^2 -> convergence (a = <w, r> per RHS)
__global__ void __launch_bounds__(kMaxBlock)
k32_gcr_update(Cfg c, void *xv, void *rv, const void *zv, const void *wv, long long Vh, int nrhs,
               RhsState *st, const double2 *cf, int max_iter, double *partials,
               unsigned int *counter)
{
    double acc[2] = {0, 0};
    {
        const int qq = threadIdx.x % (nrhs / 2);
        const C2 a = coef_lanes(cf, qq, 1.0), ma = coef_lanes(cf, qq, -1.0);
        f2 sum0 = 0ull;
        PAIR_LOOP
        {
            const long long me = s * P + q;
            const f2 m = (a0 ? 0x00000000ffffffffull : 0ull) | (a1 ? 0xffffffff00000000ull : 0ull);
            f2 nn = 0ull;
#pragma unroll
            for (int k = 0; k < 12; k++) {
                const C2 x = ld1(xv, cs, me, k);
                C2 xn = c2_lanefma(a, ld1(zv, cs, me, k), x);
                xn.re = blend(xn.re, x.re, m);
                xn.im = blend(xn.im, x.im, m);
                st1(xv, cs, me, k, xn);
                const C2 r = c2_lanefma(ma, ld1(wv, cs, me, k), ld1(rv, cs, me, k));
                st1(rv, cs, me, k, r);
                nn = ffma2(r.re, r.re, nn);
                nn = ffma2(r.im, r.im, nn);
            }
            sum0 = fadd2(sum0, nn);
        }
        add_lanes(acc[0], acc[1], sum0, a0, a1);
    }
    const int q = threadIdx.x % (nrhs / 2);
    if (!reduce_last<1, 2>(acc, c, partials, counter, nrhs / 2)) return;
    finish_cg_update(st[2 * q], acc[0], max_iter);
    finish_cg_update(st[2 * q + 1], acc[1], max_iter);
}

// out = a - b (every pair)
__global__ void k32_xmy(const float4 *a, const float4 *b, float4 *out, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const ulonglong2 x = reinterpret_cast<const ulonglong2 *>(a)[i];
    const ulonglong2 y = reinterpret_cast<const ulonglong2 *>(b)[i];
    reinterpret_cast<ulonglong2 *>(out)[i] = make_ulonglong2(fsub2(x.x, y.x), fsub2(x.y, y.y));
}

// r32 (paired) = r64 / |r| per RHS (zero for inactive RHS)
__global__ void k32_from64(const double2 *r64, float4 *r32, long long Vh, int n, const RhsState *st)
{
    const int P = n / 2;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= Vh * P) return;
    const long long s = gid / P;
    const int q = (int)(gid - s * P);
    const double i0 = st[2 * q].active ? 1.0 / st[2 * q].scale : 0.0;
    const double i1 = st[2 * q + 1].active ? 1.0 / st[2 * q + 1].scale : 0.0;
#pragma unroll
    for (int k = 0; k < 12; k++) {
        const long long b64 = ((long long)k * Vh + s) * n + 2 * q;
        const double2 u = r64[b64], v = r64[b64 + 1];
        r32[((long long)k * Vh + s) * P + q] =
            make_float4((float)(u.x * i0), (float)(v.x * i1), (float)(u.y * i0), (float)(v.y * i1));
    }
}

// x64 += |r| e32 per active RHS
__global__ void k32_acc64(double2 *x64, const float4 *e32, long long Vh, int n, const RhsState *st)
{
    const int P = n / 2;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= Vh * P) return;
    const long long s = gid / P;
    const int q = (int)(gid - s * P);
    // refined RHS take blas_acc_f32_ratio instead
    const bool a0 = st[2 * q].active != 0 && !st[2 * q].refine;
    const bool a1 = st[2 * q + 1].active != 0 && !st[2 * q + 1].refine;
    if (!a0 && !a1) return;
    const double s0 = st[2 * q].scale, s1 = st[2 * q + 1].scale;
#pragma unroll
    for (int k = 0; k < 12; k++) {
        const float4 e = e32[((long long)k * Vh + s) * P + q];
        const long long b64 = ((long long)k * Vh + s) * n + 2 * q;
        if (a0) {
            double2 x = x64[b64];
            x.x = fmx(s0, (double)e.x, x.x);
            x.y = fmx(s0, (double)e.z, x.y);
            x64[b64] = x;
        }
        if (a1) {
            double2 x = x64[b64 + 1];
            x.x = fmx(s1, (double)e.y, x.x);
            x.y = fmx(s1, (double)e.w, x.y);
            x64[b64 + 1] = x;
        }
    }
}

inline unsigned blocks_for(long long n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

cudaError_t blas32_init(BlasCtx &bc, const void *b, void *r, void *rh, long long Vh, int nrhs,
                        RhsState *st, cudaStream_t s, void *p)
{
    if (nrhs % 2) return cudaErrorInvalidValue;
    const Cfg c = cfg_wave(bc, k32_init, Vh, nrhs / 2);
    k32_init<<<c.grid, c.block, 0, s>>>(c, b, r, rh, p, Vh, nrhs, st, bc.partials, bc.counter);
    return cudaGetLastError();
}

cudaError_t blas32_s_dots(BlasCtx &bc, const void *r, const void *v, void *sv, const void *rh,
                          const void *rh2, long long Vh, int nrhs, RhsState *st, cudaStream_t s)
{
    if (nrhs % 2) return cudaErrorInvalidValue;
    const Cfg c = cfg_wave(bc, k32_s_dots, Vh, nrhs / 2);
    k32_s_dots<<<c.grid, c.block, 0, s>>>(c, r, v, sv, rh, rh2, Vh, nrhs, st, bc.partials, bc.counter);
    return cudaGetLastError();
}

cudaError_t blas32_omega_dots(BlasCtx &bc, const void *dots, long long Vh, int nrhs, RhsState *st,
                              cudaStream_t s)
{
    if (nrhs % 2) return cudaErrorInvalidValue;
    const Cfg c = cfg_wave(bc, k32_omega_dots, Vh, nrhs / 2);
    k32_omega_dots<<<c.grid, c.block, 0, s>>>(c, dots, Vh, nrhs, st, bc.partials, bc.counter);
    return cudaGetLastError();
}

cudaError_t blas32_update_pa(BlasCtx &bc, void *x, void *r, void *p, const void *sv, const void *t,
                             const void *v, const void *rh2, long long Vh, int nrhs, RhsState *st,
                             int max_iter, cudaStream_t s)
{
    if (nrhs % 2) return cudaErrorInvalidValue;
    const Cfg c = cfg_wave(bc, k32_update_pa, Vh, nrhs / 2);
    k32_update_pa<<<c.grid, c.block, 0, s>>>(c, x, r, p, sv, t, v, rh2, Vh, nrhs, st, max_iter,
                                             bc.partials, bc.counter);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return blas_count_active(bc, st, nrhs, s);
}

cudaError_t blas32_alpha(BlasCtx &bc, const void *rh, const void *v, long long Vh, int nrhs,
                         RhsState *st, cudaStream_t s)
{
    if (nrhs % 2) return cudaErrorInvalidValue;
    const Cfg c = cfg_wave(bc, k32_alpha, Vh, nrhs / 2);
    k32_alpha<<<c.grid, c.block, 0, s>>>(c, rh, v, Vh, nrhs, st, bc.partials, bc.counter);
    return cudaGetLastError();
}

cudaError_t blas32_cg_gamma(BlasCtx &bc, const void *z, long long Vh, int nrhs, RhsState *st,
                            int first, cudaStream_t s)
{
    if (nrhs % 2) return cudaErrorInvalidValue;
    const Cfg c = cfg_wave(bc, k32_cg_gamma, Vh, nrhs / 2);
    k32_cg_gamma<<<c.grid, c.block, 0, s>>>(c, z, Vh, nrhs, st, first, bc.partials, bc.counter);
    return cudaGetLastError();
}

cudaError_t blas32_cg_p(BlasCtx &bc, const void *z, void *p, long long Vh, int nrhs,
                        const RhsState *st, cudaStream_t s)
{
    if (nrhs % 2) return cudaErrorInvalidValue;
    const Cfg c = cfg_wave(bc, k32_cg_p, Vh, nrhs / 2);
    k32_cg_p<<<c.grid, c.block, 0, s>>>(c, z, p, Vh, nrhs, st);
    return cudaGetLastError();
}

cudaError_t blas32_cg_alpha(BlasCtx &bc, const void *w, long long Vh, int nrhs, RhsState *st,
                            cudaStream_t s)
{
    if (nrhs % 2) return cudaErrorInvalidValue;
    const Cfg c = cfg_wave(bc, k32_cg_alpha, Vh, nrhs / 2);
    k32_cg_alpha<<<c.grid, c.block, 0, s>>>(c, w, Vh, nrhs, st, bc.partials, bc.counter);
    return cudaGetLastError();
}

cudaError_t blas32_cg_update(BlasCtx &bc, void *x, void *r, const void *p, const void *w,
                             long long Vh, int nrhs, RhsState *st, int max_iter, cudaStream_t s)
{
    if (nrhs % 2) return cudaErrorInvalidValue;
    const Cfg c = cfg_wave(bc, k32_cg_update, Vh, nrhs / 2);
    k32_cg_update<<<c.grid, c.block, 0, s>>>(c, x, r, p, w, Vh, nrhs, st, max_iter, bc.partials,
                                             bc.counter);
    return cudaGetLastError();
}

cudaError_t blas32_dotv(BlasCtx &bc, const void *a, const void *b, long long Vh, int nrhs,
                        const RhsState *st, double2 *out, cudaStream_t s)
{
    if (nrhs % 2) return cudaErrorInvalidValue;
    const Cfg c = cfg_wave(bc, k32_dotv, Vh, nrhs / 2);
    k32_dotv<<<c.grid, c.block, 0, s>>>(c, a, b, Vh, nrhs, st, out, bc.partials, bc.counter);
    return cudaGetLastError();
}

cudaError_t blas32_norm2v(BlasCtx &bc, const void *a, long long Vh, int nrhs, const RhsState *st,
                          double *out, cudaStream_t s)
{
    if (nrhs % 2) return cudaErrorInvalidValue;
    const Cfg c = cfg_wave(bc, k32_norm2v, Vh, nrhs / 2);
    k32_norm2v<<<c.grid, c.block, 0, s>>>(c, a, Vh, nrhs, st, out, bc.partials, bc.counter);
    return cudaGetLastError();
}

cudaError_t blas32_mgs(BlasCtx &bc, void *w, void *z, const void *wi, const void *zi, long long Vh,
                       int nrhs, const RhsState *st, const double2 *cf, cudaStream_t s)
{
    if (nrhs % 2) return cudaErrorInvalidValue;
    const Cfg c = cfg_wave(bc, k32_mgs, Vh, nrhs / 2);
    k32_mgs<<<c.grid, c.block, 0, s>>>(c, w, z, wi, zi, Vh, nrhs, st, cf);
    return cudaGetLastError();
}

cudaError_t blas32_normalise(BlasCtx &bc, void *w, void *z, long long Vh, int nrhs,
                             const RhsState *st, const double *nrm, cudaStream_t s)
{
    if (nrhs % 2) return cudaErrorInvalidValue;
    const Cfg c = cfg_wave(bc, k32_normalise, Vh, nrhs / 2);
    k32_normalise<<<c.grid, c.block, 0, s>>>(c, w, z, Vh, nrhs, st, nrm);
    return cudaGetLastError();
}

cudaError_t blas32_gcr_update(BlasCtx &bc, void *x, void *r, const void *z, const void *w,
                              long long Vh, int nrhs, RhsState *st, const double2 *cf, int max_iter,
                              cudaStream_t s)
{
    if (nrhs % 2) return cudaErrorInvalidValue;
    const Cfg c = cfg_wave(bc, k32_gcr_update, Vh, nrhs / 2);
    k32_gcr_update<<<c.grid, c.block, 0, s>>>(c, x, r, z, w, Vh, nrhs, st, cf, max_iter, bc.partials,
                                              bc.counter);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return blas_count_active(bc, st, nrhs, s);
}

cudaError_t blas32_xmy(const void *a, const void *b, void *out, long long Vh, int nrhs, cudaStream_t s)
{
    const long long n = Vh * 12 * (nrhs / 2);
    k32_xmy<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(static_cast<const float4 *>(a),
                                                         static_cast<const float4 *>(b),
                                                         static_cast<float4 *>(out), n);
    return cudaGetLastError();
}

cudaError_t blas_to_f32_scaled(const double2 *r64, float4 *r32, long long Vh, int nrhs,
                               const RhsState *st, cudaStream_t s)
{
    if (nrhs % 2) return cudaErrorInvalidValue;
    k32_from64<<<blocks_for(Vh * (nrhs / 2), 256), 256, 0, s>>>(r64, r32, Vh, nrhs, st);
    return cudaGetLastError();
}

cudaError_t blas_acc_f32(double2 *x64, const float4 *e32, long long Vh, int nrhs,
                         const RhsState *st, cudaStream_t s)
{
    if (nrhs % 2) return cudaErrorInvalidValue;
    k32_acc64<<<blocks_for(Vh * (nrhs / 2), 256), 256, 0, s>>>(x64, e32, Vh, nrhs, st);
    return cudaGetLastError();
}

}  // namespace dp
