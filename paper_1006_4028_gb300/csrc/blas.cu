// BLAS-1 updates fused with the reductions of BiCGStab, per right-hand side,
// for the even-odd Schur system (FP64 vectors), and the FP64 outer-loop
// helpers.  The FP32 inner-solver kernels on the paired layout are in
// blas32.cu; the launchers below route by precision.
//
// Thread layout: a block is `lanes` sites x n RHS, thread t = lane*n + rhs, so
// every component load of the [component][site][rhs] layout is one
// contiguous run and each thread keeps one RHS for its whole grid-stride
// loop.  Reductions are deterministic (reduce.cuh): per-thread FP64 partial
// sums, a fixed tree over the lanes of a block, per-block partials in global
// scratch, and the last block to finish sums the block partials in a fixed
// order and applies the scalar recurrences (alpha, omega, rho, beta) per RHS
// on the device, so the iteration loop needs no host round trip.
#include "cplx.cuh"
#include "dp_internal.h"
#include "reduce.cuh"

namespace dp {
namespace {

struct V12 {
    Cx<double> c[12];
};

__device__ __forceinline__ V12 ld(const void *base, long long cs, long long me)
{
    V12 v;
    load_spinor(static_cast<const double2 *>(base) + me, cs, v.c);
    return v;
}
__device__ __forceinline__ void stv(void *base, long long cs, long long me, const V12 &v)
{
    store_spinor(static_cast<double2 *>(base) + me, cs, v.c);
}

// <a, b> = sum conj(a) b over one spinor
__device__ __forceinline__ Cx<double> sdot(const V12 &a, const V12 &b)
{
    Cx<double> s = {0.0, 0.0};
#pragma unroll
    for (int k = 0; k < 12; k++) s = cjfma(a.c[k], b.c[k], s);
    return s;
}
__device__ __forceinline__ double snorm(const V12 &a)
{
    double s = 0;
#pragma unroll
    for (int k = 0; k < 12; k++) {
        s = fmx(a.c[k].re, a.c[k].re, s);
        s = fmx(a.c[k].im, a.c[k].im, s);
    }
    return s;
}

#define SITE_LOOP                                                          \
    const int n = nrhs;                                                    \
    const int r = threadIdx.x % n, lane = threadIdx.x / n;                 \
    const long long cs = Vh * n;                                           \
    const bool act = st[r].active != 0;                                    \
    for (long long s = (long long)blockIdx.x * c.lanes + lane; act && s < Vh; \
         s += (long long)gridDim.x * c.lanes)

// p = r + beta (p - omega v); first iteration p = r
__global__ void __launch_bounds__(kMaxBlock) k_bicg_p(Cfg c, const void *rv, void *pv, const void *vv, long long Vh, int nrhs,
                         const RhsState *st, int first)
{
    SITE_LOOP
    {
        const long long me = s * n + r;
        V12 rr = ld(rv, cs, me);
        if (first) {
            stv(pv, cs, me, rr);
            continue;
        }
        const Cx<double> be = {st[r].beta.x, st[r].beta.y};
        const Cx<double> om = {st[r].omega.x, st[r].omega.y};
        V12 p = ld(pv, cs, me), v = ld(vv, cs, me);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            Cx<double> d = p.c[k] - cmul(om, v.c[k]);
            p.c[k] = cfma(be, d, rr.c[k]);
        }
        stv(pv, cs, me, p);
    }
}

// alpha = rho / <rhat, v>
__global__ void __launch_bounds__(kMaxBlock) k_bicg_alpha(Cfg c, const void *rh, const void *vv, long long Vh, int nrhs,
                             RhsState *st, double *partials, unsigned int *counter)
{
    double acc[2] = {0, 0};
    {
        SITE_LOOP
        {
            const long long me = s * n + r;
            Cx<double> d = sdot(ld(rh, cs, me), ld(vv, cs, me));
            acc[0] += d.re;
            acc[1] += d.im;
        }
    }
    const int r = threadIdx.x % nrhs;
    if (!reduce_last<2, 1>(acc, c, partials, counter, nrhs)) return;
    finish_alpha(st[r], acc[0], acc[1]);
}

// s = r - alpha v
__global__ void __launch_bounds__(kMaxBlock) k_bicg_s(Cfg c, const void *rv, const void *vv, void *sv, long long Vh, int nrhs,
                         const RhsState *st)
{
    SITE_LOOP
    {
        const long long me = s * n + r;
        const Cx<double> al = {-st[r].alpha.x, -st[r].alpha.y};
        V12 a = ld(rv, cs, me), v = ld(vv, cs, me);
#pragma unroll
        for (int k = 0; k < 12; k++) a.c[k] = cfma(al, v.c[k], a.c[k]);
        stv(sv, cs, me, a);
    }
}

// omega = <t, s> / <t, t>
__global__ void __launch_bounds__(kMaxBlock) k_bicg_omega(Cfg c, const void *tv, const void *sv, long long Vh, int nrhs,
                             RhsState *st, double *partials, unsigned int *counter)
{
    double acc[3] = {0, 0, 0};
    {
        SITE_LOOP
        {
            const long long me = s * n + r;
            V12 t = ld(tv, cs, me), sx = ld(sv, cs, me);
            Cx<double> d = sdot(t, sx);
            acc[0] += d.re;
            acc[1] += d.im;
            acc[2] += snorm(t);
        }
    }
    const int r = threadIdx.x % nrhs;
    if (!reduce_last<3, 1>(acc, c, partials, counter, nrhs)) return;
    finish_omega(st[r], acc[0], acc[1], acc[2]);
}

// x += alpha p + omega s; r = s - omega t; rho' = <rhat, r>; |r|^2
__global__ void __launch_bounds__(kMaxBlock) k_bicg_update(Cfg c, void *xv, void *rv, const void *pv, const void *sv,
                              const void *tv, const void *rh, long long Vh, int nrhs,
                              RhsState *st, int max_iter, double *partials, unsigned int *counter)
{
    double acc[3] = {0, 0, 0};
    {
        SITE_LOOP
        {
            const long long me = s * n + r;
            const Cx<double> al = {st[r].alpha.x, st[r].alpha.y};
            const Cx<double> om = {st[r].omega.x, st[r].omega.y};
            const Cx<double> mom = {-om.re, -om.im};
            V12 x = ld(xv, cs, me), p = ld(pv, cs, me), sx = ld(sv, cs, me);
#pragma unroll
            for (int k = 0; k < 12; k++) x.c[k] = cfma(om, sx.c[k], cfma(al, p.c[k], x.c[k]));
            stv(xv, cs, me, x);
            V12 t = ld(tv, cs, me);
#pragma unroll
            for (int k = 0; k < 12; k++) sx.c[k] = cfma(mom, t.c[k], sx.c[k]);
            stv(rv, cs, me, sx);
            Cx<double> d = sdot(ld(rh, cs, me), sx);
            acc[0] += d.re;
            acc[1] += d.im;
            acc[2] += snorm(sx);
        }
    }
    const int r = threadIdx.x % nrhs;
    if (!reduce_last<3, 1>(acc, c, partials, counter, nrhs)) return;
    finish_update(st[r], acc[0], acc[1], acc[2], max_iter);
}

// inner init: r = b, rhat = r (b may alias rhat); rho = |r|^2, tol2 *= |r|^2
__global__ void __launch_bounds__(kMaxBlock) k_bicg_init(Cfg c, const void *bv, void *rv, void *rh, long long Vh, int nrhs,
                            RhsState *st, double *partials, unsigned int *counter)
{
    double acc[1] = {0};
    {
        SITE_LOOP
        {
            const long long me = s * n + r;
            V12 b = ld(bv, cs, me);
            stv(rv, cs, me, b);
            stv(rh, cs, me, b);
            acc[0] += snorm(b);
        }
    }
    const int r = threadIdx.x % nrhs;
    if (!reduce_last<1, 1>(acc, c, partials, counter, nrhs)) return;
    finish_init(st[r], acc[0]);
}

// ---- CGNE on the normal equations (real per-RHS scalars) ----

// rho' = |z|^2, beta = rho'/rho
__global__ void __launch_bounds__(kMaxBlock) k_cg_gamma(Cfg c, const void *zv, long long Vh, int nrhs,
                                                        RhsState *st, int first, double *partials,
                                                        unsigned int *counter)
{
    double acc[1] = {0};
    {
        SITE_LOOP acc[0] += snorm(ld(zv, cs, s * n + r));
    }
    const int r = threadIdx.x % nrhs;
    if (!reduce_last<1, 1>(acc, c, partials, counter, nrhs)) return;
    finish_cg_gamma(st[r], acc[0], first);
}

// p = z + beta p
__global__ void __launch_bounds__(kMaxBlock) k_cg_p(Cfg c, const void *zv, void *pv, long long Vh, int nrhs,
                                                    const RhsState *st)
{
    SITE_LOOP
    {
        const long long me = s * n + r;
        const double be = st[r].beta.x;
        const V12 z = ld(zv, cs, me);
        V12 p = ld(pv, cs, me);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            p.c[k].re = fmx(be, p.c[k].re, z.c[k].re);
            p.c[k].im = fmx(be, p.c[k].im, z.c[k].im);
        }
        stv(pv, cs, me, p);
    }
}

// alpha = rho / |w|^2
__global__ void __launch_bounds__(kMaxBlock) k_cg_alpha(Cfg c, const void *wv, long long Vh, int nrhs,
                                                        RhsState *st, double *partials,
                                                        unsigned int *counter)
{
    double acc[1] = {0};
    {
        SITE_LOOP acc[0] += snorm(ld(wv, cs, s * n + r));
    }
    const int r = threadIdx.x % nrhs;
    if (!reduce_last<1, 1>(acc, c, partials, counter, nrhs)) return;
    finish_cg_alpha(st[r], acc[0]);
}

// x += alpha p, r -= alpha w, |r|^2
__global__ void __launch_bounds__(kMaxBlock) k_cg_update(Cfg c, void *xv, void *rv, const void *pv,
                                                         const void *wv, long long Vh, int nrhs,
                                                         RhsState *st, int max_iter, double *partials,
                                                         unsigned int *counter)
{
    double acc[1] = {0};
    {
        SITE_LOOP
        {
            const long long me = s * n + r;
            const double al = st[r].alpha.x;
            V12 x = ld(xv, cs, me);
            const V12 p = ld(pv, cs, me);
#pragma unroll
            for (int k = 0; k < 12; k++) {
                x.c[k].re = fmx(al, p.c[k].re, x.c[k].re);
                x.c[k].im = fmx(al, p.c[k].im, x.c[k].im);
            }
            stv(xv, cs, me, x);
            V12 rr = ld(rv, cs, me);
            const V12 w = ld(wv, cs, me);
#pragma unroll
            for (int k = 0; k < 12; k++) {
                rr.c[k].re = fmx(-al, w.c[k].re, rr.c[k].re);
                rr.c[k].im = fmx(-al, w.c[k].im, rr.c[k].im);
            }
            stv(rv, cs, me, rr);
            acc[0] += snorm(rr);
        }
    }
    const int r = threadIdx.x % nrhs;
    if (!reduce_last<1, 1>(acc, c, partials, counter, nrhs)) return;
    finish_cg_update(st[r], acc[0], max_iter);
}

// FP64 outer residual r = b - y and |r|^2; an RHS flagged `fresh` (x = 0)
// takes r = b and also records |b|^2, turning tol2 = r_target^2 into the
// absolute threshold r_target^2 |b|^2
__global__ void __launch_bounds__(kMaxBlock) k_residual64(Cfg c, const double2 *b, const double2 *y, double2 *rv,
                             long long Vh, int nrhs, RhsState *st, const int *mask,
                             double *partials, unsigned int *counter)
{
    double acc[2] = {0, 0};
    const bool use = !mask || mask[threadIdx.x % nrhs];
    {
        SITE_LOOP
        {
            if (!use) break;
            const long long me = s * n + r;
            V12 bb = ld(b, cs, me);
            if (st[r].fresh) {
                acc[1] += snorm(bb);
            } else {
                V12 yy = ld(y, cs, me);
#pragma unroll
                for (int k = 0; k < 12; k++) bb.c[k] = bb.c[k] - yy.c[k];
            }
            stv(rv, cs, me, bb);
            acc[0] += snorm(bb);
        }
    }
    const int r = threadIdx.x % nrhs;
    if (!reduce_last<2, 1>(acc, c, partials, counter, nrhs)) return;
    RhsState &S = st[r];
    if (!S.active || !use) return;
    if (S.fresh) {
        S.bb = acc[1];
        S.tol2 = S.tol2 * acc[1];
        S.fresh = 0;
    }
    S.rr = acc[0];
    S.scale = sqrt(acc[0]);
    if (!isfinite(acc[0])) {
        S.status = 3;
        S.active = 0;
    } else if (!S.refine && acc[0] <= S.tol2) {  // a refined RHS stops on its slices
        S.status = 1;
        S.active = 0;
    }
}

__global__ void __launch_bounds__(kMaxBlock) k_norm2(Cfg c, const double2 *v, long long Vh, int nrhs, double *out,
                        double *partials, unsigned int *counter)
{
    double acc[1] = {0};
    const int n = nrhs;
    const int r = threadIdx.x % n, lane = threadIdx.x / n;
    const long long cs = Vh * n;
    for (long long s = (long long)blockIdx.x * c.lanes + lane; s < Vh; s += (long long)gridDim.x * c.lanes)
        acc[0] += snorm(ld(v, cs, s * n + r));
    if (!reduce_last<1, 1>(acc, c, partials, counter, nrhs)) return;
    out[r] = acc[0];
}

__global__ void __launch_bounds__(kMaxBlock) k_diff_norm2(Cfg c, const double2 *a, const double2 *b, long long Vh, int nrhs,
                             double *out, double *partials, unsigned int *counter)
{
    double acc[1] = {0};
    const int n = nrhs;
    const int r = threadIdx.x % n, lane = threadIdx.x / n;
    const long long cs = Vh * n;
    for (long long s = (long long)blockIdx.x * c.lanes + lane; s < Vh; s += (long long)gridDim.x * c.lanes) {
        const long long me = s * n + r;
        V12 x = ld(a, cs, me), y = ld(b, cs, me);
#pragma unroll
        for (int k = 0; k < 12; k++) x.c[k] = x.c[k] - y.c[k];
        acc[0] += snorm(x);
    }
    if (!reduce_last<1, 1>(acc, c, partials, counter, nrhs)) return;
    out[r] = acc[0];
}

__global__ void k_count_active(const RhsState *st, int n, int *n_active)
{
    int c = 0;
    for (int r = 0; r < n; r++) c += st[r].active ? 1 : 0;
    *n_active = c;
}

// inner state from the outer one: same active set.  The outer threshold is
// tol2 = r^2 |b|^2: reducing |r| by 0.5 sqrt(tol2)/|r| already meets it, so
// the inner solve never asks for more than that (nor less than inner_tol)
__global__ void k_inner_setup(const RhsState *outer, RhsState *inner, int n, double inner_tol)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    RhsState S = {};
    S.active = outer[r].active;
    double tol = inner_tol;
    if (outer[r].refine) {
        // per-slice refinement: the round's reduction, set per job in tol2
        // (the global threshold does not apply to a refined RHS)
        const double want = sqrt(outer[r].tol2);
        if (want > tol) tol = want;
    } else if (outer[r].rr > 0) {
        const double want = 0.5 * sqrt(outer[r].tol2 / outer[r].rr);
        if (want > tol) tol = want;
    }
    if (tol > 0.5) tol = 0.5;
    S.tol2 = tol * tol;
    S.status = 0;
    inner[r] = S;
}

__global__ void k_scale64(const double2 *v, double2 *out, long long Vh, int n, const RhsState *st)
{
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= Vh * n) return;
    const int r = (int)(gid % n);
    const long long cs = Vh * n;
    const double inv = st[r].active ? 1.0 / st[r].scale : 0.0;
    V12 a = ld(v, cs, gid);
#pragma unroll
    for (int k = 0; k < 12; k++) a.c[k] = {a.c[k].re * inv, a.c[k].im * inv};
    stv(out, cs, gid, a);
}

__global__ void k_acc64(double2 *x64, const double2 *e64, long long Vh, int n, const RhsState *st)
{
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= Vh * n) return;
    const int r = (int)(gid % n);
    if (!st[r].active || st[r].refine) return;  // refined RHS: blas_acc64_ratio
    const long long cs = Vh * n;
    const double sc = st[r].scale;
    V12 x = ld(x64, cs, gid), e = ld(e64, cs, gid);
#pragma unroll
    for (int k = 0; k < 12; k++) {
        x.c[k].re = fmx(sc, e.c[k].re, x.c[k].re);
        x.c[k].im = fmx(sc, e.c[k].im, x.c[k].im);
    }
    stv(x64, cs, gid, x);
}

__global__ void k_sub64_masked(const double2 *a, const double2 *b, double2 *out, long long Vh, int n,
                               const int *mask)
{
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= Vh * n) return;
    if (!mask[gid % n]) return;
    const long long cs = Vh * n;
#pragma unroll
    for (int k = 0; k < 12; k++) {
        const double2 x = a[k * cs + gid], y = b[k * cs + gid];
        out[k * cs + gid] = make_double2(x.x - y.x, x.y - y.y);
    }
}

__global__ void k_zero_masked(double2 *v, long long Vh, int n, const int *mask)
{
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= Vh * n) return;
    if (!mask[gid % n]) return;
    const long long cs = Vh * n;
#pragma unroll
    for (int k = 0; k < 12; k++) v[k * cs + gid] = make_double2(0.0, 0.0);
}

inline unsigned blocks_for(long long n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

// ---- launchers ----------------------------------------------------------------

cudaError_t blas_zero(void *v, size_t bytes, cudaStream_t s) { return cudaMemsetAsync(v, 0, bytes, s); }

cudaError_t blas_count_active(BlasCtx &bc, const RhsState *st, int nrhs, cudaStream_t s)
{
    k_count_active<<<1, 1, 0, s>>>(st, nrhs, bc.n_active);
    return cudaGetLastError();
}

cudaError_t blas_bicg_init(BlasCtx &bc, int prec, const void *b, void *r, void *rhat, void *p,
                           void *v, void *x, long long Vh, int nrhs, RhsState *st, double tol,
                           cudaStream_t s)
{
    (void)tol;
    const size_t bytes = (size_t)Vh * nrhs * 24 * (prec == 0 ? 8 : 4);
    cudaMemsetAsync(p, 0, bytes, s);
    cudaMemsetAsync(v, 0, bytes, s);
    cudaMemsetAsync(x, 0, bytes, s);
    if (prec != 0) {
        cudaError_t e = blas32_init(bc, b, r, rhat, Vh, nrhs, st, s);
        if (e != cudaSuccess) return e;
    } else {
        const Cfg c = cfg_wave(bc, k_bicg_init, Vh, nrhs);
        k_bicg_init<<<c.grid, c.block, 0, s>>>(c, b, r, rhat, Vh, nrhs, st, bc.partials, bc.counter);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return blas_count_active(bc, st, nrhs, s);
}

cudaError_t blas_bicg_p(BlasCtx &bc, int prec, const void *r, void *p, const void *v,
                        long long Vh, int nrhs, const RhsState *st, int first, cudaStream_t s)
{
    if (prec != 0) return cudaErrorInvalidValue;  // FP32: the p update rides in blas32_update_pa
    const Cfg c = cfg_wave(bc, k_bicg_p, Vh, nrhs);
    k_bicg_p<<<c.grid, c.block, 0, s>>>(c, r, p, v, Vh, nrhs, st, first);
    return cudaGetLastError();
}

cudaError_t blas_bicg_alpha(BlasCtx &bc, int prec, const void *rhat, const void *v,
                            long long Vh, int nrhs, RhsState *st, cudaStream_t s)
{
    if (prec != 0) return blas32_alpha(bc, rhat, v, Vh, nrhs, st, s);
    const Cfg c = cfg_wave(bc, k_bicg_alpha, Vh, nrhs);
    k_bicg_alpha<<<c.grid, c.block, 0, s>>>(c, rhat, v, Vh, nrhs, st, bc.partials, bc.counter);
    return cudaGetLastError();
}

cudaError_t blas_bicg_s(BlasCtx &bc, int prec, const void *r, const void *v, void *sv,
                        long long Vh, int nrhs, const RhsState *st, cudaStream_t s)
{
    if (prec != 0) return cudaErrorInvalidValue;  // FP32: blas32_s_dots
    const Cfg c = cfg_wave(bc, k_bicg_s, Vh, nrhs);
    k_bicg_s<<<c.grid, c.block, 0, s>>>(c, r, v, sv, Vh, nrhs, st);
    return cudaGetLastError();
}

cudaError_t blas_bicg_omega(BlasCtx &bc, int prec, const void *t, const void *sv,
                            long long Vh, int nrhs, RhsState *st, cudaStream_t s)
{
    if (prec != 0) return cudaErrorInvalidValue;  // FP32: blas32_omega_dots
    const Cfg c = cfg_wave(bc, k_bicg_omega, Vh, nrhs);
    k_bicg_omega<<<c.grid, c.block, 0, s>>>(c, t, sv, Vh, nrhs, st, bc.partials, bc.counter);
    return cudaGetLastError();
}

cudaError_t blas_bicg_update(BlasCtx &bc, int prec, void *x, void *r, const void *p,
                             const void *sv, const void *t, const void *rhat, long long Vh,
                             int nrhs, RhsState *st, int max_iter, cudaStream_t s)
{
    cudaError_t e;
    if (prec != 0) {
        return cudaErrorInvalidValue;  // FP32: blas32_update_pa
    } else {
        const Cfg c = cfg_wave(bc, k_bicg_update, Vh, nrhs);
        k_bicg_update<<<c.grid, c.block, 0, s>>>(c, x, r, p, sv, t, rhat, Vh, nrhs, st, max_iter,
                                                 bc.partials, bc.counter);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    return blas_count_active(bc, st, nrhs, s);
}

cudaError_t blas_cg_gamma(BlasCtx &bc, int prec, const void *z, long long Vh, int nrhs,
                          RhsState *st, int first, cudaStream_t s)
{
    if (prec != 0) return blas32_cg_gamma(bc, z, Vh, nrhs, st, first, s);
    const Cfg c = cfg_wave(bc, k_cg_gamma, Vh, nrhs);
    k_cg_gamma<<<c.grid, c.block, 0, s>>>(c, z, Vh, nrhs, st, first, bc.partials, bc.counter);
    return cudaGetLastError();
}

cudaError_t blas_cg_p(BlasCtx &bc, int prec, const void *z, void *p, long long Vh, int nrhs,
                      const RhsState *st, cudaStream_t s)
{
    if (prec != 0) return blas32_cg_p(bc, z, p, Vh, nrhs, st, s);
    const Cfg c = cfg_wave(bc, k_cg_p, Vh, nrhs);
    k_cg_p<<<c.grid, c.block, 0, s>>>(c, z, p, Vh, nrhs, st);
    return cudaGetLastError();
}

cudaError_t blas_cg_alpha(BlasCtx &bc, int prec, const void *w, long long Vh, int nrhs,
                          RhsState *st, cudaStream_t s)
{
    if (prec != 0) return blas32_cg_alpha(bc, w, Vh, nrhs, st, s);
    const Cfg c = cfg_wave(bc, k_cg_alpha, Vh, nrhs);
    k_cg_alpha<<<c.grid, c.block, 0, s>>>(c, w, Vh, nrhs, st, bc.partials, bc.counter);
    return cudaGetLastError();
}

cudaError_t blas_cg_update(BlasCtx &bc, int prec, void *x, void *r, const void *p, const void *w,
                           long long Vh, int nrhs, RhsState *st, int max_iter, cudaStream_t s)
{
    cudaError_t e;
    if (prec != 0) {
        e = blas32_cg_update(bc, x, r, p, w, Vh, nrhs, st, max_iter, s);
    } else {
        const Cfg c = cfg_wave(bc, k_cg_update, Vh, nrhs);
        k_cg_update<<<c.grid, c.block, 0, s>>>(c, x, r, p, w, Vh, nrhs, st, max_iter, bc.partials,
                                               bc.counter);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    return blas_count_active(bc, st, nrhs, s);
}

cudaError_t blas_residual64(BlasCtx &bc, const double2 *b, const double2 *y, double2 *r,
                            long long Vh, int nrhs, RhsState *st, const int *mask, cudaStream_t s)
{
    const Cfg c = cfg_wave(bc, k_residual64, Vh, nrhs);
    k_residual64<<<c.grid, c.block, 0, s>>>(c, b, y, r, Vh, nrhs, st, mask, bc.partials, bc.counter);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return blas_count_active(bc, st, nrhs, s);
}

cudaError_t blas_norm2(BlasCtx &bc, int prec, const void *v, long long Vh, int nrhs,
                       double *out_dev, cudaStream_t s)
{
    if (prec != 0) return cudaErrorInvalidValue;  // FP64 vectors only
    const Cfg c = cfg_wave(bc, k_norm2, Vh, nrhs);
    k_norm2<<<c.grid, c.block, 0, s>>>(c, (const double2 *)v, Vh, nrhs, out_dev, bc.partials, bc.counter);
    return cudaGetLastError();
}

cudaError_t blas_diff_norm2(BlasCtx &bc, const double2 *a, const double2 *b, long long Vh,
                            int nrhs, double *out_dev, cudaStream_t s)
{
    const Cfg c = cfg_wave(bc, k_diff_norm2, Vh, nrhs);
    k_diff_norm2<<<c.grid, c.block, 0, s>>>(c, a, b, Vh, nrhs, out_dev, bc.partials, bc.counter);
    return cudaGetLastError();
}

cudaError_t blas_inner_setup(const RhsState *outer, RhsState *inner, int nrhs, double inner_tol,
                             double target, cudaStream_t s)
{
    (void)target;
    k_inner_setup<<<1, 64, 0, s>>>(outer, inner, nrhs, inner_tol);
    return cudaGetLastError();
}

cudaError_t blas_scale64(const double2 *v, double2 *out, long long Vh, int nrhs,
                         const RhsState *st, cudaStream_t s)
{
    k_scale64<<<blocks_for(Vh * nrhs, 256), 256, 0, s>>>(v, out, Vh, nrhs, st);
    return cudaGetLastError();
}

cudaError_t blas_acc64(double2 *x64, const double2 *e64, long long Vh, int nrhs,
                       const RhsState *st, cudaStream_t s)
{
    k_acc64<<<blocks_for(Vh * nrhs, 256), 256, 0, s>>>(x64, e64, Vh, nrhs, st);
    return cudaGetLastError();
}

cudaError_t blas_sub64_masked(const double2 *a, const double2 *b, double2 *out, long long Vh,
                              int nrhs, const int *mask, cudaStream_t s)
{
    k_sub64_masked<<<blocks_for(Vh * nrhs, 256), 256, 0, s>>>(a, b, out, Vh, nrhs, mask);
    return cudaGetLastError();
}

cudaError_t blas_zero_masked(double2 *v, long long Vh, int nrhs, const int *mask, cudaStream_t s)
{
    k_zero_masked<<<blocks_for(Vh * nrhs, 256), 256, 0, s>>>(v, Vh, nrhs, mask);
    return cudaGetLastError();
}

}  // namespace dp
