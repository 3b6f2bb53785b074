// BLAS-1 updates fused with the reductions of BiCGStab, per right-hand side,
// for the even-odd Schur system, plus the FP64 outer-loop helpers.
//
// Thread layout: a block is `lanes` sites x n RHS, thread t = lane*n + rhs, so
// every chunk load of the [chunk][site][rhs] layout is one contiguous run and
// each thread keeps one RHS for its whole grid-stride loop.  Reductions are
// deterministic: per-thread FP64 partial sums (each spinor's 24 products are
// formed in the vector precision), a fixed tree over the lanes of a block,
// per-block partials in global scratch, and the last block to finish sums the
// block partials in a fixed order and applies the scalar recurrences (alpha,
// omega, rho, beta) per RHS on the device, so the iteration loop needs no
// host round trip.  Per-RHS results do not depend on the other RHS.
#include <algorithm>
#include <map>
#include <mutex>

#include "cplx.cuh"
#include "dp_internal.h"

namespace dp {
namespace {

constexpr int kMaxBlock = 512;

struct Cfg {
    int lanes, block, grid;
};

Cfg cfg_for(long long Vh, int n, int max_grid)
{
    Cfg c;
    c.lanes = 256;
    while (c.lanes * n > kMaxBlock && c.lanes > 1) c.lanes >>= 1;
    c.block = c.lanes * n;
    long long g = (Vh + c.lanes - 1) / c.lanes;
    if (g > max_grid) g = max_grid;
    if (g < 1) g = 1;
    c.grid = (int)g;
    return c;
}

template <typename R>
struct V12 {
    Cx<R> c[12];
};

template <typename R>
__device__ __forceinline__ V12<R> ld(const void *base, long long cs, long long me)
{
    V12<R> v;
    load_spinor(static_cast<const typename Chunk<R>::T *>(base) + me, cs, v.c);
    return v;
}
template <typename R>
__device__ __forceinline__ void stv(void *base, long long cs, long long me, const V12<R> &v)
{
    store_spinor(static_cast<typename Chunk<R>::T *>(base) + me, cs, v.c);
}

// <a, b> = sum conj(a) b over one spinor, formed in precision R
template <typename R>
__device__ __forceinline__ Cx<R> sdot(const V12<R> &a, const V12<R> &b)
{
    Cx<R> s = {R(0), R(0)};
#pragma unroll
    for (int k = 0; k < 12; k++) s = cjfma(a.c[k], b.c[k], s);
    return s;
}
template <typename R>
__device__ __forceinline__ R snorm(const V12<R> &a)
{
    R s = 0;
#pragma unroll
    for (int k = 0; k < 12; k++) {
        s = fmx(a.c[k].re, a.c[k].re, s);
        s = fmx(a.c[k].im, a.c[k].im, s);
    }
    return s;
}

__device__ __forceinline__ double2 zdiv(double2 a, double2 b)
{
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 zmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ bool zfinite(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// Block + grid reduction of NV doubles per RHS.  Every thread passes its
// partials in `v`; returns true in exactly one thread per RHS (lane 0 of the
// last block), with the totals in `v`.
template <int NV>
__device__ bool reduce_last(double v[NV], const Cfg c, double *partials, unsigned int *counter,
                            int n)
{
    __shared__ double sh[kMaxBlock * NV];
    __shared__ bool last;
    const int t = threadIdx.x, r = t % n, lane = t / n;
#pragma unroll
    for (int k = 0; k < NV; k++) sh[t * NV + k] = v[k];
    __syncthreads();
    for (int w = c.lanes / 2; w > 0; w >>= 1) {
        if (lane < w)
#pragma unroll
            for (int k = 0; k < NV; k++) sh[t * NV + k] += sh[(t + w * n) * NV + k];
        __syncthreads();
    }
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; k++) partials[((long long)blockIdx.x * kMaxRhs + r) * 4 + k] = sh[t * NV + k];
    __threadfence();
    __syncthreads();
    if (t == 0) last = (atomicAdd(counter, 1u) == (unsigned)(gridDim.x - 1));
    __syncthreads();
    if (!last) return false;
    __threadfence();
    // last block: lane l sums blocks l, l+lanes, ... in order, then a fixed tree
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) acc[k] = 0;
    for (int b = lane; b < (int)gridDim.x; b += c.lanes)
#pragma unroll
        for (int k = 0; k < NV; k++) acc[k] += __ldcg(partials + ((long long)b * kMaxRhs + r) * 4 + k);
#pragma unroll
    for (int k = 0; k < NV; k++) sh[t * NV + k] = acc[k];
    __syncthreads();
    for (int w = c.lanes / 2; w > 0; w >>= 1) {
        if (lane < w)
#pragma unroll
            for (int k = 0; k < NV; k++) sh[t * NV + k] += sh[(t + w * n) * NV + k];
        __syncthreads();
    }
    if (t == 0) *counter = 0u;
    if (lane != 0) return false;
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = sh[t * NV + k];
    return true;
}

#define SITE_LOOP                                                          \
    const int n = nrhs;                                                    \
    const int r = threadIdx.x % n, lane = threadIdx.x / n;                 \
    const long long cs = Vh * n;                                           \
    const bool act = st[r].active != 0;                                    \
    for (long long s = (long long)blockIdx.x * c.lanes + lane; act && s < Vh; \
         s += (long long)gridDim.x * c.lanes)

// p = r + beta (p - omega v); first iteration p = r
template <typename R>
__global__ void k_bicg_p(Cfg c, const void *rv, void *pv, const void *vv, long long Vh,
                         int nrhs, const RhsState *st, int first)
{
    SITE_LOOP
    {
        const long long me = s * n + r;
        V12<R> rr = ld<R>(rv, cs, me);
        if (first) {
            stv<R>(pv, cs, me, rr);
            continue;
        }
        const Cx<R> be = {(R)st[r].beta.x, (R)st[r].beta.y};
        const Cx<R> om = {(R)st[r].omega.x, (R)st[r].omega.y};
        V12<R> p = ld<R>(pv, cs, me), v = ld<R>(vv, cs, me);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            Cx<R> d = p.c[k] - cmul(om, v.c[k]);
            p.c[k] = cfma(be, d, rr.c[k]);
        }
        stv<R>(pv, cs, me, p);
    }
}

// alpha = rho / <rhat, v>
template <typename R>
__global__ void k_bicg_alpha(Cfg c, const void *rh, const void *vv, long long Vh, int nrhs,
                             RhsState *st, double *partials, unsigned int *counter)
{
    double acc[2] = {0, 0};
    {
        SITE_LOOP
        {
            const long long me = s * n + r;
            Cx<R> d = sdot(ld<R>(rh, cs, me), ld<R>(vv, cs, me));
            acc[0] += (double)d.re;
            acc[1] += (double)d.im;
        }
    }
    const int r = threadIdx.x % nrhs;
    if (!reduce_last<2>(acc, c, partials, counter, nrhs)) return;
    RhsState &S = st[r];
    if (!S.active) return;
    const double2 rv = make_double2(acc[0], acc[1]);
    if (!zfinite(rv)) {
        S.status = 3;
        S.active = 0;
        return;
    }
    if (rv.x == 0.0 && rv.y == 0.0) {
        S.status = 2;
        S.active = 0;
        return;
    }
    S.alpha = zdiv(S.rho, rv);
}

// s = r - alpha v
template <typename R>
__global__ void k_bicg_s(Cfg c, const void *rv, const void *vv, void *sv, long long Vh,
                         int nrhs, const RhsState *st)
{
    SITE_LOOP
    {
        const long long me = s * n + r;
        const Cx<R> al = {(R)-st[r].alpha.x, (R)-st[r].alpha.y};
        V12<R> a = ld<R>(rv, cs, me), v = ld<R>(vv, cs, me);
#pragma unroll
        for (int k = 0; k < 12; k++) a.c[k] = cfma(al, v.c[k], a.c[k]);
        stv<R>(sv, cs, me, a);
    }
}

// omega = <t, s> / <t, t>
template <typename R>
__global__ void k_bicg_omega(Cfg c, const void *tv, const void *sv, long long Vh, int nrhs,
                             RhsState *st, double *partials, unsigned int *counter)
{
    double acc[3] = {0, 0, 0};
    {
        SITE_LOOP
        {
            const long long me = s * n + r;
            V12<R> t = ld<R>(tv, cs, me), sx = ld<R>(sv, cs, me);
            Cx<R> d = sdot(t, sx);
            acc[0] += (double)d.re;
            acc[1] += (double)d.im;
            acc[2] += (double)snorm(t);
        }
    }
    const int r = threadIdx.x % nrhs;
    if (!reduce_last<3>(acc, c, partials, counter, nrhs)) return;
    RhsState &S = st[r];
    if (!S.active) return;
    if (!(isfinite(acc[0]) && isfinite(acc[1]) && isfinite(acc[2]))) {
        S.status = 3;
        S.active = 0;
        return;
    }
    S.omega = acc[2] > 0 ? make_double2(acc[0] / acc[2], acc[1] / acc[2]) : make_double2(0.0, 0.0);
}

// x += alpha p + omega s; r = s - omega t; rho' = <rhat, r>; |r|^2;
// beta = (rho'/rho)(alpha/omega); convergence and iteration cap
template <typename R>
__global__ void k_bicg_update(Cfg c, void *xv, void *rv, const void *pv, const void *sv,
                              const void *tv, const void *rh, long long Vh, int nrhs,
                              RhsState *st, int max_iter, double *partials,
                              unsigned int *counter, int *n_active)
{
    double acc[3] = {0, 0, 0};
    {
        SITE_LOOP
        {
            const long long me = s * n + r;
            const Cx<R> al = {(R)st[r].alpha.x, (R)st[r].alpha.y};
            const Cx<R> om = {(R)st[r].omega.x, (R)st[r].omega.y};
            const Cx<R> mom = {-om.re, -om.im};
            V12<R> x = ld<R>(xv, cs, me), p = ld<R>(pv, cs, me), sx = ld<R>(sv, cs, me);
#pragma unroll
            for (int k = 0; k < 12; k++) x.c[k] = cfma(om, sx.c[k], cfma(al, p.c[k], x.c[k]));
            stv<R>(xv, cs, me, x);
            V12<R> t = ld<R>(tv, cs, me);
#pragma unroll
            for (int k = 0; k < 12; k++) sx.c[k] = cfma(mom, t.c[k], sx.c[k]);
            stv<R>(rv, cs, me, sx);
            Cx<R> d = sdot(ld<R>(rh, cs, me), sx);
            acc[0] += (double)d.re;
            acc[1] += (double)d.im;
            acc[2] += (double)snorm(sx);
        }
    }
    const int r = threadIdx.x % nrhs;
    if (!reduce_last<3>(acc, c, partials, counter, nrhs)) return;
    RhsState &S = st[r];
    if (S.active) {
        S.iters++;
        const double2 rho_new = make_double2(acc[0], acc[1]);
        S.rr = acc[2];
        if (!(zfinite(rho_new) && isfinite(acc[2]))) {
            S.status = 3;
            S.active = 0;
        } else if (S.rr <= S.tol2) {
            S.status = 1;
            S.active = 0;
        } else if (S.iters >= max_iter) {
            S.status = 4;
            S.active = 0;
        } else if ((S.omega.x == 0.0 && S.omega.y == 0.0) || (rho_new.x == 0.0 && rho_new.y == 0.0)) {
            S.status = 2;
            S.active = 0;
        } else {
            S.beta = zmul(zdiv(rho_new, S.rho), zdiv(S.alpha, S.omega));
            S.rho = rho_new;
        }
    }
}

// inner init: r = b (normalised outer residual), rhat = r, p = v = x = 0 done by
// the caller via memset; rho = |r|^2, tol2 = tol^2 |r|^2
template <typename R>
__global__ void k_bicg_init(Cfg c, const void *bv, void *rv, void *rh, long long Vh, int nrhs,
                            RhsState *st, double *partials, unsigned int *counter)
{
    double acc[1] = {0};
    {
        SITE_LOOP
        {
            const long long me = s * n + r;
            V12<R> b = ld<R>(bv, cs, me);
            stv<R>(rv, cs, me, b);
            stv<R>(rh, cs, me, b);
            acc[0] += (double)snorm(b);
        }
    }
    const int r = threadIdx.x % nrhs;
    if (!reduce_last<1>(acc, c, partials, counter, nrhs)) return;
    RhsState &S = st[r];
    if (!S.active) return;
    S.rr = acc[0];
    S.bb = acc[0];
    S.tol2 = S.tol2 * acc[0];  // tol2 holds tol^2 on entry
    S.rho = make_double2(acc[0], 0.0);
    S.alpha = make_double2(1.0, 0.0);
    S.omega = make_double2(1.0, 0.0);
    S.beta = make_double2(0.0, 0.0);
    S.iters = 0;
    if (!isfinite(acc[0])) {
        S.status = 3;
        S.active = 0;
    } else if (acc[0] <= S.tol2) {
        S.status = 1;
        S.active = 0;
    }
}

// FP64 outer residual r = b - y and |r|^2; an RHS flagged `fresh` (x = 0)
// takes r = b and also records |b|^2, turning tol2 = r_target^2 into the
// absolute threshold r_target^2 |b|^2
__global__ void k_residual64(Cfg c, const double2 *b, const double2 *y, double2 *rv,
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
            V12<double> bb = ld<double>(b, cs, me);
            if (st[r].fresh) {
                acc[1] += snorm(bb);
            } else {
                V12<double> yy = ld<double>(y, cs, me);
#pragma unroll
                for (int k = 0; k < 12; k++) bb.c[k] = bb.c[k] - yy.c[k];
            }
            stv<double>(rv, cs, me, bb);
            acc[0] += snorm(bb);
        }
    }
    const int r = threadIdx.x % nrhs;
    if (!reduce_last<2>(acc, c, partials, counter, nrhs)) return;
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
    } else if (acc[0] <= S.tol2) {
        S.status = 1;
        S.active = 0;
    }
}

__global__ void k_norm2(Cfg c, int prec, const void *v, long long Vh, int nrhs, double *out,
                        double *partials, unsigned int *counter, const RhsState *st_unused)
{
    double acc[1] = {0};
    const int n = nrhs;
    const int r = threadIdx.x % n, lane = threadIdx.x / n;
    const long long cs = Vh * n;
    for (long long s = (long long)blockIdx.x * c.lanes + lane; s < Vh; s += (long long)gridDim.x * c.lanes) {
        const long long me = s * n + r;
        if (prec == 0)
            acc[0] += snorm(ld<double>(v, cs, me));
        else
            acc[0] += (double)snorm(ld<float>(v, cs, me));
    }
    (void)st_unused;
    if (!reduce_last<1>(acc, c, partials, counter, nrhs)) return;
    out[r] = acc[0];
}

__global__ void k_to_f32_scaled(const double2 *r64, float4 *r32, long long Vh, int n,
                                const RhsState *st)
{
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= Vh * n) return;
    const int r = (int)(gid % n);
    const long long cs = Vh * n;
    const double inv = st[r].active ? 1.0 / st[r].scale : 0.0;
    V12<double> a = ld<double>(r64, cs, gid);
    V12<float> o;
#pragma unroll
    for (int k = 0; k < 12; k++) o.c[k] = {(float)(a.c[k].re * inv), (float)(a.c[k].im * inv)};
    stv<float>(r32, cs, gid, o);
}

__global__ void k_acc_f32(double2 *x64, const float4 *e32, long long Vh, int n,
                          const RhsState *st)
{
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= Vh * n) return;
    const int r = (int)(gid % n);
    if (!st[r].active) return;
    const long long cs = Vh * n;
    const double sc = st[r].scale;
    V12<double> x = ld<double>(x64, cs, gid);
    V12<float> e = ld<float>(e32, cs, gid);
#pragma unroll
    for (int k = 0; k < 12; k++) {
        x.c[k].re = fmx(sc, (double)e.c[k].re, x.c[k].re);
        x.c[k].im = fmx(sc, (double)e.c[k].im, x.c[k].im);
    }
    stv<double>(x64, cs, gid, x);
}

__global__ void k_count_active(const RhsState *st, int n, int *n_active)
{
    int c = 0;
    for (int r = 0; r < n; r++) c += st[r].active ? 1 : 0;
    *n_active = c;
}

// inner state from the outer one: same active set; inner tolerance per RHS is
// max(inner_tol, 0.5 * target |b| / |r|): no need to go below what the outer
// loop asks for
__global__ void k_inner_setup(const RhsState *outer, RhsState *inner, int n, double inner_tol,
                              double target)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    RhsState S = {};
    S.active = outer[r].active;
    // the outer threshold is tol2 = r^2 |b|^2: reducing |r| by
    // 0.5 sqrt(tol2)/|r| already meets it, so never ask the inner solve for more
    double tol = inner_tol;
    (void)target;
    if (outer[r].rr > 0) {
        const double want = 0.5 * sqrt(outer[r].tol2 / outer[r].rr);
        if (want > tol) tol = want;
    }
    if (tol > 0.5) tol = 0.5;
    S.tol2 = tol * tol;
    S.status = 0;
    inner[r] = S;
}

}  // namespace

// Grid of a grid-stride reduction: one full wave (resident blocks per SM x
// SMs, from the occupancy calculator), so no partial second wave idles the
// machine at the end; never more blocks than the scratch holds.
template <typename K>
static int one_wave(K kernel, int block, int cap)
{
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair((const void *)kernel, block);
    auto it = cache.find(key);
    if (it != cache.end()) return std::min(it->second, cap);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, block, 0) != cudaSuccess || per < 1)
        per = 1;
    cudaGetLastError();
    const int w = std::max(1, per * std::max(1, sms));
    cache[key] = w;
    return std::min(w, cap);
}

static Cfg cfg(const BlasCtx &bc, long long Vh, int n) { return cfg_for(Vh, n, bc.blocks); }

template <typename K>
static Cfg cfg_wave(const BlasCtx &bc, K kernel, long long Vh, int n)
{
    Cfg c = cfg_for(Vh, n, bc.blocks);
    c.grid = std::min(c.grid, one_wave(kernel, c.block, bc.blocks));
    return c;
}

cudaError_t blas_zero(void *v, size_t bytes, cudaStream_t s) { return cudaMemsetAsync(v, 0, bytes, s); }

#define DISPATCH(prec, KERNEL, ...)                                              \
    do {                                                                         \
        (void)c;                                                                 \
        if ((prec) == 0) {                                                       \
            const Cfg cw = cfg_wave(bc, KERNEL<double>, Vh, nrhs);               \
            KERNEL<double><<<cw.grid, cw.block, 0, s>>>(cw, __VA_ARGS__);        \
        } else {                                                                 \
            const Cfg cw = cfg_wave(bc, KERNEL<float>, Vh, nrhs);                \
            KERNEL<float><<<cw.grid, cw.block, 0, s>>>(cw, __VA_ARGS__);         \
        }                                                                        \
    } while (0)

cudaError_t blas_bicg_init(BlasCtx &bc, int prec, const void *b, void *r, void *rhat, void *p,
                           void *v, void *x, long long Vh, int nrhs, RhsState *st, double tol,
                           cudaStream_t s)
{
    (void)tol;
    const size_t bytes = (size_t)Vh * nrhs * 24 * (prec == 0 ? 8 : 4);
    cudaMemsetAsync(p, 0, bytes, s);
    cudaMemsetAsync(v, 0, bytes, s);
    cudaMemsetAsync(x, 0, bytes, s);
    Cfg c = cfg(bc, Vh, nrhs);
    DISPATCH(prec, k_bicg_init, b, r, rhat, Vh, nrhs, st, bc.partials, bc.counter);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_count_active<<<1, 1, 0, s>>>(st, nrhs, bc.n_active);
    return cudaGetLastError();
}

cudaError_t blas_bicg_p(BlasCtx &bc, int prec, const void *r, void *p, const void *v,
                        long long Vh, int nrhs, const RhsState *st, int first, cudaStream_t s)
{
    Cfg c = cfg(bc, Vh, nrhs);
    DISPATCH(prec, k_bicg_p, r, p, v, Vh, nrhs, st, first);
    return cudaGetLastError();
}

cudaError_t blas_bicg_alpha(BlasCtx &bc, int prec, const void *rhat, const void *v,
                            long long Vh, int nrhs, RhsState *st, cudaStream_t s)
{
    Cfg c = cfg(bc, Vh, nrhs);
    DISPATCH(prec, k_bicg_alpha, rhat, v, Vh, nrhs, st, bc.partials, bc.counter);
    return cudaGetLastError();
}

cudaError_t blas_bicg_s(BlasCtx &bc, int prec, const void *r, const void *v, void *sv,
                        long long Vh, int nrhs, const RhsState *st, cudaStream_t s)
{
    Cfg c = cfg(bc, Vh, nrhs);
    DISPATCH(prec, k_bicg_s, r, v, sv, Vh, nrhs, st);
    return cudaGetLastError();
}

cudaError_t blas_bicg_omega(BlasCtx &bc, int prec, const void *t, const void *sv,
                            long long Vh, int nrhs, RhsState *st, cudaStream_t s)
{
    Cfg c = cfg(bc, Vh, nrhs);
    DISPATCH(prec, k_bicg_omega, t, sv, Vh, nrhs, st, bc.partials, bc.counter);
    return cudaGetLastError();
}

cudaError_t blas_bicg_update(BlasCtx &bc, int prec, void *x, void *r, const void *p,
                             const void *sv, const void *t, const void *rhat, long long Vh,
                             int nrhs, RhsState *st, int max_iter, cudaStream_t s)
{
    Cfg c = cfg(bc, Vh, nrhs);
    DISPATCH(prec, k_bicg_update, x, r, p, sv, t, rhat, Vh, nrhs, st, max_iter, bc.partials,
             bc.counter, bc.n_active);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_count_active<<<1, 1, 0, s>>>(st, nrhs, bc.n_active);
    return cudaGetLastError();
}

cudaError_t blas_residual64(BlasCtx &bc, const double2 *b, const double2 *y, double2 *r,
                            long long Vh, int nrhs, RhsState *st, const int *mask, cudaStream_t s)
{
    const Cfg c = cfg_wave(bc, k_residual64, Vh, nrhs);
    k_residual64<<<c.grid, c.block, 0, s>>>(c, b, y, r, Vh, nrhs, st, mask, bc.partials, bc.counter);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_count_active<<<1, 1, 0, s>>>(st, nrhs, bc.n_active);
    return cudaGetLastError();
}

cudaError_t blas_to_f32_scaled(const double2 *r64, float4 *r32, long long Vh, int nrhs,
                               const RhsState *st, cudaStream_t s)
{
    const long long n = Vh * nrhs;
    k_to_f32_scaled<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(r64, r32, Vh, nrhs, st);
    return cudaGetLastError();
}

cudaError_t blas_acc_f32(double2 *x64, const float4 *e32, long long Vh, int nrhs,
                         const RhsState *st, cudaStream_t s)
{
    const long long n = Vh * nrhs;
    k_acc_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x64, e32, Vh, nrhs, st);
    return cudaGetLastError();
}

cudaError_t blas_norm2(BlasCtx &bc, int prec, const void *v, long long Vh, int nrhs,
                       double *out_dev, cudaStream_t s)
{
    Cfg c = cfg(bc, Vh, nrhs);
    k_norm2<<<c.grid, c.block, 0, s>>>(c, prec, v, Vh, nrhs, out_dev, bc.partials, bc.counter,
                                       nullptr);
    return cudaGetLastError();
}

cudaError_t blas_inner_setup(const RhsState *outer, RhsState *inner, int nrhs, double inner_tol,
                             double target, cudaStream_t s)
{
    k_inner_setup<<<1, 64, 0, s>>>(outer, inner, nrhs, inner_tol, target);
    return cudaGetLastError();
}

namespace {
__global__ void k_scale64(const double2 *v, double2 *out, long long Vh, int n, const RhsState *st)
{
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= Vh * n) return;
    const int r = (int)(gid % n);
    const long long cs = Vh * n;
    const double inv = st[r].active ? 1.0 / st[r].scale : 0.0;
    V12<double> a = ld<double>(v, cs, gid);
#pragma unroll
    for (int k = 0; k < 12; k++) a.c[k] = {a.c[k].re * inv, a.c[k].im * inv};
    stv<double>(out, cs, gid, a);
}

__global__ void k_acc64(double2 *x64, const double2 *e64, long long Vh, int n, const RhsState *st)
{
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= Vh * n) return;
    const int r = (int)(gid % n);
    if (!st[r].active) return;
    const long long cs = Vh * n;
    const double sc = st[r].scale;
    V12<double> x = ld<double>(x64, cs, gid), e = ld<double>(e64, cs, gid);
#pragma unroll
    for (int k = 0; k < 12; k++) {
        x.c[k].re = fmx(sc, e.c[k].re, x.c[k].re);
        x.c[k].im = fmx(sc, e.c[k].im, x.c[k].im);
    }
    stv<double>(x64, cs, gid, x);
}

__global__ void k_diff_norm2(Cfg c, const double2 *a, const double2 *b, long long Vh, int nrhs,
                             double *out, double *partials, unsigned int *counter)
{
    double acc[1] = {0};
    const int n = nrhs;
    const int r = threadIdx.x % n, lane = threadIdx.x / n;
    const long long cs = Vh * n;
    for (long long s = (long long)blockIdx.x * c.lanes + lane; s < Vh; s += (long long)gridDim.x * c.lanes) {
        const long long me = s * n + r;
        V12<double> x = ld<double>(a, cs, me), y = ld<double>(b, cs, me);
#pragma unroll
        for (int k = 0; k < 12; k++) x.c[k] = x.c[k] - y.c[k];
        acc[0] += snorm(x);
    }
    if (!reduce_last<1>(acc, c, partials, counter, nrhs)) return;
    out[r] = acc[0];
}
}  // namespace

cudaError_t blas_scale64(const double2 *v, double2 *out, long long Vh, int nrhs,
                         const RhsState *st, cudaStream_t s)
{
    const long long n = Vh * nrhs;
    k_scale64<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v, out, Vh, nrhs, st);
    return cudaGetLastError();
}

cudaError_t blas_acc64(double2 *x64, const double2 *e64, long long Vh, int nrhs,
                       const RhsState *st, cudaStream_t s)
{
    const long long n = Vh * nrhs;
    k_acc64<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x64, e64, Vh, nrhs, st);
    return cudaGetLastError();
}

cudaError_t blas_diff_norm2(BlasCtx &bc, const double2 *a, const double2 *b, long long Vh,
                            int nrhs, double *out_dev, cudaStream_t s)
{
    Cfg c = cfg(bc, Vh, nrhs);
    k_diff_norm2<<<c.grid, c.block, 0, s>>>(c, a, b, Vh, nrhs, out_dev, bc.partials, bc.counter);
    return cudaGetLastError();
}

namespace {
__global__ void k_zero_masked(double2 *v, long long Vh, int n, const int *mask)
{
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= Vh * n) return;
    if (!mask[gid % n]) return;
    const long long cs = Vh * n;
#pragma unroll
    for (int k = 0; k < 12; k++) v[k * cs + gid] = make_double2(0.0, 0.0);
}
}  // namespace

namespace {
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
}  // namespace

cudaError_t blas_sub64_masked(const double2 *a, const double2 *b, double2 *out, long long Vh,
                              int nrhs, const int *mask, cudaStream_t s)
{
    const long long n = Vh * nrhs;
    k_sub64_masked<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, b, out, Vh, nrhs, mask);
    return cudaGetLastError();
}

cudaError_t blas_zero_masked(double2 *v, long long Vh, int nrhs, const int *mask, cudaStream_t s)
{
    const long long n = Vh * nrhs;
    k_zero_masked<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v, Vh, nrhs, mask);
    return cudaGetLastError();
}

cudaError_t blas_count_active(BlasCtx &bc, const RhsState *st, int nrhs, cudaStream_t s)
{
    k_count_active<<<1, 1, 0, s>>>(st, nrhs, bc.n_active);
    return cudaGetLastError();
}

}  // namespace dp
