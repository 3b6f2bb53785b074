// The outer loop's Schur operator in double-float arithmetic: every real is
// an unevaluated sum hi + lo of two FP32 numbers (|lo| <= ulp(hi)/2 when
// normalised), which carries about 48 significant bits.  Products use the
// FMA error-free product (p = a*b, e = fma(a, b, -p) is exact), sums the
// Knuth two-sum (s = a + b and its exact rounding error from six FP32
// operations); accumulators stay unnormalised (the high parts through
// two-sum, the low parts plainly added) and are normalised once per use.
// GB300 runs FP32 at 64 times its FP64 rate, so this replaces the FP64
// dslash of the true-residual recomputation where 1e-14 relative accuracy
// suffices (residues r >= 1e-12).
//
// Layouts (one parity, n RHS), same byte sizes as the FP64 ones:
//   spinor  float4 [12][Vh][n]  (re_hi, re_lo, im_hi, im_lo) per component
//   links   float4 [4][9][Vh]   per complex element, from the FP64 links
//   clover  float4 [36][Vh]     per pair of reals of the FP64 inverse
//   hops    float2 [group][8][Lmax]
#include "cplx.cuh"
#include "sites.cuh"
#include "dp_internal.h"

namespace dp {
namespace {

struct D2 {  // double-float real: value = x + y
    float x, y;
};
struct DC {  // double-float complex
    D2 re, im;
};

__device__ __forceinline__ D2 dneg(D2 a) { return {-a.x, -a.y}; }

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// normalise: |y| <= ulp(x)/2 (fast two-sum, valid when |x| >= |y|)
__device__ __forceinline__ D2 norm(D2 v)
{
    const float s = __fadd_rn(v.x, v.y);
    return {s, __fsub_rn(v.y, __fsub_rn(s, v.x))};
}

// acc += a * b (lazy)
__device__ __forceinline__ void mac(D2 &acc, D2 a, D2 b)
{
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    float s, r;
    two_sum(acc.x, p, s, r);
    acc.x = s;
    acc.y = __fadd_rn(acc.y, __fadd_rn(r, e));
}

// acc += t (lazy)
__device__ __forceinline__ void acc_add(D2 &acc, D2 t)
{
    float s, r;
    two_sum(acc.x, t.x, s, r);
    acc.x = s;
    acc.y = __fadd_rn(acc.y, __fadd_rn(r, t.y));
}

__device__ __forceinline__ D2 dadd(D2 a, D2 b)
{
    D2 s = a;
    acc_add(s, b);
    return norm(s);
}
__device__ __forceinline__ D2 dsub(D2 a, D2 b) { return dadd(a, dneg(b)); }

__device__ __forceinline__ DC cadd(DC a, DC b) { return {dadd(a.re, b.re), dadd(a.im, b.im)}; }
__device__ __forceinline__ DC csub(DC a, DC b) { return {dsub(a.re, b.re), dsub(a.im, b.im)}; }
__device__ __forceinline__ DC cmi(DC a) { return {a.im, dneg(a.re)}; }   // -i a
__device__ __forceinline__ DC cpi(DC a) { return {dneg(a.im), a.re}; }   // i a
__device__ __forceinline__ DC cneg(DC a) { return {dneg(a.re), dneg(a.im)}; }

// acc += u * h  or  conj(u) * h
__device__ __forceinline__ void cmac(DC &acc, DC u, DC h)
{
    mac(acc.re, u.re, h.re);
    mac(acc.re, dneg(u.im), h.im);
    mac(acc.im, u.re, h.im);
    mac(acc.im, u.im, h.re);
}
__device__ __forceinline__ void cjmac(DC &acc, DC u, DC h)
{
    mac(acc.re, u.re, h.re);
    mac(acc.re, u.im, h.im);
    mac(acc.im, u.re, h.im);
    mac(acc.im, dneg(u.im), h.re);
}
__device__ __forceinline__ DC cnorm(DC a) { return {norm(a.re), norm(a.im)}; }

__device__ __forceinline__ DC ldc(const float4 *p)
{
    const float4 v = __ldg(p);
    return {{v.x, v.y}, {v.z, v.w}};
}

// one hop: acc += c (1 + SG gamma_mu) (U or U^dag) psi(neighbour)
template <int MU, int SG>
__device__ __forceinline__ void hop_df(DC acc[12], const float4 *nb, long long cs, const float4 *lk,
                                       long long Vh, long long lsite, D2 c)
{
    const float4 *l = lk + (long long)MU * 9 * Vh + lsite;
    DC u[9];
#pragma unroll
    for (int k = 0; k < 9; k++) u[k] = ldc(l + k * Vh);
    // spin projection, colour by colour: h = upper spins of (1 + SG gamma_mu) psi
    DC h[6];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const DC p0 = ldc(nb + (0 + a) * cs), p1 = ldc(nb + (3 + a) * cs);
        const DC p2 = ldc(nb + (6 + a) * cs), p3 = ldc(nb + (9 + a) * cs);
        if (MU == 0) {
            h[a] = SG < 0 ? cadd(p0, p2) : csub(p0, p2);
            h[3 + a] = SG < 0 ? cadd(p1, p3) : csub(p1, p3);
        } else if (MU == 1) {
            h[a] = SG < 0 ? cadd(p0, cpi(p3)) : csub(p0, cpi(p3));
            h[3 + a] = SG < 0 ? cadd(p1, cpi(p2)) : csub(p1, cpi(p2));
        } else if (MU == 2) {
            h[a] = SG < 0 ? cadd(p0, p3) : csub(p0, p3);
            h[3 + a] = SG < 0 ? csub(p1, p2) : cadd(p1, p2);
        } else {
            h[a] = SG < 0 ? cadd(p0, cpi(p2)) : csub(p0, cpi(p2));
            h[3 + a] = SG < 0 ? csub(p1, cpi(p3)) : cadd(p1, cpi(p3));
        }
    }
    // scale the half spinor by the hop factor once (12 reals)
#pragma unroll
    for (int k = 0; k < 6; k++) {
        D2 r = {0.f, 0.f}, i = {0.f, 0.f};
        mac(r, c, h[k].re);
        mac(i, c, h[k].im);
        h[k] = {norm(r), norm(i)};
    }
    // uh = U h (forward) or U^dag h (backward), then the lower spins
#pragma unroll
    for (int a = 0; a < 3; a++) {
        DC t0 = {{0.f, 0.f}, {0.f, 0.f}}, t1 = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
        for (int b = 0; b < 3; b++) {
            if (SG < 0) {
                cmac(t0, u[3 * a + b], h[b]);
                cmac(t1, u[3 * a + b], h[3 + b]);
            } else {
                cjmac(t0, u[3 * b + a], h[b]);
                cjmac(t1, u[3 * b + a], h[3 + b]);
            }
        }
        t0 = cnorm(t0);
        t1 = cnorm(t1);
        acc_add(acc[a].re, t0.re);
        acc_add(acc[a].im, t0.im);
        acc_add(acc[3 + a].re, t1.re);
        acc_add(acc[3 + a].im, t1.im);
        DC l2, l3;
        if (MU == 0) {
            l2 = SG < 0 ? t0 : cneg(t0);
            l3 = SG < 0 ? t1 : cneg(t1);
        } else if (MU == 1) {
            l2 = SG < 0 ? cmi(t1) : cpi(t1);
            l3 = SG < 0 ? cmi(t0) : cpi(t0);
        } else if (MU == 2) {
            l2 = SG < 0 ? cneg(t1) : t1;
            l3 = SG < 0 ? t0 : cneg(t0);
        } else {
            l2 = SG < 0 ? cmi(t0) : cpi(t0);
            l3 = SG < 0 ? cpi(t1) : cmi(t1);
        }
        acc_add(acc[6 + a].re, l2.re);
        acc_add(acc[6 + a].im, l2.im);
        acc_add(acc[9 + a].re, l3.re);
        acc_add(acc[9 + a].im, l3.im);
    }
}

// y = M x for one packed Hermitian 6x6 block of the clover inverse in
// double-float (6 real diagonal entries, then (re, im) of the upper triangle)
__device__ __forceinline__ void herm6_df(const float4 *m, long long Vh, const DC *x, DC *y)
{
    // 36 reals = 18 float4 (two reals each)
    D2 r[36];
#pragma unroll
    for (int k = 0; k < 18; k++) {
        const float4 v = __ldg(m + k * Vh);
        r[2 * k] = {v.x, v.y};
        r[2 * k + 1] = {v.z, v.w};
    }
    DC acc[6];
#pragma unroll
    for (int i = 0; i < 6; i++) {
        acc[i] = {{0.f, 0.f}, {0.f, 0.f}};
        mac(acc[i].re, r[i], x[i].re);
        mac(acc[i].im, r[i], x[i].im);
    }
    int k = 6;
#pragma unroll
    for (int i = 0; i < 6; i++) {
#pragma unroll
        for (int j = i + 1; j < 6; j++) {
            const DC a = {r[k], r[k + 1]};
            k += 2;
            cmac(acc[i], a, x[j]);
            cjmac(acc[j], a, x[i]);
        }
    }
#pragma unroll
    for (int i = 0; i < 6; i++) y[i] = cnorm(acc[i]);
}

// EPI_AINV: out (double-float) = A^-1 D in
// EPI_XMY_AINV: out (FP64 double2) = x - A^-1 D in, x double-float
template <int EPI>
__global__ void __launch_bounds__(128, 3) k_dslash_df(const DslashParams p)
{
    const Geom &g = p.g;
    const int n = p.nrhs;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long s = gid / n;
    const int r = (int)(gid - s * n);
    if (s >= g.Vh) return;
    if (p.active && !p.active[r * p.active_stride]) return;
    const Nbr nb = neighbours(g, s, p.parity);
    const long long cs = g.Vh * n;
    const float4 *in = static_cast<const float4 *>(p.in) + r;
    const int grp = p.grp_of[r];
    const float2 *ht = static_cast<const float2 *>(p.hop) + (long long)grp * 8 * g.Lmax;
    const float4 *lown = static_cast<const float4 *>(p.links[p.parity]);
    const float4 *loth = static_cast<const float4 *>(p.links[1 - p.parity]);
    const long long Vh = g.Vh;
    auto hc = [&](int k, int x) {
        const float2 v = __ldg(ht + k * g.Lmax + x);
        return D2{v.x, v.y};
    };
    DC acc[12];
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = {{0.f, 0.f}, {0.f, 0.f}};
    hop_df<0, -1>(acc, in + (long long)nb.f[0] * n, cs, lown, Vh, s, hc(0, nb.t));
    hop_df<0, +1>(acc, in + (long long)nb.b[0] * n, cs, loth, Vh, nb.b[0], hc(1, nb.t));
    hop_df<1, -1>(acc, in + (long long)nb.f[1] * n, cs, lown, Vh, s, hc(2, nb.x));
    hop_df<1, +1>(acc, in + (long long)nb.b[1] * n, cs, loth, Vh, nb.b[1], hc(3, nb.x));
    hop_df<2, -1>(acc, in + (long long)nb.f[2] * n, cs, lown, Vh, s, hc(4, nb.y));
    hop_df<2, +1>(acc, in + (long long)nb.b[2] * n, cs, loth, Vh, nb.b[2], hc(5, nb.y));
    hop_df<3, -1>(acc, in + (long long)nb.f[3] * n, cs, lown, Vh, s, hc(6, nb.z));
    hop_df<3, +1>(acc, in + (long long)nb.b[3] * n, cs, loth, Vh, nb.b[3], hc(7, nb.z));
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = cnorm(acc[k]);
    DC w[12];
    const float4 *cl = static_cast<const float4 *>(p.clov[grp]) + s;
    herm6_df(cl, Vh, acc, w);
    herm6_df(cl + 18 * Vh, Vh, acc + 6, w + 6);
    const long long me = s * n + r;
    if (EPI == EPI_AINV) {
        float4 *out = static_cast<float4 *>(p.out) + me;
#pragma unroll
        for (int k = 0; k < 12; k++) out[k * cs] = make_float4(w[k].re.x, w[k].re.y, w[k].im.x, w[k].im.y);
    } else {
        const float4 *xin = static_cast<const float4 *>(p.x) + me;
        double2 *out = static_cast<double2 *>(p.out) + me;
#pragma unroll
        for (int k = 0; k < 12; k++) {
            const DC xv = ldc(xin + k * cs);
            const DC d = csub(xv, w[k]);
            out[k * cs] = make_double2((double)d.re.x + (double)d.re.y, (double)d.im.x + (double)d.im.y);
        }
    }
}

// FP64 -> double-float (hi = nearest float, lo = nearest float of the rest)
__global__ void k_to_df(const double2 *in, float4 *out, long long count, const int *mask, int n,
                        int mask_stride)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    if (mask && !mask[(int)(i % n) * mask_stride]) return;
    const double2 v = in[i];
    const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
    out[i] = make_float4(rh, __double2float_rn(v.x - (double)rh), ih, __double2float_rn(v.y - (double)ih));
}

// double-float -> FP64
__global__ void k_from_df(const float4 *in, double2 *out, long long count, const int *mask, int n,
                          int mask_stride)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    if (mask && !mask[(int)(i % n) * mask_stride]) return;
    const float4 v = in[i];
    out[i] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}

inline unsigned blocks_for(long long n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

cudaError_t launch_dslash_df(const DslashParams &p, int epi, int block, cudaStream_t st)
{
    if (block <= 0 || block > 128 || (block & 31) || p.nrhs < 1 || p.nrhs > kMaxRhs)
        return cudaErrorInvalidValue;
    const long long threads = p.g.Vh * p.nrhs;
    const unsigned grid = blocks_for(threads, block);
    if (epi == EPI_AINV)
        k_dslash_df<EPI_AINV><<<grid, block, 0, st>>>(p);
    else if (epi == EPI_XMY_AINV)
        k_dslash_df<EPI_XMY_AINV><<<grid, block, 0, st>>>(p);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_to_df(const double2 *in, float4 *out, long long count, const int *mask, int n,
                         int mask_stride, cudaStream_t st)
{
    k_to_df<<<blocks_for(count, 256), 256, 0, st>>>(in, out, count, mask, n, mask_stride);
    return cudaGetLastError();
}

cudaError_t launch_from_df(const float4 *in, double2 *out, long long count, const int *mask, int n,
                           int mask_stride, cudaStream_t st)
{
    k_from_df<<<blocks_for(count, 256), 256, 0, st>>>(in, out, count, mask, n, mask_stride);
    return cudaGetLastError();
}

}  // namespace dp
