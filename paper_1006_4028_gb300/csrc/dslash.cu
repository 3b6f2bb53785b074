// Hopping term of the distance-preconditioned Wilson operator, one parity to
// the other, for n right-hand sides, with fused clover-inverse epilogues.
//
//   (D psi)(x) = sum_mu [ f_mu(x_mu) (1-gamma_mu) U_mu(x) psi(x+mu)
//                        + b_mu(x_mu) (1+gamma_mu) U_mu(x-mu)^dag psi(x-mu) ]
//
// with the profile hop factors of the paper's modified covariant derivatives
// (Sec. II for the time direction, Sec. III eq. redefcovs for all four):
// f = -1/2 alpha_B(x_mu)/alpha_B(x_mu+1), b = -1/2 alpha_B(x_mu)/alpha_B(x_mu-1),
// and the antiperiodic sign on the time seam (eq. redeftbc), read from a small
// per-group table.
//
// Spin projection in the chiral basis gamma_mu = [[0, e_mu], [e_mu^dag, 0]]
// (e_0 = -1, e_k = -i sigma_k): (1 -/+ gamma_mu) psi = [h; -/+ e_mu^dag h] with
// h = psi_up -/+ e_mu psi_down, so only the 2-spin half spinor h is multiplied
// by the link and the lower spins are rebuilt from U h.
//
// Kernels:
//  * FP64, one thread per (output site, RHS), scalar double arithmetic (the
//    FP64 pipe is the bound on GB300);
//  * FP32, one thread per (output site, 1 or 2 RHS pairs) on the paired layout
//    of pair.cuh: every arithmetic step is one packed f32x2 instruction for two
//    RHS, with links, hop factors and the clover inverse loaded once per
//    thread and broadcast to both lanes.  Variants for one pair per thread
//    differ in how the neighbour data arrives: direct loads; spinor and link
//    staged through shared memory (k_dslash32s, or k_dslash32p in one
//    persistent wave); direct loads with an L1 prefetch (k_dslash32f); the
//    spinor alone staged with the link read from L1 at 16 warps per SM
//    (k_dslash32t, the tuner's choice on the benchmark lattice).  All give
//    bit-identical results; the tuner picks per volume and RHS count.
// RHS (pairs) are the fastest index: the RHS of a site sit in adjacent threads
// of one warp, every component load of the [component][site][rhs] layout is
// one contiguous 128-bit run per warp, and the RHS threads of a site share
// their link and clover loads in L1.  Neighbour spinors are re-read by the 8
// neighbours through L1/L2 (the 129 MB L2 holds several time slices of a
// 12-RHS field).
#include <type_traits>

#include "cplx.cuh"
#include "hop_pair.cuh"
#include "sites.cuh"
#include "dp_internal.h"
#include "pair.cuh"

namespace dp {
namespace {

// ---- FP64 (scalar) -------------------------------------------------------------

// h = upper two spins of (1 + SG*gamma_mu) psi, SG = -1 forward, +1 backward
template <int MU, int SG, typename R>
__device__ __forceinline__ void project(const Cx<R> ps[12], Cx<R> h[6])
{
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const Cx<R> p0 = ps[a], p1 = ps[3 + a], p2 = ps[6 + a], p3 = ps[9 + a];
        if (MU == 0) {
            h[a] = SG < 0 ? p0 + p2 : p0 - p2;
            h[3 + a] = SG < 0 ? p1 + p3 : p1 - p3;
        } else if (MU == 1) {
            h[a] = SG < 0 ? p0 + mul_i(p3) : p0 - mul_i(p3);
            h[3 + a] = SG < 0 ? p1 + mul_i(p2) : p1 - mul_i(p2);
        } else if (MU == 2) {
            h[a] = SG < 0 ? p0 + p3 : p0 - p3;
            h[3 + a] = SG < 0 ? p1 - p2 : p1 + p2;
        } else {
            h[a] = SG < 0 ? p0 + mul_i(p2) : p0 - mul_i(p2);
            h[3 + a] = SG < 0 ? p1 - mul_i(p3) : p1 + mul_i(p3);
        }
    }
}

template <typename R>
__device__ __forceinline__ void axpy(R c, Cx<R> v, Cx<R> &acc)
{
    acc.re = fmx(c, v.re, acc.re);
    acc.im = fmx(c, v.im, acc.im);
}

// acc += c * (1 + SG*gamma_mu) psi given uh = U h (the upper spins); the lower
// spins are -SG e_mu^dag uh, written out per direction
template <int MU, int SG, typename R>
__device__ __forceinline__ void accumulate(Cx<R> acc[12], const Cx<R> uh[6], R c)
{
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const Cx<R> h0 = uh[a], h1 = uh[3 + a];
        axpy(c, h0, acc[a]);
        axpy(c, h1, acc[3 + a]);
        Cx<R> l2, l3;
        if (MU == 0) {
            l2 = SG < 0 ? h0 : -h0;
            l3 = SG < 0 ? h1 : -h1;
        } else if (MU == 1) {
            l2 = SG < 0 ? mul_mi(h1) : mul_i(h1);
            l3 = SG < 0 ? mul_mi(h0) : mul_i(h0);
        } else if (MU == 2) {
            l2 = SG < 0 ? -h1 : h1;
            l3 = SG < 0 ? h0 : -h0;
        } else {
            l2 = SG < 0 ? mul_mi(h0) : mul_i(h0);
            l3 = SG < 0 ? mul_i(h1) : mul_mi(h1);
        }
        axpy(c, l2, acc[6 + a]);
        axpy(c, l3, acc[9 + a]);
    }
}

// one hop (SG = -1: forward with U, SG = +1: backward with U^dag)
template <int MU, int SG>
__device__ __forceinline__ void hop64(Cx<double> acc[12], const double2 *nb, long long cs,
                                      const void *lk, long long Vh, long long lsite, double c)
{
    Cx<double> u[9];
    load_link<LINK_F64_18, double>(lk, Vh, lsite, MU, u);
    Cx<double> ps[12];
    load_spinor(nb, cs, ps);
    Cx<double> h[6];
    project<MU, SG>(ps, h);
    Cx<double> uh[6];
#pragma unroll
    for (int sp = 0; sp < 2; sp++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            Cx<double> t;
            if (SG < 0) {
                t = cmul(u[3 * a], h[3 * sp]);
                t = cfma(u[3 * a + 1], h[3 * sp + 1], t);
                t = cfma(u[3 * a + 2], h[3 * sp + 2], t);
            } else {
                t = cjmul(u[a], h[3 * sp]);
                t = cjfma(u[3 + a], h[3 * sp + 1], t);
                t = cjfma(u[6 + a], h[3 * sp + 2], t);
            }
            uh[3 * sp + a] = t;
        }
    accumulate<MU, SG>(acc, uh, c);
}

template <int EPI>
__global__ void __launch_bounds__(256) k_dslash64(const DslashParams p)
{
    const Geom &g = p.g;
    const int n = p.nrhs;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long s = gid / n;
    const int r = (int)(gid - s * n);
    if (s >= g.Vh) return;
    if (p.active && !p.active[r * p.active_stride]) return;  // converged RHS
    const Nbr nb = neighbours(g, s, p.parity);
    const long long cs = g.Vh * n;
    const double2 *in = static_cast<const double2 *>(p.in) + r;
    const int grp = p.grp_of[r];
    const double *ht = static_cast<const double *>(p.hop) + (long long)grp * 8 * g.Lmax;
    const void *lown = p.links[p.parity], *loth = p.links[1 - p.parity];
    const long long Vh = g.Vh;
    Cx<double> acc[12];
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = {0.0, 0.0};
    hop64<0, -1>(acc, in + nb.f[0] * n, cs, lown, Vh, s, ht[0 * g.Lmax + nb.t]);
    hop64<0, +1>(acc, in + nb.b[0] * n, cs, loth, Vh, nb.b[0], ht[1 * g.Lmax + nb.t]);
    hop64<1, -1>(acc, in + nb.f[1] * n, cs, lown, Vh, s, ht[2 * g.Lmax + nb.x]);
    hop64<1, +1>(acc, in + nb.b[1] * n, cs, loth, Vh, nb.b[1], ht[3 * g.Lmax + nb.x]);
    hop64<2, -1>(acc, in + nb.f[2] * n, cs, lown, Vh, s, ht[4 * g.Lmax + nb.y]);
    hop64<2, +1>(acc, in + nb.b[2] * n, cs, loth, Vh, nb.b[2], ht[5 * g.Lmax + nb.y]);
    hop64<3, -1>(acc, in + nb.f[3] * n, cs, lown, Vh, s, ht[6 * g.Lmax + nb.z]);
    hop64<3, +1>(acc, in + nb.b[3] * n, cs, loth, Vh, nb.b[3], ht[7 * g.Lmax + nb.z]);

    const long long me = s * n + r;
    double2 *out = static_cast<double2 *>(p.out) + me;
    const double2 *xin = static_cast<const double2 *>(p.x) + me;
    Cx<double> v[12];
    if (EPI == EPI_HOP || EPI == EPI_XPY || EPI == EPI_XMY_G5) {
        if (EPI == EPI_XPY) {
            load_spinor(xin, cs, v);
#pragma unroll
            for (int j = 0; j < 12; j++) acc[j] = v[j] + acc[j];
        }
        if (EPI == EPI_XMY_G5) {  // gamma5 = +1 on spins 0, 1 and -1 on spins 2, 3
            load_spinor(xin, cs, v);
#pragma unroll
            for (int j = 0; j < 12; j++) acc[j] = j < 6 ? v[j] - acc[j] : v[j] + acc[j];
        }
        store_spinor(out, cs, acc);
        return;
    }
    if (EPI == EPI_AINV_XMY) {
        load_spinor(xin, cs, v);
#pragma unroll
        for (int j = 0; j < 12; j++) acc[j] = v[j] - acc[j];
    }
    const double2 *cl = static_cast<const double2 *>(p.clov[grp]);
    Cx<double> w[12];
#pragma unroll
    for (int blk = 0; blk < 2; blk++) {
        double m[36];
        load_clover_block(cl, Vh, s, blk, m);
        herm6_apply(m, acc + 6 * blk, w + 6 * blk);
    }
    if (EPI == EPI_XMY_AINV) {
        load_spinor(xin, cs, v);
#pragma unroll
        for (int j = 0; j < 12; j++) w[j] = v[j] - w[j];
    }
    store_spinor(out, cs, w);
}

// ---- FP32, two RHS per packed lane pair ------------------------------------------

// one hop for the PPT pairs of this thread, neighbour spinors from global memory
template <int LF, int MU, int SG, int PPT>
__device__ __forceinline__ void hop_pair(C2 (&acc)[PPT][12], const float4 *nb, long long cs,
                                         const void *lk, long long Vh, long long lsite, float c,
                                         const bool (&act)[PPT])
{
    Cx<float> u[9];
    load_link<LF, float>(lk, Vh, lsite, MU, u);
    const f2 C = bc(c), MC = bc(-c);
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        if (!act[k]) continue;
        // project colour by colour: only the 4 spins of one colour are live
        const ulonglong2 *src = reinterpret_cast<const ulonglong2 *>(nb + k);
        C2 h[6];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            C2 q[4];
#pragma unroll
            for (int sp = 0; sp < 4; sp++) {
                const ulonglong2 v = __ldg(src + (sp * 3 + a) * cs);
                q[sp] = {v.x, v.y};
            }
            project_pair<MU, SG>(q[0], q[1], q[2], q[3], h[a], h[3 + a]);
        }
        hop_apply<MU, SG>(acc[k], h, u, C, MC);
    }
}

// links as staged in shared memory next to the spinor (slot components 12-14):
// 12-real FP32 as three float4; 16-bit as three uint2 and the FP32 scale
template <int LF>
__device__ __forceinline__ void link_smem(const float4 *sl, int bd, Cx<float> u[9])
{
    if constexpr (LF == LINK_F32_12) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float4 v = sl[k * bd];
            u[2 * k] = {v.x, v.y};
            u[2 * k + 1] = {v.z, v.w};
        }
    } else {
        using H2 = typename std::conditional<LF == LINK_H16_12, __half2, __nv_bfloat162>::type;
        const uint4 a = *reinterpret_cast<const uint4 *>(sl);
        const uint4 b = *reinterpret_cast<const uint4 *>(sl + bd);
        const unsigned w[6] = {a.x, a.y, a.z, a.w, b.x, b.y};
        const float sc = __uint_as_float(b.z);
#pragma unroll
        for (int k = 0; k < 6; k++) {
            const float2 f = h2f<H2>(w[k]);
            u[k] = {sc * f.x, sc * f.y};
        }
    }
    Cx<float> a = cmul(u[1], u[5]) - cmul(u[2], u[4]);
    Cx<float> b = cmul(u[2], u[3]) - cmul(u[0], u[5]);
    Cx<float> c = cmul(u[0], u[4]) - cmul(u[1], u[3]);
    u[6] = {a.re, -a.im};
    u[7] = {b.re, -b.im};
    u[8] = {c.re, -c.im};
}

// one hop from a neighbour spinor and link staged in shared memory:
// component k of this thread's slot at sb[k * bd], the link from k = 12
template <int LF, int MU, int SG>
__device__ __forceinline__ void hop_smem(C2 (&acc)[12], const float4 *sb, int bd, float c)
{
    Cx<float> u[9];
    link_smem<LF>(sb + 12 * bd, bd, u);
    const f2 C = bc(c), MC = bc(-c);
    C2 h[6];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        C2 q[4];
#pragma unroll
        for (int sp = 0; sp < 4; sp++) {
            const ulonglong2 v = reinterpret_cast<const ulonglong2 *>(sb)[(sp * 3 + a) * bd];
            q[sp] = {v.x, v.y};
        }
        project_pair<MU, SG>(q[0], q[1], q[2], q[3], h[a], h[3 + a]);
    }
    hop_apply<MU, SG>(acc, h, u, C, MC);
}

// ---- asynchronous global -> shared copies: group bookkeeping, L1 prefetch ----
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
__device__ __forceinline__ void prefetch_l1(const void *p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

// epilogue of the FP32 kernels: x + D, x - g5 D, or the A^-1 forms
template <int EPI, int PPT>
__device__ __forceinline__ void finish32(const DslashParams &p, C2 (&acc)[PPT][12],
                                         const bool (&act)[PPT], long long s, int q0, int grp,
                                         long long cs)
{
    const int P = p.nrhs / 2;
    const long long Vh = p.g.Vh;
    const long long me = s * P + q0;
    float4 *out = static_cast<float4 *>(p.out) + me;
    const float4 *xin = static_cast<const float4 *>(p.x) + me;
    if (EPI == EPI_HOP || EPI == EPI_XPY || EPI == EPI_XMY_G5) {
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            if (!act[k]) continue;
            if (EPI == EPI_XPY) {
                C2 v[12];
                load_pair(xin + k, cs, v);
#pragma unroll
                for (int j = 0; j < 12; j++) acc[k][j] = c2_add(v[j], acc[k][j]);
            }
            if (EPI == EPI_XMY_G5) {  // gamma5 = +1 on spins 0, 1 and -1 on spins 2, 3
                C2 v[12];
                load_pair(xin + k, cs, v);
#pragma unroll
                for (int j = 0; j < 12; j++)
                    acc[k][j] = j < 6 ? c2_sub(v[j], acc[k][j]) : c2_add(v[j], acc[k][j]);
            }
            store_pair(out + k, cs, acc[k]);
        }
        return;
    }
    if (EPI == EPI_AINV_XMY) {
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            if (!act[k]) continue;
            C2 v[12];
            load_pair(xin + k, cs, v);
#pragma unroll
            for (int j = 0; j < 12; j++) acc[k][j] = c2_sub(v[j], acc[k][j]);
        }
    }
    // A^-1 of the output parity for this group's mass, loaded once per thread
    const float4 *cl = static_cast<const float4 *>(p.clov[grp]);
#pragma unroll
    for (int blk = 0; blk < 2; blk++) {
        float m[36];
        load_clover_block(cl, Vh, s, blk, m);
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            C2 w[6];
            herm6_pair(m, acc[k] + 6 * blk, w);
#pragma unroll
            for (int j = 0; j < 6; j++) acc[k][6 * blk + j] = w[j];
        }
    }
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        if (!act[k]) continue;
        if (EPI == EPI_XMY_AINV) {
            const ulonglong2 *xp = reinterpret_cast<const ulonglong2 *>(xin + k);
            if (p.dots) {
                // BiCGStab's <t, s> and |t|^2 for this site (t = out, s = x),
                // component by component so that x is not held whole
                f2 tsr = 0ull, tsi = 0ull, tt = 0ull;
#pragma unroll
                for (int j = 0; j < 12; j++) {
                    const ulonglong2 w = __ldg(xp + j * cs);
                    const C2 v = {w.x, w.y};
                    const C2 t = c2_sub(v, acc[k][j]);
                    acc[k][j] = t;
                    tsr = ffma2(t.re, v.re, tsr);
                    tsr = ffma2(t.im, v.im, tsr);
                    tsi = ffma2(t.re, v.im, tsi);
                    tsi = ffma2(fneg2(t.im), v.re, tsi);
                    tt = ffma2(t.re, t.re, tt);
                    tt = ffma2(t.im, t.im, tt);
                }
                f2 *d = static_cast<f2 *>(p.dots) + me + k;
                d[0] = tsr;
                d[cs] = tsi;
                d[2 * cs] = tt;
            } else {
#pragma unroll
                for (int j = 0; j < 12; j++) {
                    const ulonglong2 w = __ldg(xp + j * cs);
                    acc[k][j] = c2_sub(C2{w.x, w.y}, acc[k][j]);
                }
            }
        }
        store_pair(out + k, cs, acc[k]);
    }
}

template <int LF, int EPI, int PPT>
__global__ void __launch_bounds__(256) k_dslash32(const DslashParams p)
{
    const Geom &g = p.g;
    const int P = p.nrhs / 2;  // RHS pairs
    const int per_site = P / PPT;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long s = gid / per_site;
    const int q0 = (int)(gid - s * per_site) * PPT;
    if (s >= g.Vh) return;
    bool act[PPT];
    bool any = false;
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        const int r = 2 * (q0 + k);
        // a pair is computed while either of its RHS is still iterating
        act[k] = !p.active || p.active[r * p.active_stride] || p.active[(r + 1) * p.active_stride];
        any = any || act[k];
    }
    if (!any) return;
    const Nbr nb = neighbours(g, s, p.parity);
    const long long cs = g.Vh * P;
    const float4 *in = static_cast<const float4 *>(p.in) + q0;
    const int grp = p.grp_of[2 * q0];  // the RHS of a thread share their group
    const float *ht = static_cast<const float *>(p.hop) + (long long)grp * 8 * g.Lmax;
    const void *lown = p.links[p.parity], *loth = p.links[1 - p.parity];
    const long long Vh = g.Vh;
    C2 acc[PPT][12];
#pragma unroll
    for (int k = 0; k < PPT; k++)
#pragma unroll
        for (int j = 0; j < 12; j++) acc[k][j] = {0ull, 0ull};
    hop_pair<LF, 0, -1, PPT>(acc, in + nb.f[0] * P, cs, lown, Vh, s, ht[0 * g.Lmax + nb.t], act);
    hop_pair<LF, 0, +1, PPT>(acc, in + nb.b[0] * P, cs, loth, Vh, nb.b[0], ht[1 * g.Lmax + nb.t], act);
    hop_pair<LF, 1, -1, PPT>(acc, in + nb.f[1] * P, cs, lown, Vh, s, ht[2 * g.Lmax + nb.x], act);
    hop_pair<LF, 1, +1, PPT>(acc, in + nb.b[1] * P, cs, loth, Vh, nb.b[1], ht[3 * g.Lmax + nb.x], act);
    hop_pair<LF, 2, -1, PPT>(acc, in + nb.f[2] * P, cs, lown, Vh, s, ht[4 * g.Lmax + nb.y], act);
    hop_pair<LF, 2, +1, PPT>(acc, in + nb.b[2] * P, cs, loth, Vh, nb.b[2], ht[5 * g.Lmax + nb.y], act);
    hop_pair<LF, 3, -1, PPT>(acc, in + nb.f[3] * P, cs, lown, Vh, s, ht[6 * g.Lmax + nb.z], act);
    hop_pair<LF, 3, +1, PPT>(acc, in + nb.b[3] * P, cs, loth, Vh, nb.b[3], ht[7 * g.Lmax + nb.z], act);

    finish32<EPI, PPT>(p, acc, act, s, q0, grp, cs);
}

// ---- FP32, one RHS pair per thread, neighbour spinors and links staged
// through shared memory: direction d + ST is copied asynchronously (cp.async,
// no registers held) while direction d is computed, so ST directions' loads
// are in flight per thread and no global load sits on the hop's critical
// path; the epilogue's clover inverse (and x) are prefetched into L1 at the
// start.  Each thread reads only the slots it filled itself: no block barrier.
// The block size BD is a template parameter so that every shared-memory
// offset is an immediate; each direction's copies are one asm sequence that
// walks the global address itself (no per-copy address registers to keep).
constexpr int kSlot = 15;  // float4 per stage and thread: 12 spinor + 3 link

#define DP_CPA16(OFF) "cp.async.cg.shared.global [%0+" #OFF "*%3], [a], 16;\n\tadd.u64 a, a, %2;\n\t"

// 12 spinor components: shared [sdst + k*BD*16], global src + k*cs_bytes
template <int BD>
__device__ __forceinline__ void stage_spinor(unsigned sdst, const void *src, long long cs_bytes)
{
    asm volatile("{\n\t.reg .u64 a;\n\tmov.u64 a, %1;\n\t"
                 DP_CPA16(0) DP_CPA16(1) DP_CPA16(2) DP_CPA16(3) DP_CPA16(4) DP_CPA16(5)
                 DP_CPA16(6) DP_CPA16(7) DP_CPA16(8) DP_CPA16(9) DP_CPA16(10) DP_CPA16(11)
                 "}\n" ::"r"(sdst), "l"(src), "l"(cs_bytes), "n"(BD * 16)
                 : "memory");
}

// the link of one direction: shared [sdst + k*BD*16] (k = 0..2), global
// stride vh_bytes between its three chunks
template <int BD>
__device__ __forceinline__ void stage_link12(unsigned sdst, const void *src, long long vh_bytes)
{
    asm volatile("{\n\t.reg .u64 a;\n\tmov.u64 a, %1;\n\t"
                 DP_CPA16(0) DP_CPA16(1) DP_CPA16(2)
                 "}\n" ::"r"(sdst), "l"(src), "l"(vh_bytes), "n"(BD * 16)
                 : "memory");
}
#undef DP_CPA16

// 16-bit link: three 8-byte chunks (stride vh_bytes) and the 4-byte scale,
// packed as bytes 0-7, 8-15 of slot 12 and 0-7, 8-11 of slot 13
template <int BD>
__device__ __forceinline__ void stage_link16(unsigned sdst, const void *src, long long vh_bytes,
                                             const void *scale)
{
    asm volatile("{\n\t.reg .u64 a;\n\tmov.u64 a, %1;\n\t"
                 "cp.async.ca.shared.global [%0], [a], 8;\n\tadd.u64 a, a, %2;\n\t"
                 "cp.async.ca.shared.global [%0+8], [a], 8;\n\tadd.u64 a, a, %2;\n\t"
                 "cp.async.ca.shared.global [%0+%3], [a], 8;\n\t"
                 "cp.async.ca.shared.global [%0+%4], [%5], 4;\n\t"
                 "}\n" ::"r"(sdst), "l"(src), "l"(vh_bytes), "n"(BD * 16), "n"(BD * 16 + 8),
                 "l"(scale)
                 : "memory");
}

template <int LF, int BD>
__device__ __forceinline__ void stage_issue(unsigned sslot, const float4 *src, long long cs,
                                            const void *lk, long long Vh, long long lsite, int mu)
{
    stage_spinor<BD>(sslot, src, cs * 16);
    const unsigned sl = sslot + 12 * BD * 16;
    if constexpr (LF == LINK_F32_12) {
        stage_link12<BD>(sl, static_cast<const float4 *>(lk) + (long long)mu * 3 * Vh + lsite, Vh * 16);
    } else {
        const uint2 *l = static_cast<const uint2 *>(lk) + (long long)mu * 3 * Vh + lsite;
        const float *scl = reinterpret_cast<const float *>(static_cast<const uint2 *>(lk) + 12 * Vh) +
                           (long long)mu * Vh + lsite;
        stage_link16<BD>(sl, l, Vh * 8, scl);
    }
}

template <int LF, int ST, int BD, int D>
__device__ __forceinline__ void staged_step(C2 (&acc)[12], const float4 *mine, unsigned smine,
                                            const int (&nbi)[8], const float4 *in, int P,
                                            long long cs, const Nbr &nb, long long s,
                                            const void *lown, const void *loth, long long Vh,
                                            const float (&hc)[8])
{
    constexpr int MU = D / 2;
    constexpr int SLOT = (D % ST) * kSlot * BD;  // in float4
    cp_async_wait<ST - 1>();                       // groups 0..D have landed
    hop_smem<LF, MU, (D & 1) ? +1 : -1>(acc, mine + SLOT, BD, hc[D]);
    if constexpr (D + ST < 8) {
        constexpr int E = D + ST, ME = E / 2;
        stage_issue<LF, BD>(smine + SLOT * 16, in + (long long)nbi[E] * P, cs, (E & 1) ? loth : lown, Vh,
                            (E & 1) ? (long long)nb.b[ME] : s, ME);
    }
    cp_async_commit();  // (possibly empty) group D + ST keeps the count uniform
}

template <int LF, int EPI, int ST, int BD>
__global__ void __launch_bounds__(BD) k_dslash32s(const DslashParams p)
{
    extern __shared__ float4 sbuf[];
    const Geom &g = p.g;
    const int P = p.nrhs / 2;
    const long long gid = (long long)blockIdx.x * BD + threadIdx.x;
    const long long s = gid / P;
    const int q0 = (int)(gid - s * P);
    if (s >= g.Vh) return;
    bool act[1];
    act[0] = !p.active || p.active[2 * q0 * p.active_stride] || p.active[(2 * q0 + 1) * p.active_stride];
    if (!act[0]) return;
    const Nbr nb = neighbours(g, s, p.parity);
    const long long cs = g.Vh * P;
    const float4 *in = static_cast<const float4 *>(p.in) + q0;
    const int grp = p.grp_of[2 * q0];
    const void *lown = p.links[p.parity], *loth = p.links[1 - p.parity];
    const long long Vh = g.Vh;
    const float4 *mine = sbuf + threadIdx.x;
    const unsigned smine = (unsigned)__cvta_generic_to_shared(mine);
    const int nbi[8] = {nb.f[0], nb.b[0], nb.f[1], nb.b[1], nb.f[2], nb.b[2], nb.f[3], nb.b[3]};
#pragma unroll
    for (int d = 0; d < ST; d++) {
        const int mu = d / 2;
        stage_issue<LF, BD>(smine + d * kSlot * BD * 16, in + (long long)nbi[d] * P, cs,
                            (d & 1) ? loth : lown, Vh, (d & 1) ? (long long)nb.b[mu] : s, mu);
        cp_async_commit();
    }
    // the epilogue's operands: into L1 now, read at the end
    {
        const float4 *cl = static_cast<const float4 *>(p.clov[grp]) + s;
#pragma unroll 1
        for (int k = 0; k < 18; k++) prefetch_l1(cl + k * Vh);
        if (EPI == EPI_XMY_AINV) {
            const float4 *xin = static_cast<const float4 *>(p.x) + s * P + q0;
#pragma unroll 1
            for (int k = 0; k < 12; k++) prefetch_l1(xin + k * cs);
        }
    }
    const float *ht = static_cast<const float *>(p.hop) + (long long)grp * 8 * g.Lmax;
    const float hc[8] = {ht[0 * g.Lmax + nb.t], ht[1 * g.Lmax + nb.t], ht[2 * g.Lmax + nb.x],
                         ht[3 * g.Lmax + nb.x], ht[4 * g.Lmax + nb.y], ht[5 * g.Lmax + nb.y],
                         ht[6 * g.Lmax + nb.z], ht[7 * g.Lmax + nb.z]};
    C2 acc[1][12];
#pragma unroll
    for (int j = 0; j < 12; j++) acc[0][j] = {0ull, 0ull};
    staged_step<LF, ST, BD, 0>(acc[0], mine, smine, nbi, in, P, cs, nb, s, lown, loth, Vh, hc);
    staged_step<LF, ST, BD, 1>(acc[0], mine, smine, nbi, in, P, cs, nb, s, lown, loth, Vh, hc);
    staged_step<LF, ST, BD, 2>(acc[0], mine, smine, nbi, in, P, cs, nb, s, lown, loth, Vh, hc);
    staged_step<LF, ST, BD, 3>(acc[0], mine, smine, nbi, in, P, cs, nb, s, lown, loth, Vh, hc);
    staged_step<LF, ST, BD, 4>(acc[0], mine, smine, nbi, in, P, cs, nb, s, lown, loth, Vh, hc);
    staged_step<LF, ST, BD, 5>(acc[0], mine, smine, nbi, in, P, cs, nb, s, lown, loth, Vh, hc);
    staged_step<LF, ST, BD, 6>(acc[0], mine, smine, nbi, in, P, cs, nb, s, lown, loth, Vh, hc);
    staged_step<LF, ST, BD, 7>(acc[0], mine, smine, nbi, in, P, cs, nb, s, lown, loth, Vh, hc);
    finish32<EPI, 1>(p, acc, act, s, q0, grp, cs);
}

// ---- direct loads with an L1 prefetch DIST (= 2) directions ahead: the neighbour
// spinor's 12 components and the link of direction d + DIST are requested
// into L1 (no registers, no shared memory) while direction d is loaded and
// computed from L1.
#define DP_PF "prefetch.global.L1 [a];\n\tadd.u64 a, a, %1;\n\t"
__device__ __forceinline__ void prefetch12(const void *src, long long stride_bytes)
{
    asm volatile("{\n\t.reg .u64 a;\n\tmov.u64 a, %0;\n\t" DP_PF DP_PF DP_PF DP_PF DP_PF DP_PF DP_PF
                 DP_PF DP_PF DP_PF DP_PF DP_PF "}\n" ::"l"(src), "l"(stride_bytes));
}
__device__ __forceinline__ void prefetch3(const void *src, long long stride_bytes)
{
    asm volatile("{\n\t.reg .u64 a;\n\tmov.u64 a, %0;\n\t" DP_PF DP_PF DP_PF "}\n" ::"l"(src),
                 "l"(stride_bytes));
}
#undef DP_PF

template <int LF>
__device__ __forceinline__ void prefetch_dir(const float4 *nbp, long long cs, const void *lk,
                                             long long Vh, long long lsite, int mu)
{
    prefetch12(nbp, cs * 16);
    if constexpr (LF == LINK_F32_12)
        prefetch3(static_cast<const float4 *>(lk) + (long long)mu * 3 * Vh + lsite, Vh * 16);
    else
        prefetch3(static_cast<const uint2 *>(lk) + (long long)mu * 3 * Vh + lsite, Vh * 8);
}

template <int LF, int DIST, int D>
__device__ __forceinline__ void pf_step(C2 (&acc)[1][12], const bool (&act)[1], const float4 *in, int P,
                                        long long cs, const Nbr &nb, long long s, const void *lown,
                                        const void *loth, long long Vh, const float *ht, int Lmax)
{
    if constexpr (D + DIST < 8) {
        constexpr int E = D + DIST, ME = E / 2;
        prefetch_dir<LF>(in + (long long)((E & 1) ? nb.b[ME] : nb.f[ME]) * P, cs, (E & 1) ? loth : lown, Vh,
                         (E & 1) ? (long long)nb.b[ME] : s, ME);
    }
    constexpr int MU = D / 2;
    const int crd = MU == 0 ? nb.t : MU == 1 ? nb.x : MU == 2 ? nb.y : nb.z;
    if (D & 1)
        hop_pair<LF, MU, +1, 1>(acc, in + (long long)nb.b[MU] * P, cs, loth, Vh, nb.b[MU],
                                ht[D * Lmax + crd], act);
    else
        hop_pair<LF, MU, -1, 1>(acc, in + (long long)nb.f[MU] * P, cs, lown, Vh, s, ht[D * Lmax + crd], act);
}

template <int LF, int EPI, int DIST>
__global__ void __launch_bounds__(256, 2) k_dslash32f(const DslashParams p)
{
    const Geom &g = p.g;
    const int P = p.nrhs / 2;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long s = gid / P;
    const int q0 = (int)(gid - s * P);
    if (s >= g.Vh) return;
    bool act[1];
    act[0] = !p.active || p.active[2 * q0 * p.active_stride] || p.active[(2 * q0 + 1) * p.active_stride];
    if (!act[0]) return;
    const Nbr nb = neighbours(g, s, p.parity);
    const long long cs = g.Vh * P;
    const float4 *in = static_cast<const float4 *>(p.in) + q0;
    const int grp = p.grp_of[2 * q0];
    const float *ht = static_cast<const float *>(p.hop) + (long long)grp * 8 * g.Lmax;
    const void *lown = p.links[p.parity], *loth = p.links[1 - p.parity];
    const long long Vh = g.Vh;
#pragma unroll
    for (int d = 0; d < DIST; d++) {
        const int mu = d / 2;
        prefetch_dir<LF>(in + (long long)((d & 1) ? nb.b[mu] : nb.f[mu]) * P, cs, (d & 1) ? loth : lown, Vh,
                         (d & 1) ? (long long)nb.b[mu] : s, mu);
    }
    {
        const float4 *cl = static_cast<const float4 *>(p.clov[grp]) + s;
#pragma unroll 1
        for (int k = 0; k < 18; k++) prefetch_l1(cl + k * Vh);
    }
    C2 acc[1][12];
#pragma unroll
    for (int j = 0; j < 12; j++) acc[0][j] = {0ull, 0ull};
    pf_step<LF, DIST, 0>(acc, act, in, P, cs, nb, s, lown, loth, Vh, ht, g.Lmax);
    pf_step<LF, DIST, 1>(acc, act, in, P, cs, nb, s, lown, loth, Vh, ht, g.Lmax);
    pf_step<LF, DIST, 2>(acc, act, in, P, cs, nb, s, lown, loth, Vh, ht, g.Lmax);
    pf_step<LF, DIST, 3>(acc, act, in, P, cs, nb, s, lown, loth, Vh, ht, g.Lmax);
    pf_step<LF, DIST, 4>(acc, act, in, P, cs, nb, s, lown, loth, Vh, ht, g.Lmax);
    pf_step<LF, DIST, 5>(acc, act, in, P, cs, nb, s, lown, loth, Vh, ht, g.Lmax);
    pf_step<LF, DIST, 6>(acc, act, in, P, cs, nb, s, lown, loth, Vh, ht, g.Lmax);
    pf_step<LF, DIST, 7>(acc, act, in, P, cs, nb, s, lown, loth, Vh, ht, g.Lmax);
    finish32<EPI, 1>(p, acc, act, s, q0, grp, cs);
}

// ---- spinor-only staging: as k_dslash32s with 2 stages, but only the
// neighbour spinor goes through shared memory (12 slots a stage); the link
// is requested into L1 when the spinor copy is issued and read from there
// (the lanes of one site read the same link: one request).  A thread needs
// 384 B of shared memory instead of 480, and the launch bound of 512/BD
// blocks caps it at 128 registers: 16 resident warps per SM against 14 for
// the link-staging kernel (0.275 vs 0.317 ms at 48x24^3, 12 RHS).
constexpr int kSlotT = 12;

template <int LF>
__device__ __forceinline__ void prefetch_link(const void *lk, long long Vh, long long lsite, int mu)
{
    if constexpr (LF == LINK_F32_12) {
        prefetch3(static_cast<const float4 *>(lk) + (long long)mu * 3 * Vh + lsite, Vh * 16);
    } else if constexpr (LF == LINK_F32_18) {
        const float4 *l = static_cast<const float4 *>(lk) + (long long)mu * 4 * Vh + lsite;
        prefetch3(l, Vh * 16);
        prefetch_l1(l + 3 * Vh);
        prefetch_l1(reinterpret_cast<const float2 *>(static_cast<const float4 *>(lk) + 16 * Vh) +
                    (long long)mu * Vh + lsite);
    } else {
        prefetch3(static_cast<const uint2 *>(lk) + (long long)mu * 3 * Vh + lsite, Vh * 8);
        prefetch_l1(reinterpret_cast<const float *>(static_cast<const uint2 *>(lk) + 12 * Vh) +
                    (long long)mu * Vh + lsite);
    }
}

template <int LF, int MU, int SG>
__device__ __forceinline__ void hop_smem_l1(C2 (&acc)[12], const float4 *sb, int bd, const void *lk,
                                            long long Vh, long long lsite, float c)
{
    Cx<float> u[9];
    load_link<LF, float>(lk, Vh, lsite, MU, u);
    const f2 C = bc(c), MC = bc(-c);
    C2 h[6];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        C2 q[4];
#pragma unroll
        for (int sp = 0; sp < 4; sp++) {
            const ulonglong2 v = reinterpret_cast<const ulonglong2 *>(sb)[(sp * 3 + a) * bd];
            q[sp] = {v.x, v.y};
        }
        project_pair<MU, SG>(q[0], q[1], q[2], q[3], h[a], h[3 + a]);
    }
    hop_apply<MU, SG>(acc, h, u, C, MC);
}

template <int LF, int BD, int D>
__device__ __forceinline__ void tstep(C2 (&acc)[12], const float4 *mine, unsigned smine,
                                      const int (&nbi)[8], const float4 *in, int P, long long cs,
                                      const Nbr &nb, long long s, const void *lown, const void *loth,
                                      long long Vh, const float *ht, int Lmax)
{
    constexpr int MU = D / 2;
    constexpr int SLOT = (D % 2) * kSlotT * BD;
    const int crd = MU == 0 ? nb.t : MU == 1 ? nb.x : MU == 2 ? nb.y : nb.z;
    const float c = __ldg(ht + D * Lmax + crd);
    cp_async_wait<1>();
    hop_smem_l1<LF, MU, (D & 1) ? +1 : -1>(acc, mine + SLOT, BD, (D & 1) ? loth : lown, Vh,
                                           (D & 1) ? (long long)nb.b[MU] : s, c);
    if constexpr (D + 2 < 8) {
        constexpr int E = D + 2, ME = E / 2;
        stage_spinor<BD>(smine + SLOT * 16, in + (long long)nbi[E] * P, cs * 16);
        prefetch_link<LF>((E & 1) ? loth : lown, Vh, (E & 1) ? (long long)nb.b[ME] : s, ME);
    }
    cp_async_commit();
}

template <int LF, int EPI, int BD>
__global__ void __launch_bounds__(BD, 512 / BD) k_dslash32t(const DslashParams p)
{
    extern __shared__ float4 sbuf[];
    const Geom &g = p.g;
    const int P = p.nrhs / 2;
    // 32-bit division: the launcher keeps Vh * P below 2^32
    const unsigned gid = blockIdx.x * BD + threadIdx.x;
    const long long s = gid / (unsigned)P;
    const int q0 = (int)(gid - (unsigned)s * (unsigned)P);
    if (s >= g.Vh) return;
    bool act[1];
    act[0] = !p.active || p.active[2 * q0 * p.active_stride] || p.active[(2 * q0 + 1) * p.active_stride];
    if (!act[0]) return;
    const Nbr nb = neighbours(g, s, p.parity);
    const long long cs = g.Vh * P;
    const float4 *in = static_cast<const float4 *>(p.in) + q0;
    const int grp = p.grp_of[2 * q0];
    const void *lown = p.links[p.parity], *loth = p.links[1 - p.parity];
    const long long Vh = g.Vh;
    const float4 *mine = sbuf + threadIdx.x;
    const unsigned smine = (unsigned)__cvta_generic_to_shared(mine);
    const int nbi[8] = {nb.f[0], nb.b[0], nb.f[1], nb.b[1], nb.f[2], nb.b[2], nb.f[3], nb.b[3]};
#pragma unroll
    for (int d = 0; d < 2; d++) {
        stage_spinor<BD>(smine + d * kSlotT * BD * 16, in + (long long)nbi[d] * P, cs * 16);
        prefetch_link<LF>((d & 1) ? loth : lown, Vh, (d & 1) ? (long long)nb.b[0] : s, 0);
        cp_async_commit();
    }
    {
        if (EPI != EPI_XMY_G5) {
            const float4 *cl = static_cast<const float4 *>(p.clov[grp]) + s;
#pragma unroll 1
            for (int k = 0; k < 18; k++) prefetch_l1(cl + k * Vh);
        }
        if (EPI == EPI_XMY_AINV || EPI == EPI_XMY_G5) {
            const float4 *xin = static_cast<const float4 *>(p.x) + s * P + q0;
#pragma unroll 1
            for (int k = 0; k < 12; k++) prefetch_l1(xin + k * cs);
        }
    }
    const float *ht = static_cast<const float *>(p.hop) + (long long)grp * 8 * g.Lmax;
    C2 acc[1][12];
#pragma unroll
    for (int j = 0; j < 12; j++) acc[0][j] = {0ull, 0ull};
    tstep<LF, BD, 0>(acc[0], mine, smine, nbi, in, P, cs, nb, s, lown, loth, Vh, ht, g.Lmax);
    tstep<LF, BD, 1>(acc[0], mine, smine, nbi, in, P, cs, nb, s, lown, loth, Vh, ht, g.Lmax);
    tstep<LF, BD, 2>(acc[0], mine, smine, nbi, in, P, cs, nb, s, lown, loth, Vh, ht, g.Lmax);
    tstep<LF, BD, 3>(acc[0], mine, smine, nbi, in, P, cs, nb, s, lown, loth, Vh, ht, g.Lmax);
    tstep<LF, BD, 4>(acc[0], mine, smine, nbi, in, P, cs, nb, s, lown, loth, Vh, ht, g.Lmax);
    tstep<LF, BD, 5>(acc[0], mine, smine, nbi, in, P, cs, nb, s, lown, loth, Vh, ht, g.Lmax);
    tstep<LF, BD, 6>(acc[0], mine, smine, nbi, in, P, cs, nb, s, lown, loth, Vh, ht, g.Lmax);
    tstep<LF, BD, 7>(acc[0], mine, smine, nbi, in, P, cs, nb, s, lown, loth, Vh, ht, g.Lmax);
    finish32<EPI, 1>(p, acc, act, s, q0, grp, cs);
}

// ---- persistent staged variant: one wave of blocks, each thread walks the
// (site, pair) items w, w + G, w + 2G, ... (G = threads in the grid) with two
// stages; the next item's first two directions are copied while the current
// item finishes its last two directions and its epilogue, so neither the
// start-up nor the epilogue of an item waits on memory.  8 directions per
// item and 2 slots keep every direction in the same slot for all items.
template <int LF, int BD, int D>
__device__ __forceinline__ void pstep(C2 (&acc)[12], const float4 *mine, unsigned smine,
                                      const Nbr &nb, long long s, const float4 *in, int P,
                                      long long cs, const void *lown, const void *loth,
                                      long long Vh, float c, bool next, const Nbr &nbn,
                                      long long sn, const float4 *inn)
{
    constexpr int MU = D / 2;
    constexpr int SLOT = (D % 2) * kSlot * BD;
    cp_async_wait<1>();
    hop_smem<LF, MU, (D & 1) ? +1 : -1>(acc, mine + SLOT, BD, c);
    if constexpr (D + 2 < 8) {
        constexpr int E = D + 2, ME = E / 2;
        const int ni = (E & 1) ? nb.b[ME] : nb.f[ME];
        stage_issue<LF, BD>(smine + SLOT * 16, in + (long long)ni * P, cs, (E & 1) ? loth : lown, Vh,
                            (E & 1) ? (long long)nb.b[ME] : s, ME);
    } else {
        constexpr int E = D + 2 - 8;  // direction 0 or 1 (mu = 0) of the next item
        if (next)
            stage_issue<LF, BD>(smine + SLOT * 16, inn + (long long)(E ? nbn.b[0] : nbn.f[0]) * P, cs,
                                E ? loth : lown, Vh, E ? (long long)nbn.b[0] : sn, 0);
    }
    cp_async_commit();
}

template <int LF, int EPI, int BD>
__global__ void __launch_bounds__(BD) k_dslash32p(const DslashParams p)
{
    extern __shared__ float4 sbuf[];
    const Geom &g = p.g;
    const int P = p.nrhs / 2;
    const long long items = g.Vh * P;
    const long long G = (long long)gridDim.x * BD;
    auto live = [&](long long w) {
        const int q = (int)(w % P);
        return !p.active || p.active[2 * q * p.active_stride] || p.active[(2 * q + 1) * p.active_stride];
    };
    long long w = (long long)blockIdx.x * BD + threadIdx.x;
    while (w < items && !live(w)) w += G;
    if (w >= items) return;
    const long long cs = g.Vh * P;
    const long long Vh = g.Vh;
    const void *lown = p.links[p.parity], *loth = p.links[1 - p.parity];
    const float4 *mine = sbuf + threadIdx.x;
    const unsigned smine = (unsigned)__cvta_generic_to_shared(mine);
    long long s = w / P;
    int q0 = (int)(w - s * P);
    Nbr nb = neighbours(g, s, p.parity);
    const float4 *in = static_cast<const float4 *>(p.in) + q0;
    stage_issue<LF, BD>(smine, in + (long long)nb.f[0] * P, cs, lown, Vh, s, 0);
    cp_async_commit();
    stage_issue<LF, BD>(smine + kSlot * BD * 16, in + (long long)nb.b[0] * P, cs, loth, Vh, nb.b[0], 0);
    cp_async_commit();
    for (;;) {
        long long wn = w + G;
        while (wn < items && !live(wn)) wn += G;
        const bool next = wn < items;
        const long long sn = next ? wn / P : s;
        const int qn = next ? (int)(wn - sn * P) : q0;
        const Nbr nbn = next ? neighbours(g, sn, p.parity) : nb;
        const float4 *inn = static_cast<const float4 *>(p.in) + qn;
        const int grp = p.grp_of[2 * q0];
        {
            const float4 *cl = static_cast<const float4 *>(p.clov[grp]) + s;
#pragma unroll 1
            for (int k = 0; k < 18; k++) prefetch_l1(cl + k * Vh);
            if (EPI == EPI_XMY_AINV) {
                const float4 *xin = static_cast<const float4 *>(p.x) + s * P + q0;
#pragma unroll 1
                for (int k = 0; k < 12; k++) prefetch_l1(xin + k * cs);
            }
        }
        const float *ht = static_cast<const float *>(p.hop) + (long long)grp * 8 * g.Lmax;
        C2 acc[1][12];
#pragma unroll
        for (int j = 0; j < 12; j++) acc[0][j] = {0ull, 0ull};
        pstep<LF, BD, 0>(acc[0], mine, smine, nb, s, in, P, cs, lown, loth, Vh, ht[0 * g.Lmax + nb.t], next, nbn, sn, inn);
        pstep<LF, BD, 1>(acc[0], mine, smine, nb, s, in, P, cs, lown, loth, Vh, ht[1 * g.Lmax + nb.t], next, nbn, sn, inn);
        pstep<LF, BD, 2>(acc[0], mine, smine, nb, s, in, P, cs, lown, loth, Vh, ht[2 * g.Lmax + nb.x], next, nbn, sn, inn);
        pstep<LF, BD, 3>(acc[0], mine, smine, nb, s, in, P, cs, lown, loth, Vh, ht[3 * g.Lmax + nb.x], next, nbn, sn, inn);
        pstep<LF, BD, 4>(acc[0], mine, smine, nb, s, in, P, cs, lown, loth, Vh, ht[4 * g.Lmax + nb.y], next, nbn, sn, inn);
        pstep<LF, BD, 5>(acc[0], mine, smine, nb, s, in, P, cs, lown, loth, Vh, ht[5 * g.Lmax + nb.y], next, nbn, sn, inn);
        pstep<LF, BD, 6>(acc[0], mine, smine, nb, s, in, P, cs, lown, loth, Vh, ht[6 * g.Lmax + nb.z], next, nbn, sn, inn);
        pstep<LF, BD, 7>(acc[0], mine, smine, nb, s, in, P, cs, lown, loth, Vh, ht[7 * g.Lmax + nb.z], next, nbn, sn, inn);
        bool act[1] = {true};
        finish32<EPI, 1>(p, acc, act, s, q0, grp, cs);
        if (!next) break;
        w = wn;
        s = sn;
        q0 = qn;
        nb = nbn;
        in = inn;
    }
}

template <int EPI>
cudaError_t launch64(const DslashParams &p, int block, cudaStream_t st)
{
    const long long threads = p.g.Vh * p.nrhs;
    const unsigned grid = (unsigned)((threads + block - 1) / block);
    k_dslash64<EPI><<<grid, block, 0, st>>>(p);
    return cudaGetLastError();
}

template <int LF, int PPT>
cudaError_t launch32(const DslashParams &p, int epi, int block, cudaStream_t st)
{
    const long long threads = p.g.Vh * (p.nrhs / 2 / PPT);
    const unsigned grid = (unsigned)((threads + block - 1) / block);
    if (PPT > 1) {
        // two pairs per thread only for the two Schur-operator launches
        switch (epi) {
        case EPI_AINV: k_dslash32<LF, EPI_AINV, PPT><<<grid, block, 0, st>>>(p); break;
        case EPI_XMY_AINV: k_dslash32<LF, EPI_XMY_AINV, PPT><<<grid, block, 0, st>>>(p); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    switch (epi) {
    case EPI_HOP: k_dslash32<LF, EPI_HOP, 1><<<grid, block, 0, st>>>(p); break;
    case EPI_AINV: k_dslash32<LF, EPI_AINV, 1><<<grid, block, 0, st>>>(p); break;
    case EPI_XMY_AINV: k_dslash32<LF, EPI_XMY_AINV, 1><<<grid, block, 0, st>>>(p); break;
    case EPI_AINV_XMY: k_dslash32<LF, EPI_AINV_XMY, 1><<<grid, block, 0, st>>>(p); break;
    case EPI_XPY: k_dslash32<LF, EPI_XPY, 1><<<grid, block, 0, st>>>(p); break;
    case EPI_XMY_G5: k_dslash32<LF, EPI_XMY_G5, 1><<<grid, block, 0, st>>>(p); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// the largest staged shape (3 stages x 128 threads) needs 90 KB of dynamic
// shared memory; the opt-in is set once per kernel, outside any capture
template <int LF, int EPI, int ST, int BD>
cudaError_t launch32s_k(const DslashParams &p, cudaStream_t st)
{
    constexpr int smem = ST * kSlot * BD * 16;
    static const cudaError_t attr = cudaFuncSetAttribute(
        k_dslash32s<LF, EPI, ST, BD>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (attr != cudaSuccess) return attr;
    const long long threads = p.g.Vh * (p.nrhs / 2);
    const unsigned grid = (unsigned)((threads + BD - 1) / BD);
    k_dslash32s<LF, EPI, ST, BD><<<grid, BD, smem, st>>>(p);
    return cudaGetLastError();
}

template <int LF, int EPI, int ST>
cudaError_t launch32s_b(const DslashParams &p, int block, cudaStream_t st)
{
    switch (block) {
    case 64: return launch32s_k<LF, EPI, ST, 64>(p, st);
    case 96: return launch32s_k<LF, EPI, ST, 96>(p, st);
    case 128: return launch32s_k<LF, EPI, ST, 128>(p, st);
    default: return cudaErrorInvalidValue;
    }
}

// persistent: one wave, sized from the occupancy calculator (cached)
template <int LF, int EPI, int BD>
cudaError_t launch32p_k(const DslashParams &p, cudaStream_t st)
{
    constexpr int smem = 2 * kSlot * BD * 16;
    static const cudaError_t attr = cudaFuncSetAttribute(
        k_dslash32p<LF, EPI, BD>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (attr != cudaSuccess) return attr;
    static const int per_sm = [] {
        int n = 0, dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_dslash32p<LF, EPI, BD>, BD, smem) !=
                cudaSuccess || n < 1)
            n = 1;
        cudaGetLastError();
        return n * (sms > 0 ? sms : 1);
    }();
    const long long threads = p.g.Vh * (p.nrhs / 2);
    const long long need = (threads + BD - 1) / BD;
    const unsigned grid = (unsigned)(need < per_sm ? need : per_sm);
    k_dslash32p<LF, EPI, BD><<<grid, BD, smem, st>>>(p);
    return cudaGetLastError();
}

template <int LF, int EPI>
cudaError_t launch32s(const DslashParams &p, int block, int stages, cudaStream_t st)
{
    switch (stages) {
    case 2: return launch32s_b<LF, EPI, 2>(p, block, st);
    case 3: return launch32s_b<LF, EPI, 3>(p, block, st);
    case 4:
        switch (block) {
        case 64: return launch32p_k<LF, EPI, 64>(p, st);
        case 96: return launch32p_k<LF, EPI, 96>(p, st);
        case 128: return launch32p_k<LF, EPI, 128>(p, st);
        default: return cudaErrorInvalidValue;
        }
    default: return cudaErrorInvalidValue;
    }
}

template <int LF, int DIST>
cudaError_t launch32f(const DslashParams &p, int epi, int block, cudaStream_t st)
{
    const long long threads = p.g.Vh * (p.nrhs / 2);
    const unsigned grid = (unsigned)((threads + block - 1) / block);
    if (epi == EPI_AINV)
        k_dslash32f<LF, EPI_AINV, DIST><<<grid, block, 0, st>>>(p);
    else
        k_dslash32f<LF, EPI_XMY_AINV, DIST><<<grid, block, 0, st>>>(p);
    return cudaGetLastError();
}

template <int LF, int EPI, int BD>
cudaError_t launch32t_k(const DslashParams &p, cudaStream_t st)
{
    constexpr int smem = 2 * kSlotT * BD * 16;
    static const cudaError_t attr = cudaFuncSetAttribute(
        k_dslash32t<LF, EPI, BD>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (attr != cudaSuccess) return attr;
    const long long threads = p.g.Vh * (p.nrhs / 2);
    if (threads + BD >= (1ll << 32)) return cudaErrorInvalidValue;
    const unsigned grid = (unsigned)((threads + BD - 1) / BD);
    k_dslash32t<LF, EPI, BD><<<grid, BD, smem, st>>>(p);
    return cudaGetLastError();
}

template <int LF, int EPI>
cudaError_t launch32t(const DslashParams &p, int block, cudaStream_t st)
{
    switch (block) {
    case 64: return launch32t_k<LF, EPI, 64>(p, st);
    case 96: return launch32t_k<LF, EPI, 96>(p, st);
    case 128: return launch32t_k<LF, EPI, 128>(p, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int LF>
cudaError_t launch32s_epi(const DslashParams &p, int epi, int block, int stages, int rpt,
                          cudaStream_t st)
{
    (void)rpt;
    if (stages == 5) return launch32f<LF, 2>(p, epi, block, st);
    if (stages == 6)
        return epi == EPI_AINV       ? launch32t<LF, EPI_AINV>(p, block, st)
               : epi == EPI_XMY_G5 ? launch32t<LF, EPI_XMY_G5>(p, block, st)
                                   : launch32t<LF, EPI_XMY_AINV>(p, block, st);
    if (epi == EPI_AINV) return launch32s<LF, EPI_AINV>(p, block, stages, st);
    return launch32s<LF, EPI_XMY_AINV>(p, block, stages, st);
}

}  // namespace

bool dslash_rpt_ok(int nrhs, int rpt, int prec, int epi)
{
    if (prec == 0) return rpt == 1;
    // FP32 works on RHS pairs: nrhs even; 4 RHS per thread (two pairs) only
    // for the Schur launches, with the 4 RHS inside one 12-RHS group
    if (nrhs % 2) return false;
    if (rpt == 2) return true;
    return rpt == 4 && nrhs % 4 == 0 && (epi == EPI_AINV || epi == EPI_XMY_AINV);
}

bool dslash_staged_ok(int prec, int link_fmt, int epi, int rpt, int stages, int block)
{
    if (prec == 1 && rpt == 2 && stages == 5 && block >= 32 && block <= 256 &&
        block % 32 == 0 && (epi == EPI_AINV || epi == EPI_XMY_AINV) &&
        (link_fmt == LINK_F32_12 || link_fmt == LINK_H16_12 || link_fmt == LINK_B16_12))
        return true;
    // the spinor-staged kernel also serves the adjoint's x - g5 D launch
    if (prec == 1 && rpt == 2 && stages == 6 && (block == 64 || block == 96 || block == 128) &&
        (epi == EPI_AINV || epi == EPI_XMY_AINV || epi == EPI_XMY_G5))
        return true;
    return prec == 1 && rpt == 2 && ((stages >= 2 && stages <= 4) || stages == 6) &&
           (block == 64 || block == 96 || block == 128) &&
           (epi == EPI_AINV || epi == EPI_XMY_AINV) &&
           (link_fmt == LINK_F32_12 || link_fmt == LINK_H16_12 || link_fmt == LINK_B16_12);
}

cudaError_t launch_dslash(const DslashParams &p, int prec, int link_fmt, int epi, int block,
                          int rpt, cudaStream_t st, int stages)
{
    if (block <= 0 || block > 256 || (block & 31)) return cudaErrorInvalidValue;
    if (p.nrhs < 1 || p.nrhs > kMaxRhs || !dslash_rpt_ok(p.nrhs, rpt, prec, epi))
        return cudaErrorInvalidValue;
    if (prec == 0) {
        if (link_fmt != LINK_F64_18) return cudaErrorInvalidValue;
        switch (epi) {
        case EPI_HOP: return launch64<EPI_HOP>(p, block, st);
        case EPI_AINV: return launch64<EPI_AINV>(p, block, st);
        case EPI_XMY_AINV: return launch64<EPI_XMY_AINV>(p, block, st);
        case EPI_AINV_XMY: return launch64<EPI_AINV_XMY>(p, block, st);
        case EPI_XPY: return launch64<EPI_XPY>(p, block, st);
        case EPI_XMY_G5: return launch64<EPI_XMY_G5>(p, block, st);
        default: return cudaErrorInvalidValue;
        }
    }
    if (stages > 0) {
        if (!dslash_staged_ok(prec, link_fmt, epi, rpt, stages, block)) return cudaErrorInvalidValue;
        if (link_fmt == LINK_F32_18)  // spinor staging only (stages == 6)
            return epi == EPI_AINV       ? launch32t<LINK_F32_18, EPI_AINV>(p, block, st)
                   : epi == EPI_XMY_G5 ? launch32t<LINK_F32_18, EPI_XMY_G5>(p, block, st)
                                       : launch32t<LINK_F32_18, EPI_XMY_AINV>(p, block, st);
        if (link_fmt == LINK_F32_12) return launch32s_epi<LINK_F32_12>(p, epi, block, stages, rpt, st);
        if (link_fmt == LINK_H16_12) return launch32s_epi<LINK_H16_12>(p, epi, block, stages, rpt, st);
        return launch32s_epi<LINK_B16_12>(p, epi, block, stages, rpt, st);
    }
    const int ppt = rpt / 2;
    if (link_fmt == LINK_F32_12)
        return ppt == 2 ? launch32<LINK_F32_12, 2>(p, epi, block, st) : launch32<LINK_F32_12, 1>(p, epi, block, st);
    if (link_fmt == LINK_F32_18)
        return ppt == 2 ? launch32<LINK_F32_18, 2>(p, epi, block, st) : launch32<LINK_F32_18, 1>(p, epi, block, st);
    if (link_fmt == LINK_H16_12)
        return ppt == 2 ? launch32<LINK_H16_12, 2>(p, epi, block, st) : launch32<LINK_H16_12, 1>(p, epi, block, st);
    if (link_fmt == LINK_B16_12)
        return ppt == 2 ? launch32<LINK_B16_12, 2>(p, epi, block, st) : launch32<LINK_B16_12, 1>(p, epi, block, st);
    return cudaErrorInvalidValue;
}

}  // namespace dp
