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
// Thread mapping: one thread per (output site, RPT consecutive RHS), RHS
// fastest.  The RHS of a site sit in adjacent threads of one warp; for every
// chunk of the spinor layout [chunk][site][rhs] a warp reads one contiguous
// run, so all loads are 128-bit and coalesced.  A thread loads (and, for
// 12-real storage, rebuilds) each link once and applies it to its RPT
// spinors, and loads the clover inverse once for them: RPT > 1 trades
// registers for fewer instructions per RHS (the tuner picks it).  Neighbour
// spinors are re-read by the 8 neighbours through L1/L2 (the 129 MB L2 holds
// several time slices of a 12-RHS field); links and the clover inverse are
// read once per site.
//
// Spin projection in the chiral basis gamma_mu = [[0, e_mu], [e_mu^dag, 0]]
// (e_0 = -1, e_k = -i sigma_k): (1 -/+ gamma_mu) psi = [h; -/+ e_mu^dag h] with
// h = psi_up -/+ e_mu psi_down, so only the 2-spin half spinor h is multiplied
// by the link and the lower spins are rebuilt from U h.
#include "cplx.cuh"
#include "dp_internal.h"

namespace dp {
namespace {

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

// one hop (SG = -1: forward with U, SG = +1: backward with U^dag) applied to
// the RPT spinors of this thread; `nb` points at the neighbour's first RHS
template <typename R, int LF, int MU, int SG, int RPT>
__device__ __forceinline__ void hop(Cx<R> (&acc)[RPT][12], const typename Chunk<R>::T *nb,
                                    long long cs, const void *lk, long long Vh, long long lsite,
                                    R c, const bool (&act)[RPT])
{
    Cx<R> u[9];
    load_link<LF, R>(lk, Vh, lsite, MU, u);
#pragma unroll
    for (int k = 0; k < RPT; k++) {
        if (!act[k]) continue;
        Cx<R> ps[12];
        load_spinor(nb + k, cs, ps);
        Cx<R> h[6];
        project<MU, SG>(ps, h);
        Cx<R> uh[6];
#pragma unroll
        for (int sp = 0; sp < 2; sp++)
#pragma unroll
            for (int a = 0; a < 3; a++) {
                Cx<R> t;
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
        accumulate<MU, SG>(acc[k], uh, c);
    }
}

template <typename R, int LF, int EPI, int RPT>
__global__ void __launch_bounds__(256) k_dslash(const DslashParams p)
{
    using CT = typename Chunk<R>::T;
    const Geom &g = p.g;
    const int n = p.nrhs;
    const int per_site = n / RPT;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long s = gid / per_site;
    const int r0 = (int)(gid - s * per_site) * RPT;
    if (s >= g.Vh) return;
    bool act[RPT];
    bool any = false;
#pragma unroll
    for (int k = 0; k < RPT; k++) {
        act[k] = !p.active || p.active[(r0 + k) * p.active_stride];  // skip converged RHS
        any = any || act[k];
    }
    if (!any) return;

    const int xh = (int)(s % g.Lxh);
    long long q = s / g.Lxh;
    const int y = (int)(q % g.Ly);
    q /= g.Ly;
    const int z = (int)(q % g.Lz);
    const int t = (int)(q / g.Lz);
    const int x = 2 * xh + ((t + y + z + p.parity) & 1);

    const long long cs = g.Vh * n;
    const CT *in = static_cast<const CT *>(p.in) + r0;
    const int grp = p.grp_of[r0];  // the RPT RHS of a thread share their group
    const R *hop_t = static_cast<const R *>(p.hop) + (long long)grp * 8 * g.Lmax;
    const void *lown = p.links[p.parity];
    const void *loth = p.links[1 - p.parity];
    const long long Vh = g.Vh;

    Cx<R> acc[RPT][12];
#pragma unroll
    for (int k = 0; k < RPT; k++)
#pragma unroll
        for (int j = 0; j < 12; j++) acc[k][j] = {R(0), R(0)};

    auto row = [&](int tt, int zz, int yy) -> long long {
        return (((long long)tt * g.Lz + zz) * g.Ly + yy) * g.Lxh;
    };
    // time
    {
        const int tp = (t + 1 == g.T) ? 0 : t + 1, tm = (t == 0) ? g.T - 1 : t - 1;
        const long long sf = row(tp, z, y) + xh, sb = row(tm, z, y) + xh;
        hop<R, LF, 0, -1, RPT>(acc, in + sf * n, cs, lown, Vh, s, hop_t[(0 * 2 + 0) * g.Lmax + t], act);
        hop<R, LF, 0, +1, RPT>(acc, in + sb * n, cs, loth, Vh, sb, hop_t[(0 * 2 + 1) * g.Lmax + t], act);
    }
    // x
    {
        const int xp = (x + 1 == g.Lx) ? 0 : x + 1, xm = (x == 0) ? g.Lx - 1 : x - 1;
        const long long r0w = row(t, z, y);
        const long long sf = r0w + (xp >> 1), sb = r0w + (xm >> 1);
        hop<R, LF, 1, -1, RPT>(acc, in + sf * n, cs, lown, Vh, s, hop_t[(1 * 2 + 0) * g.Lmax + x], act);
        hop<R, LF, 1, +1, RPT>(acc, in + sb * n, cs, loth, Vh, sb, hop_t[(1 * 2 + 1) * g.Lmax + x], act);
    }
    // y
    {
        const int yp = (y + 1 == g.Ly) ? 0 : y + 1, ym = (y == 0) ? g.Ly - 1 : y - 1;
        const long long sf = row(t, z, yp) + xh, sb = row(t, z, ym) + xh;
        hop<R, LF, 2, -1, RPT>(acc, in + sf * n, cs, lown, Vh, s, hop_t[(2 * 2 + 0) * g.Lmax + y], act);
        hop<R, LF, 2, +1, RPT>(acc, in + sb * n, cs, loth, Vh, sb, hop_t[(2 * 2 + 1) * g.Lmax + y], act);
    }
    // z
    {
        const int zp = (z + 1 == g.Lz) ? 0 : z + 1, zm = (z == 0) ? g.Lz - 1 : z - 1;
        const long long sf = row(t, zp, y) + xh, sb = row(t, zm, y) + xh;
        hop<R, LF, 3, -1, RPT>(acc, in + sf * n, cs, lown, Vh, s, hop_t[(3 * 2 + 0) * g.Lmax + z], act);
        hop<R, LF, 3, +1, RPT>(acc, in + sb * n, cs, loth, Vh, sb, hop_t[(3 * 2 + 1) * g.Lmax + z], act);
    }

    const long long me = s * n + r0;
    CT *out = static_cast<CT *>(p.out) + me;
    const CT *xin = static_cast<const CT *>(p.x) + me;
    if (EPI == EPI_HOP || EPI == EPI_XPY) {
#pragma unroll
        for (int k = 0; k < RPT; k++) {
            if (!act[k]) continue;
            if (EPI == EPI_XPY) {
                Cx<R> v[12];
                load_spinor(xin + k, cs, v);
#pragma unroll
                for (int j = 0; j < 12; j++) acc[k][j] = v[j] + acc[k][j];
            }
            store_spinor(out + k, cs, acc[k]);
        }
        return;
    }
    if (EPI == EPI_AINV_XMY) {
#pragma unroll
        for (int k = 0; k < RPT; k++) {
            if (!act[k]) continue;
            Cx<R> v[12];
            load_spinor(xin + k, cs, v);
#pragma unroll
            for (int j = 0; j < 12; j++) acc[k][j] = v[j] - acc[k][j];
        }
    }
    // A^-1 of the output parity for the mass of this group, loaded once per
    // site and applied to every RHS of the thread
    const CT *cl = static_cast<const CT *>(p.clov[grp]);
#pragma unroll
    for (int blk = 0; blk < 2; blk++) {
        R m[36];
        load_clover_block(cl, Vh, s, blk, m);
#pragma unroll
        for (int k = 0; k < RPT; k++) {
            Cx<R> w[6];
            herm6_apply(m, acc[k] + 6 * blk, w);
#pragma unroll
            for (int j = 0; j < 6; j++) acc[k][6 * blk + j] = w[j];
        }
    }
#pragma unroll
    for (int k = 0; k < RPT; k++) {
        if (!act[k]) continue;
        if (EPI == EPI_XMY_AINV) {
            Cx<R> v[12];
            load_spinor(xin + k, cs, v);
#pragma unroll
            for (int j = 0; j < 12; j++) acc[k][j] = v[j] - acc[k][j];
        }
        store_spinor(out + k, cs, acc[k]);
    }
}

template <typename R, int LF, int RPT>
cudaError_t launch_rpt(const DslashParams &p, int epi, int block, cudaStream_t st)
{
    const long long threads = p.g.Vh * (p.nrhs / RPT);
    const unsigned grid = (unsigned)((threads + block - 1) / block);
    if (RPT > 1) {
        // several RHS per thread only for the two Schur-operator launches
        switch (epi) {
        case EPI_AINV: k_dslash<R, LF, EPI_AINV, RPT><<<grid, block, 0, st>>>(p); break;
        case EPI_XMY_AINV: k_dslash<R, LF, EPI_XMY_AINV, RPT><<<grid, block, 0, st>>>(p); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    switch (epi) {
    case EPI_HOP: k_dslash<R, LF, EPI_HOP, RPT><<<grid, block, 0, st>>>(p); break;
    case EPI_AINV: k_dslash<R, LF, EPI_AINV, RPT><<<grid, block, 0, st>>>(p); break;
    case EPI_XMY_AINV: k_dslash<R, LF, EPI_XMY_AINV, RPT><<<grid, block, 0, st>>>(p); break;
    case EPI_AINV_XMY: k_dslash<R, LF, EPI_AINV_XMY, RPT><<<grid, block, 0, st>>>(p); break;
    case EPI_XPY: k_dslash<R, LF, EPI_XPY, RPT><<<grid, block, 0, st>>>(p); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename R, int LF>
cudaError_t launch_fmt(const DslashParams &p, int epi, int block, int rpt, cudaStream_t st)
{
    switch (rpt) {
    case 1: return launch_rpt<R, LF, 1>(p, epi, block, st);
    case 2: return launch_rpt<R, LF, 2>(p, epi, block, st);
    case 3: return launch_rpt<R, LF, 3>(p, epi, block, st);
    case 4: return launch_rpt<R, LF, 4>(p, epi, block, st);
    default: return cudaErrorInvalidValue;
    }
}

// ---- staged variant: FP32, 12-real links, one RHS per thread ----------------
//
// Every thread first issues asynchronous global->shared copies (cp.async,
// 16 bytes each) of its 8 neighbour spinors, and the threads of a site share
// the copies of the site's 8 links; after one wait and a block barrier
// everything is computed from shared memory.  No register is held by a load
// in flight, so many more bytes are in flight per SM than in the register
// path, whose threads each wait on one neighbour at a time.  A block holds
// whole sites (sites_per_block x n threads) so a site's threads share its
// staged links.  Shared memory per block: 768 B per thread (spinors) plus
// 384 B per site (links).

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// rows 0, 1 from three float4; row 2 = conj(row0 x row1)
__device__ __forceinline__ void link12(const float4 *l, Cx<float> u[9])
{
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const float4 v = l[k];
        u[2 * k] = {v.x, v.y};
        u[2 * k + 1] = {v.z, v.w};
    }
    const Cx<float> a = cmul(u[1], u[5]) - cmul(u[2], u[4]);
    const Cx<float> b = cmul(u[2], u[3]) - cmul(u[0], u[5]);
    const Cx<float> c = cmul(u[0], u[4]) - cmul(u[1], u[3]);
    u[6] = {a.re, -a.im};
    u[7] = {b.re, -b.im};
    u[8] = {c.re, -c.im};
}

template <int MU, int SG>
__device__ __forceinline__ void hop_smem(Cx<float> acc[12], const float4 *sp, int nt,
                                         const float4 *lk, float c)
{
    Cx<float> ps[12];
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const float4 v = sp[k * nt];
        ps[2 * k] = {v.x, v.y};
        ps[2 * k + 1] = {v.z, v.w};
    }
    Cx<float> h[6];
    project<MU, SG>(ps, h);
    Cx<float> u[9];
    link12(lk, u);
    Cx<float> uh[6];
#pragma unroll
    for (int s2 = 0; s2 < 2; s2++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            Cx<float> t;
            if (SG < 0) {
                t = cmul(u[3 * a], h[3 * s2]);
                t = cfma(u[3 * a + 1], h[3 * s2 + 1], t);
                t = cfma(u[3 * a + 2], h[3 * s2 + 2], t);
            } else {
                t = cjmul(u[a], h[3 * s2]);
                t = cjfma(u[3 + a], h[3 * s2 + 1], t);
                t = cjfma(u[6 + a], h[3 * s2 + 2], t);
            }
            uh[3 * s2 + a] = t;
        }
    accumulate<MU, SG>(acc, uh, c);
}

template <int EPI>
__global__ void __launch_bounds__(96) k_dslash_staged(const DslashParams p, int spb)
{
    extern __shared__ float4 smem[];
    const Geom &g = p.g;
    const int n = p.nrhs, nt = blockDim.x;
    float4 *sp = smem;            // [8 neighbours][6 chunks][nt]
    float4 *sl = smem + 48 * nt;  // [site][8 links: 4 forward (own), 4 backward][3]
    const int tid = threadIdx.x;
    const int ls = tid / n, r = tid - ls * n;
    const long long s = (long long)blockIdx.x * spb + ls;
    const bool valid = s < g.Vh;
    const bool act = valid && (!p.active || p.active[r * p.active_stride]);
    const long long cs = g.Vh * n;
    const float4 *in = static_cast<const float4 *>(p.in);
    int x = 0, y = 0, z = 0, t = 0;
    long long nb[8];  // forward t, x, y, z then backward t, x, y, z
    if (valid) {
        const int xh = (int)(s % g.Lxh);
        long long q = s / g.Lxh;
        y = (int)(q % g.Ly);
        q /= g.Ly;
        z = (int)(q % g.Lz);
        t = (int)(q / g.Lz);
        x = 2 * xh + ((t + y + z + p.parity) & 1);
        auto row = [&](int tt, int zz, int yy) -> long long {
            return (((long long)tt * g.Lz + zz) * g.Ly + yy) * g.Lxh;
        };
        const int tp = (t + 1 == g.T) ? 0 : t + 1, tm = (t == 0) ? g.T - 1 : t - 1;
        const int xp = (x + 1 == g.Lx) ? 0 : x + 1, xm = (x == 0) ? g.Lx - 1 : x - 1;
        const int yp = (y + 1 == g.Ly) ? 0 : y + 1, ym = (y == 0) ? g.Ly - 1 : y - 1;
        const int zp = (z + 1 == g.Lz) ? 0 : z + 1, zm = (z == 0) ? g.Lz - 1 : z - 1;
        const long long r0 = row(t, z, y);
        nb[0] = row(tp, z, y) + xh;
        nb[1] = r0 + (xp >> 1);
        nb[2] = row(t, z, yp) + xh;
        nb[3] = row(t, zp, y) + xh;
        nb[4] = row(tm, z, y) + xh;
        nb[5] = r0 + (xm >> 1);
        nb[6] = row(t, z, ym) + xh;
        nb[7] = row(t, zm, y) + xh;
        if (act) {
#pragma unroll
            for (int d = 0; d < 8; d++) {
                const float4 *src = in + nb[d] * n + r;
#pragma unroll
                for (int c = 0; c < 6; c++) cp_async16(&sp[(d * 6 + c) * nt + tid], src + c * cs);
            }
        }
        // the site's 24 link chunks, shared out over its n threads
        const float4 *lown = static_cast<const float4 *>(p.links[p.parity]);
        const float4 *loth = static_cast<const float4 *>(p.links[1 - p.parity]);
        for (int qc = r; qc < 24; qc += n) {
            const int d = qc / 3, c = qc - 3 * (qc / 3);
            const float4 *src = d < 4 ? lown + ((long long)d * 3 + c) * g.Vh + s
                                      : loth + ((long long)(d - 4) * 3 + c) * g.Vh + nb[d];
            cp_async16(&sl[(ls * 8 + d) * 3 + c], src);
        }
    }
    cp_async_wait_all();
    __syncthreads();
    if (!act) return;

    const int grp = p.grp_of[r];
    const float *ht = static_cast<const float *>(p.hop) + (long long)grp * 8 * g.Lmax;
    const float4 *myl = sl + ls * 24;
    const float4 *mys = sp + tid;
    Cx<float> acc[12];
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = {0.f, 0.f};
    // same accumulation order as the register kernel (per direction: forward,
    // backward), so both give bit-identical results
    hop_smem<0, -1>(acc, mys + 0 * 6 * nt, nt, myl + 0 * 3, ht[(0 * 2 + 0) * g.Lmax + t]);
    hop_smem<0, +1>(acc, mys + 4 * 6 * nt, nt, myl + 4 * 3, ht[(0 * 2 + 1) * g.Lmax + t]);
    hop_smem<1, -1>(acc, mys + 1 * 6 * nt, nt, myl + 1 * 3, ht[(1 * 2 + 0) * g.Lmax + x]);
    hop_smem<1, +1>(acc, mys + 5 * 6 * nt, nt, myl + 5 * 3, ht[(1 * 2 + 1) * g.Lmax + x]);
    hop_smem<2, -1>(acc, mys + 2 * 6 * nt, nt, myl + 2 * 3, ht[(2 * 2 + 0) * g.Lmax + y]);
    hop_smem<2, +1>(acc, mys + 6 * 6 * nt, nt, myl + 6 * 3, ht[(2 * 2 + 1) * g.Lmax + y]);
    hop_smem<3, -1>(acc, mys + 3 * 6 * nt, nt, myl + 3 * 3, ht[(3 * 2 + 0) * g.Lmax + z]);
    hop_smem<3, +1>(acc, mys + 7 * 6 * nt, nt, myl + 7 * 3, ht[(3 * 2 + 1) * g.Lmax + z]);

    const long long me = s * n + r;
    float4 *out = static_cast<float4 *>(p.out) + me;
    const float4 *xin = static_cast<const float4 *>(p.x) + me;
    if (EPI == EPI_AINV_XMY) {
        Cx<float> v[12];
        load_spinor(xin, cs, v);
#pragma unroll
        for (int j = 0; j < 12; j++) acc[j] = v[j] - acc[j];
    }
    const float4 *cl = static_cast<const float4 *>(p.clov[grp]);
    Cx<float> w[12];
#pragma unroll
    for (int blk = 0; blk < 2; blk++) {
        float m[36];
        load_clover_block(cl, g.Vh, s, blk, m);
        herm6_apply(m, acc + 6 * blk, w + 6 * blk);
    }
    if (EPI == EPI_XMY_AINV) {
        Cx<float> v[12];
        load_spinor(xin, cs, v);
#pragma unroll
        for (int j = 0; j < 12; j++) w[j] = v[j] - w[j];
    }
    store_spinor(out, cs, w);
}

int staged_sites_per_block(int nrhs) { return nrhs >= 96 ? 1 : 96 / nrhs; }

size_t staged_smem_bytes(int nrhs)
{
    const int spb = staged_sites_per_block(nrhs);
    const int nt = spb * nrhs;
    return (size_t)(48 * nt + 24 * spb) * sizeof(float4);
}

template <int EPI>
cudaError_t launch_staged_epi(const DslashParams &p, cudaStream_t st)
{
    const int spb = staged_sites_per_block(p.nrhs);
    const int nt = spb * p.nrhs;
    const size_t sm = staged_smem_bytes(p.nrhs);
    static bool attr_set[kMaxRhs + 1] = {};
    if (!attr_set[p.nrhs]) {
        cudaError_t e = cudaFuncSetAttribute(k_dslash_staged<EPI>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr_set[p.nrhs] = true;
    }
    const unsigned grid = (unsigned)((p.g.Vh + spb - 1) / spb);
    k_dslash_staged<EPI><<<grid, nt, sm, st>>>(p, spb);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_dslash_staged(const DslashParams &p, int epi, cudaStream_t st)
{
    if (p.nrhs < 1 || p.nrhs > kMaxRhs || p.nrhs > 96 || 96 % p.nrhs != 0)
        return cudaErrorInvalidValue;
    switch (epi) {
    case EPI_AINV: return launch_staged_epi<EPI_AINV>(p, st);
    case EPI_XMY_AINV: return launch_staged_epi<EPI_XMY_AINV>(p, st);
    case EPI_AINV_XMY: return launch_staged_epi<EPI_AINV_XMY>(p, st);
    default: return cudaErrorInvalidValue;
    }
}

bool dslash_rpt_ok(int nrhs, int rpt, int prec, int epi)
{
    // rpt 0: the shared-memory staged kernel (FP32, one RHS per thread, whole
    // sites per block of 96 threads, so nrhs must divide 96)
    if (rpt == 0)
        return prec != 0 && nrhs >= 1 && nrhs <= 96 && 96 % nrhs == 0 &&
               (epi == EPI_AINV || epi == EPI_XMY_AINV || epi == EPI_AINV_XMY);
    // the RHS of one thread must share a point-source group (12-aligned);
    // FP64 keeps one RHS per thread (more would spill), and only the Schur
    // launches have multi-RHS-per-thread variants
    if (rpt == 1) return true;
    return prec != 0 && rpt >= 2 && rpt <= 4 && nrhs % rpt == 0 && 12 % rpt == 0 &&
           (epi == EPI_AINV || epi == EPI_XMY_AINV);
}

cudaError_t launch_dslash(const DslashParams &p, int prec, int link_fmt, int epi, int block,
                          int rpt, cudaStream_t st)
{
    if (block <= 0 || block > 256 || (block & 31)) return cudaErrorInvalidValue;
    if (p.nrhs < 1 || p.nrhs > kMaxRhs || !dslash_rpt_ok(p.nrhs, rpt, prec, epi))
        return cudaErrorInvalidValue;
    if (rpt == 0) {
        if (link_fmt != LINK_F32_12) return cudaErrorInvalidValue;
        return launch_dslash_staged(p, epi, st);
    }
    if (prec == 0) {
        if (link_fmt != LINK_F64_18) return cudaErrorInvalidValue;
        return launch_rpt<double, LINK_F64_18, 1>(p, epi, block, st);
    }
    if (link_fmt == LINK_F32_12) return launch_fmt<float, LINK_F32_12>(p, epi, block, rpt, st);
    if (link_fmt == LINK_F32_18) return launch_fmt<float, LINK_F32_18>(p, epi, block, rpt, st);
    return cudaErrorInvalidValue;
}

}  // namespace dp
