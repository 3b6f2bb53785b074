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
// per-profile table.
//
// One thread per (output site, RHS), RHS fastest: the RHS threads of a site
// sit in the same warp and load the same links (one transaction), and for
// every chunk of the spinor layout [chunk][site][rhs] a warp reads one
// contiguous run, so all loads are 128-bit and coalesced.  Neighbour spinors
// are re-read by the 8 neighbours through L1/L2 (129 MB L2 holds several time
// slices of a 12-RHS field); links and the clover inverse are read once.
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

// forward hop: c (1 - gamma_mu) U_mu(x) psi(x+mu); U at the output site
template <typename R, int LF, int MU>
__device__ __forceinline__ void hop_fwd(Cx<R> acc[12], const typename Chunk<R>::T *in,
                                        long long cs, long long nb, const void *lk, long long Vh,
                                        long long site, R c)
{
    Cx<R> ps[12];
    load_spinor(in + nb, cs, ps);
    Cx<R> h[6];
    project<MU, -1>(ps, h);
    Cx<R> u[9];
    load_link<LF, R>(lk, Vh, site, MU, u);
    Cx<R> uh[6];
#pragma unroll
    for (int sp = 0; sp < 2; sp++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            Cx<R> t = cmul(u[3 * a], h[3 * sp]);
            t = cfma(u[3 * a + 1], h[3 * sp + 1], t);
            t = cfma(u[3 * a + 2], h[3 * sp + 2], t);
            uh[3 * sp + a] = t;
        }
    accumulate<MU, -1>(acc, uh, c);
}

// backward hop: c (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu); U at the neighbour
template <typename R, int LF, int MU>
__device__ __forceinline__ void hop_bwd(Cx<R> acc[12], const typename Chunk<R>::T *in,
                                        long long cs, long long nb, const void *lk, long long Vh,
                                        long long nsite, R c)
{
    Cx<R> ps[12];
    load_spinor(in + nb, cs, ps);
    Cx<R> h[6];
    project<MU, +1>(ps, h);
    Cx<R> u[9];
    load_link<LF, R>(lk, Vh, nsite, MU, u);
    Cx<R> uh[6];
#pragma unroll
    for (int sp = 0; sp < 2; sp++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            Cx<R> t = cjmul(u[a], h[3 * sp]);
            t = cjfma(u[3 + a], h[3 * sp + 1], t);
            t = cjfma(u[6 + a], h[3 * sp + 2], t);
            uh[3 * sp + a] = t;
        }
    accumulate<MU, +1>(acc, uh, c);
}

template <typename R, int LF, int EPI>
__global__ void __launch_bounds__(256) k_dslash(const DslashParams p)
{
    using CT = typename Chunk<R>::T;
    const Geom &g = p.g;
    const int n = p.nrhs;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long s = gid / n;
    const int r = (int)(gid - s * n);
    if (s >= g.Vh) return;
    if (p.active && !p.active[r * p.active_stride]) return;  // converged or unused RHS

    const int xh = (int)(s % g.Lxh);
    long long q = s / g.Lxh;
    const int y = (int)(q % g.Ly);
    q /= g.Ly;
    const int z = (int)(q % g.Lz);
    const int t = (int)(q / g.Lz);
    const int x = 2 * xh + ((t + y + z + p.parity) & 1);

    const long long cs = g.Vh * n;
    const CT *in = static_cast<const CT *>(p.in) + r;
    const int grp = p.grp_of[r];
    const R *hop = static_cast<const R *>(p.hop) + (long long)grp * 8 * g.Lmax;
    const void *lown = p.links[p.parity];
    const void *loth = p.links[1 - p.parity];
    const long long Vh = g.Vh;

    Cx<R> acc[12];
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = {R(0), R(0)};

    auto row = [&](int tt, int zz, int yy) -> long long {
        return (((long long)tt * g.Lz + zz) * g.Ly + yy) * g.Lxh;
    };
    // time
    {
        const int tp = (t + 1 == g.T) ? 0 : t + 1, tm = (t == 0) ? g.T - 1 : t - 1;
        const long long sf = row(tp, z, y) + xh, sb = row(tm, z, y) + xh;
        hop_fwd<R, LF, 0>(acc, in, cs, sf * n, lown, Vh, s, hop[(0 * 2 + 0) * g.Lmax + t]);
        hop_bwd<R, LF, 0>(acc, in, cs, sb * n, loth, Vh, sb, hop[(0 * 2 + 1) * g.Lmax + t]);
    }
    // x
    {
        const int xp = (x + 1 == g.Lx) ? 0 : x + 1, xm = (x == 0) ? g.Lx - 1 : x - 1;
        const long long r0 = row(t, z, y);
        const long long sf = r0 + (xp >> 1), sb = r0 + (xm >> 1);
        hop_fwd<R, LF, 1>(acc, in, cs, sf * n, lown, Vh, s, hop[(1 * 2 + 0) * g.Lmax + x]);
        hop_bwd<R, LF, 1>(acc, in, cs, sb * n, loth, Vh, sb, hop[(1 * 2 + 1) * g.Lmax + x]);
    }
    // y
    {
        const int yp = (y + 1 == g.Ly) ? 0 : y + 1, ym = (y == 0) ? g.Ly - 1 : y - 1;
        const long long sf = row(t, z, yp) + xh, sb = row(t, z, ym) + xh;
        hop_fwd<R, LF, 2>(acc, in, cs, sf * n, lown, Vh, s, hop[(2 * 2 + 0) * g.Lmax + y]);
        hop_bwd<R, LF, 2>(acc, in, cs, sb * n, loth, Vh, sb, hop[(2 * 2 + 1) * g.Lmax + y]);
    }
    // z
    {
        const int zp = (z + 1 == g.Lz) ? 0 : z + 1, zm = (z == 0) ? g.Lz - 1 : z - 1;
        const long long sf = row(t, zp, y) + xh, sb = row(t, zm, y) + xh;
        hop_fwd<R, LF, 3>(acc, in, cs, sf * n, lown, Vh, s, hop[(3 * 2 + 0) * g.Lmax + z]);
        hop_bwd<R, LF, 3>(acc, in, cs, sb * n, loth, Vh, sb, hop[(3 * 2 + 1) * g.Lmax + z]);
    }

    const long long me = s * n + r;
    CT *out = static_cast<CT *>(p.out) + me;
    if (EPI == EPI_HOP) {
        store_spinor(out, cs, acc);
        return;
    }
    Cx<R> v[12];
    if (EPI == EPI_XPY || EPI == EPI_XMY_AINV || EPI == EPI_AINV_XMY)
        load_spinor(static_cast<const CT *>(p.x) + me, cs, v);
    if (EPI == EPI_XPY) {
#pragma unroll
        for (int k = 0; k < 12; k++) v[k] = v[k] + acc[k];
        store_spinor(out, cs, v);
        return;
    }
    if (EPI == EPI_AINV_XMY) {
#pragma unroll
        for (int k = 0; k < 12; k++) acc[k] = v[k] - acc[k];
    }
    // A^-1 of the output parity for the mass of this RHS's group
    const CT *cl = static_cast<const CT *>(p.clov[grp]);
    Cx<R> w[12];
#pragma unroll
    for (int blk = 0; blk < 2; blk++) {
        R m[36];
        load_clover_block(cl, Vh, s, blk, m);
        herm6_apply(m, acc + 6 * blk, w + 6 * blk);
    }
    if (EPI == EPI_XMY_AINV) {
#pragma unroll
        for (int k = 0; k < 12; k++) w[k] = v[k] - w[k];
    }
    store_spinor(out, cs, w);
}

template <typename R, int LF>
cudaError_t launch_epi(const DslashParams &p, int epi, int block, cudaStream_t st)
{
    const long long threads = p.g.Vh * p.nrhs;
    const unsigned grid = (unsigned)((threads + block - 1) / block);
    switch (epi) {
    case EPI_HOP: k_dslash<R, LF, EPI_HOP><<<grid, block, 0, st>>>(p); break;
    case EPI_AINV: k_dslash<R, LF, EPI_AINV><<<grid, block, 0, st>>>(p); break;
    case EPI_XMY_AINV: k_dslash<R, LF, EPI_XMY_AINV><<<grid, block, 0, st>>>(p); break;
    case EPI_AINV_XMY: k_dslash<R, LF, EPI_AINV_XMY><<<grid, block, 0, st>>>(p); break;
    case EPI_XPY: k_dslash<R, LF, EPI_XPY><<<grid, block, 0, st>>>(p); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_dslash(const DslashParams &p, int prec, int link_fmt, int epi, int block,
                          cudaStream_t st)
{
    if (block <= 0 || block > 256 || (block & 31)) return cudaErrorInvalidValue;
    if (p.nrhs < 1 || p.nrhs > kMaxRhs) return cudaErrorInvalidValue;
    if (prec == 0) {
        if (link_fmt != LINK_F64_18) return cudaErrorInvalidValue;
        return launch_epi<double, LINK_F64_18>(p, epi, block, st);
    }
    if (link_fmt == LINK_F32_12) return launch_epi<float, LINK_F32_12>(p, epi, block, st);
    if (link_fmt == LINK_F32_18) return launch_epi<float, LINK_F32_18>(p, epi, block, st);
    return cudaErrorInvalidValue;
}

}  // namespace dp
