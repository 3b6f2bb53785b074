// Schwarz alternating procedure (SAP) on the even-odd Schur operator: the
// preconditioner of the SAP+GCR solver the paper's measurements use (Sec.
// III, Table I; Luscher's domain-decomposition solver).  The lattice is cut
// into blocks (4^4 where the extents allow); a block's Schur operator
//   Mhat_B = 1 - A_pp^-1 D_pq|_B A_qq^-1 D_qp|_B
// keeps only the hops between sites of the block (Dirichlet block
// boundaries).  One launch updates the blocks of one colour (block
// coordinate sum even or odd): each CTA holds one block and one RHS pair in
// shared memory, runs n_mr minimal-residual steps on Mhat_B delta = res_B and
// adds delta to the global correction z.  The caller alternates colours and
// recomputes the global residual in between.
//
// Paired FP32 layout of pair.cuh ([12][Vh][nrhs/2] float4), FP32 12-real or
// 18-real or 16-bit links, FP32 clover inverses [18][Vh] float4.
#include "cplx.cuh"
#include "dp_internal.h"
#include "hop_pair.cuh"
#include "pair.cuh"

namespace dp {
namespace {

struct LocalSite {
    int lt, lx, ly, lz;  // coordinates inside the block
    long long s;         // global half-site index
    int t, x, y, z;      // global coordinates
};

// local half-site i of parity par (block origin has an even coordinate sum,
// so local and global parity agree)
__device__ __forceinline__ LocalSite local_site(const SapParams &p, int i, int par, int ot, int ox,
                                                int oy, int oz)
{
    LocalSite o;
    const int bxh = p.bs[1] / 2;
    const int xh = i % bxh;
    int r = i / bxh;
    o.ly = r % p.bs[2];
    r /= p.bs[2];
    o.lz = r % p.bs[3];
    o.lt = r / p.bs[3];
    o.lx = 2 * xh + ((o.lt + o.ly + o.lz + par) & 1);
    o.t = ot + o.lt;
    o.x = ox + o.lx;
    o.y = oy + o.ly;
    o.z = oz + o.lz;
    o.s = ((((long long)o.t * p.g.Lz + o.z) * p.g.Ly + o.y) * p.g.Lx + o.x) >> 1;
    return o;
}

__device__ __forceinline__ int local_index(const SapParams &p, int lt, int lx, int ly, int lz)
{
    return (((lt * p.bs[3] + lz) * p.bs[2] + ly) * p.bs[1] + lx) >> 1;
}

// acc += hop from a neighbour held in shared memory (sm: [12][vbh] pairs)
template <int LF, int MU, int SG>
__device__ __forceinline__ void hop_local(C2 (&acc)[12], const ulonglong2 *sm, int vbh, int j,
                                          const void *lk, long long Vh, long long lsite, float c)
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
            const ulonglong2 v = sm[(sp * 3 + a) * vbh + j];
            q[sp] = {v.x, v.y};
        }
        project_pair<MU, SG>(q[0], q[1], q[2], q[3], h[a], h[3 + a]);
    }
    hop_apply<MU, SG>(acc, h, u, C, MC);
}

// sum of the hops of output site o (parity par) from the neighbours of the
// other parity that lie inside the block; sm holds those neighbours
template <int LF>
__device__ __forceinline__ void block_hops(const SapParams &p, const LocalSite &o, int par,
                                           const ulonglong2 *sm, int vbh, const float *ht,
                                           C2 (&acc)[12])
{
    const Geom &g = p.g;
    const long long Vh = g.Vh;
    const void *lown = p.links[par], *loth = p.links[1 - par];
#pragma unroll
    for (int j = 0; j < 12; j++) acc[j] = {0ull, 0ull};
    // neighbour global half index (no wrap inside a block)
    auto gidx = [&](int t, int x, int y, int z) {
        return ((((long long)t * g.Lz + z) * g.Ly + y) * g.Lx + x) >> 1;
    };
    if (o.lt + 1 < p.bs[0])
        hop_local<LF, 0, -1>(acc, sm, vbh, local_index(p, o.lt + 1, o.lx, o.ly, o.lz), lown, Vh, o.s,
                             ht[0 * g.Lmax + o.t]);
    if (o.lt > 0)
        hop_local<LF, 0, +1>(acc, sm, vbh, local_index(p, o.lt - 1, o.lx, o.ly, o.lz), loth, Vh,
                             gidx(o.t - 1, o.x, o.y, o.z), ht[1 * g.Lmax + o.t]);
    if (o.lx + 1 < p.bs[1])
        hop_local<LF, 1, -1>(acc, sm, vbh, local_index(p, o.lt, o.lx + 1, o.ly, o.lz), lown, Vh, o.s,
                             ht[2 * g.Lmax + o.x]);
    if (o.lx > 0)
        hop_local<LF, 1, +1>(acc, sm, vbh, local_index(p, o.lt, o.lx - 1, o.ly, o.lz), loth, Vh,
                             gidx(o.t, o.x - 1, o.y, o.z), ht[3 * g.Lmax + o.x]);
    if (o.ly + 1 < p.bs[2])
        hop_local<LF, 2, -1>(acc, sm, vbh, local_index(p, o.lt, o.lx, o.ly + 1, o.lz), lown, Vh, o.s,
                             ht[4 * g.Lmax + o.y]);
    if (o.ly > 0)
        hop_local<LF, 2, +1>(acc, sm, vbh, local_index(p, o.lt, o.lx, o.ly - 1, o.lz), loth, Vh,
                             gidx(o.t, o.x, o.y - 1, o.z), ht[5 * g.Lmax + o.y]);
    if (o.lz + 1 < p.bs[3])
        hop_local<LF, 3, -1>(acc, sm, vbh, local_index(p, o.lt, o.lx, o.ly, o.lz + 1), lown, Vh, o.s,
                             ht[6 * g.Lmax + o.z]);
    if (o.lz > 0)
        hop_local<LF, 3, +1>(acc, sm, vbh, local_index(p, o.lt, o.lx, o.ly, o.lz - 1), loth, Vh,
                             gidx(o.t, o.x, o.y, o.z - 1), ht[7 * g.Lmax + o.z]);
}

__device__ __forceinline__ void clover_inv_apply(const float4 *cl, long long Vh, long long s,
                                                 C2 (&v)[12])
{
#pragma unroll
    for (int blk = 0; blk < 2; blk++) {
        float m[36];
        load_clover_block(cl, Vh, s, blk, m);
        C2 w[6];
        herm6_pair(m, v + 6 * blk, w);
#pragma unroll
        for (int j = 0; j < 6; j++) v[6 * blk + j] = w[j];
    }
}

// per-lane sums of 6 floats over the CTA (warp shuffles, then shared memory)
__device__ __forceinline__ void block_sum6(float (&v)[6], float *red)
{
#pragma unroll
    for (int k = 0; k < 6; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < 6; k++) red[w * 6 + k] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 6; k++) {
        float s = 0.f;
        for (int i = 0; i < nw; i++) s += red[i * 6 + k];
        v[k] = s;
    }
}

// Grid: x = RHS pair (fastest, so the pair-CTAs of one block run together
// and share its links and clover inverses in L1/L2), y = the blocks of this
// colour (when the x-block count is even; otherwise all blocks, the other
// colour exiting at once).  Shared memory per CTA: the block residual rho
// (parity p), the correction delta (parity p) and t, then q (parity q / p).
template <int LF>
__global__ void __launch_bounds__(128, 3) k_sap_block(const SapParams p)
{
    extern __shared__ ulonglong2 sm[];  // R, D: [12][vbh] (parity p); T: [12][vbh]
    __shared__ float red[4 * 6];
    const int vbh = p.bs[0] * p.bs[1] * p.bs[2] * p.bs[3] / 2;
    ulonglong2 *R = sm, *Tq = sm + 12 * vbh, *D = sm + 24 * vbh;
    // block coordinates and colour
    int b = blockIdx.y;
    int bx, by, bz, bt;
    if (p.nb[1] % 2 == 0) {
        const int nxh = p.nb[1] / 2;
        const int j = b % nxh;
        b /= nxh;
        by = b % p.nb[2];
        b /= p.nb[2];
        bz = b % p.nb[3];
        bt = b / p.nb[3];
        bx = 2 * j + ((bt + by + bz + p.colour) & 1);
    } else {
        bx = b % p.nb[1];
        b /= p.nb[1];
        by = b % p.nb[2];
        b /= p.nb[2];
        bz = b % p.nb[3];
        bt = b / p.nb[3];
        if (((bt + bx + by + bz) & 1) != p.colour) return;
    }
    const int q0 = blockIdx.x;  // RHS pair
    if (p.active && !p.active[2 * q0 * p.active_stride] && !p.active[(2 * q0 + 1) * p.active_stride])
        return;
    const int ot = bt * p.bs[0], ox = bx * p.bs[1], oy = by * p.bs[2], oz = bz * p.bs[3];
    const int i = threadIdx.x;
    const bool live = i < vbh;
    const int P = p.nrhs / 2;
    const long long Vh = p.g.Vh, cs = Vh * P;
    const int pp = p.parity, qq = 1 - p.parity;
    const int grp = p.grp_of[2 * q0];
    const float *ht = static_cast<const float *>(p.hop) + (long long)grp * 8 * p.g.Lmax;
    LocalSite sp_{}, sq_{};
    if (live) {
        sp_ = local_site(p, i, pp, ot, ox, oy, oz);
        sq_ = local_site(p, i, qq, ot, ox, oy, oz);
        const ulonglong2 *src = static_cast<const ulonglong2 *>(p.res) + sp_.s * P + q0;
#pragma unroll
        for (int k = 0; k < 12; k++) {
            R[k * vbh + i] = __ldg(src + k * cs);
            D[k * vbh + i] = make_ulonglong2(0ull, 0ull);
        }
    }
    for (int it = 0; it < p.n_mr; it++) {
        __syncthreads();
        C2 acc[12];
        if (live) {
            // t (q-site i) = A_qq^-1 D_qp|_B rho
            block_hops<LF>(p, sq_, qq, R, vbh, ht, acc);
            clover_inv_apply(static_cast<const float4 *>(p.clov[qq][grp]), Vh, sq_.s, acc);
#pragma unroll
            for (int k = 0; k < 12; k++) Tq[k * vbh + i] = make_ulonglong2(acc[k].re, acc[k].im);
        }
        __syncthreads();
        if (live) {
            // A_pp^-1 D_pq|_B t (p-site i)
            block_hops<LF>(p, sp_, pp, Tq, vbh, ht, acc);
            clover_inv_apply(static_cast<const float4 *>(p.clov[pp][grp]), Vh, sp_.s, acc);
        }
        __syncthreads();  // every t read: T now holds q
        float d[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // <q, rho> re, im per lane; |q|^2 per lane
        if (live) {
            // q = rho - A_pp^-1 D_pq|_B t
            f2 dre = 0ull, dim = 0ull, nn = 0ull;
#pragma unroll
            for (int k = 0; k < 12; k++) {
                const ulonglong2 rv = R[k * vbh + i];
                const C2 rho = {rv.x, rv.y};
                const C2 q = c2_sub(rho, acc[k]);
                Tq[k * vbh + i] = make_ulonglong2(q.re, q.im);
                dre = ffma2(q.re, rho.re, dre);
                dre = ffma2(q.im, rho.im, dre);
                dim = ffma2(q.re, rho.im, dim);
                dim = ffma2(fneg2(q.im), rho.re, dim);
                nn = ffma2(q.re, q.re, nn);
                nn = ffma2(q.im, q.im, nn);
            }
            upk(dre, d[0], d[1]);
            upk(dim, d[2], d[3]);
            upk(nn, d[4], d[5]);
        }
        block_sum6(d, red);
        if (live) {
            // omega = <q, rho> / |q|^2 per lane; delta += omega rho, rho -= omega q.
            // Far from a point source a block's residual can be so small that
            // |q|^2 is subnormal: such a block is left alone (omega = 0)
            const bool ok0 = d[4] > 1e-30f, ok1 = d[5] > 1e-30f;
            const C2 om = {pk(ok0 ? d[0] / d[4] : 0.f, ok1 ? d[1] / d[5] : 0.f),
                           pk(ok0 ? d[2] / d[4] : 0.f, ok1 ? d[3] / d[5] : 0.f)};
            const C2 mom = {fneg2(om.re), fneg2(om.im)};
#pragma unroll
            for (int k = 0; k < 12; k++) {
                const ulonglong2 rv = R[k * vbh + i], qv = Tq[k * vbh + i], dv = D[k * vbh + i];
                C2 rho = {rv.x, rv.y};
                const C2 dl = c2_lanefma(om, rho, C2{dv.x, dv.y});
                rho = c2_lanefma(mom, C2{qv.x, qv.y}, rho);
                R[k * vbh + i] = make_ulonglong2(rho.re, rho.im);
                D[k * vbh + i] = make_ulonglong2(dl.re, dl.im);
            }
        }
    }
    if (live) {
        ulonglong2 *z = static_cast<ulonglong2 *>(p.z) + sp_.s * P + q0;
#pragma unroll
        for (int k = 0; k < 12; k++) {
            const ulonglong2 zv = z[k * cs], dv = D[k * vbh + i];
            const C2 s = c2_add({zv.x, zv.y}, C2{dv.x, dv.y});
            z[k * cs] = make_ulonglong2(s.re, s.im);
        }
    }
}

// 4^4 blocks need 72 KB of dynamic shared memory plus the reduction scratch:
// opt in once per kernel
template <int LF>
cudaError_t launch_sap_k(const SapParams &p, dim3 grid, int threads, size_t smem, cudaStream_t st)
{
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_sap_block<LF>, cudaFuncAttributeMaxDynamicSharedMemorySize, 80 * 1024);
    if (attr != cudaSuccess) return attr;
    k_sap_block<LF><<<grid, threads, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace

bool sap_blocks(const Geom &g, int bs[4], int nb[4])
{
    const int L[4] = {g.T, g.Lx, g.Ly, g.Lz};
    for (int mu = 0; mu < 4; mu++) {
        bs[mu] = (L[mu] % 4 == 0) ? 4 : (L[mu] % 2 == 0 ? 2 : 0);
        if (!bs[mu]) return false;
        nb[mu] = L[mu] / bs[mu];
    }
    return true;
}

cudaError_t launch_sap_block(const SapParams &p, int link_fmt, cudaStream_t st)
{
    const int vbh = p.bs[0] * p.bs[1] * p.bs[2] * p.bs[3] / 2;
    if (vbh < 1 || vbh > 128 || p.nrhs % 2) return cudaErrorInvalidValue;
    const int threads = (vbh + 31) / 32 * 32;
    const size_t smem = (size_t)3 * 12 * vbh * sizeof(ulonglong2);
    const int nbt = p.nb[0] * p.nb[1] * p.nb[2] * p.nb[3];
    dim3 grid(p.nrhs / 2, p.nb[1] % 2 == 0 ? nbt / 2 : nbt);
    switch (link_fmt) {
    case LINK_F32_12: return launch_sap_k<LINK_F32_12>(p, grid, threads, smem, st);
    case LINK_F32_18: return launch_sap_k<LINK_F32_18>(p, grid, threads, smem, st);
    case LINK_H16_12: return launch_sap_k<LINK_H16_12>(p, grid, threads, smem, st);
    case LINK_B16_12: return launch_sap_k<LINK_B16_12>(p, grid, threads, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace dp
