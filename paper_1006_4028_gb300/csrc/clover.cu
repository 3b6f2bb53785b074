// Clover term of the O(a)-improved Wilson operator (Sec. II), its inverse with
// the mass diagonal, and stand-alone application kernels.
//
// Fhat_{mu nu}(x) = (Q_{mu nu}(x) - Q_{mu nu}(x)^dag)/8, Q the sum of the four
// plaquette leaves at x, and the term c_sw (i/4) sum_{mu,nu} sigma_{mu nu}
// Fhat_{mu nu}.  In the chiral basis sigma_{0k} = diag(s_k, -s_k) and
// sigma_{jk} = -eps_{jkl} diag(s_l, s_l) (s = Pauli matrices), so the term is
// block diagonal in chirality:
//   upper (spins 0,1): sum_l s_l (x) X_l,  X_l = +c_sw (i/2) (Fhat_0l - B_l)
//   lower (spins 2,3): sum_l s_l (x) Y_l,  Y_l = -c_sw (i/2) (Fhat_0l + B_l)
// with B_1 = Fhat_23, B_2 = Fhat_31, B_3 = Fhat_12; each block is the 6x6
// Hermitian matrix [[Z_3, Z_1 - i Z_2], [Z_1 + i Z_2, -Z_3]].
#include "cplx.cuh"
#include "dp_internal.h"
#include "pair.cuh"
#include "reduce.cuh"

namespace dp {
namespace {

using C = Cx<double>;

struct M3 {
    C a[9];
};

__device__ __forceinline__ M3 mmul(const M3 &A, const M3 &B)
{
    M3 Cm;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            C s = cmul(A.a[3 * i], B.a[j]);
            s = cfma(A.a[3 * i + 1], B.a[3 + j], s);
            s = cfma(A.a[3 * i + 2], B.a[6 + j], s);
            Cm.a[3 * i + j] = s;
        }
    return Cm;
}

__device__ __forceinline__ M3 mdag(const M3 &A)
{
    M3 B;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) B.a[3 * i + j] = {A.a[3 * j + i].re, -A.a[3 * j + i].im};
    return B;
}

struct LinkView {
    const double2 *l[2];
    Geom g;
    // U_mu at full coordinates (t, x, y, z), periodic wrap
    __device__ M3 get(int t, int x, int y, int z, int mu) const
    {
        t = (t + g.T) % g.T;
        x = (x + g.Lx) % g.Lx;
        y = (y + g.Ly) % g.Ly;
        z = (z + g.Lz) % g.Lz;
        const int par = (t + x + y + z) & 1;
        const long long s = ((((long long)t * g.Lz + z) * g.Ly + y) * g.Lx + x) >> 1;
        const double2 *b = l[par] + (long long)mu * 9 * g.Vh + s;
        M3 U;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            double2 v = b[k * g.Vh];
            U.a[k] = {v.x, v.y};
        }
        return U;
    }
};

// Fhat_{mu nu} at c = (t, x, y, z), mu < nu
__device__ M3 field_strength(const LinkView &L, const int c[4], int mu, int nu)
{
    int e[4][4] = {{1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}};
    auto at = [&](int sm, int sn, int dir) {
        return L.get(c[0] + sm * e[mu][0] + sn * e[nu][0], c[1] + sm * e[mu][1] + sn * e[nu][1],
                     c[2] + sm * e[mu][2] + sn * e[nu][2], c[3] + sm * e[mu][3] + sn * e[nu][3],
                     dir);
    };
    M3 Q;
    // x -> x+mu -> x+mu+nu -> x+nu -> x
    M3 P = mmul(mmul(at(0, 0, mu), at(1, 0, nu)), mmul(mdag(at(0, 1, mu)), mdag(at(0, 0, nu))));
    Q = P;
    // x -> x+nu -> x+nu-mu -> x-mu -> x
    P = mmul(mmul(at(0, 0, nu), mdag(at(-1, 1, mu))), mmul(mdag(at(-1, 0, nu)), at(-1, 0, mu)));
#pragma unroll
    for (int k = 0; k < 9; k++) Q.a[k] = Q.a[k] + P.a[k];
    // x -> x-mu -> x-mu-nu -> x-nu -> x
    P = mmul(mmul(mdag(at(-1, 0, mu)), mdag(at(-1, -1, nu))), mmul(at(-1, -1, mu), at(0, -1, nu)));
#pragma unroll
    for (int k = 0; k < 9; k++) Q.a[k] = Q.a[k] + P.a[k];
    // x -> x-nu -> x-nu+mu -> x+mu -> x
    P = mmul(mmul(mdag(at(0, -1, nu)), at(0, -1, mu)), mmul(at(1, -1, nu), mdag(at(0, 0, mu))));
#pragma unroll
    for (int k = 0; k < 9; k++) Q.a[k] = Q.a[k] + P.a[k];
    M3 F;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const C q = Q.a[3 * i + j], qt = Q.a[3 * j + i];
            F.a[3 * i + j] = {(q.re - qt.re) * 0.125, (q.im + qt.im) * 0.125};
        }
    return F;
}

// pack Hermitian 6x6 [[Z3, Z1 - i Z2], [Z1 + i Z2, -Z3]] into 36 reals
__device__ void pack_block(const M3 Z[3], double *m)
{
    C H[36];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            const C z1 = Z[0].a[3 * a + b], z2 = Z[1].a[3 * a + b], z3 = Z[2].a[3 * a + b];
            H[a * 6 + b] = z3;
            H[a * 6 + 3 + b] = z1 - mul_i(z2);
            H[(3 + a) * 6 + b] = z1 + mul_i(z2);
            H[(3 + a) * 6 + 3 + b] = -z3;
        }
    for (int i = 0; i < 6; i++) m[i] = H[i * 6 + i].re;
    int k = 6;
    for (int i = 0; i < 6; i++)
        for (int j = i + 1; j < 6; j++) {
            m[k++] = H[i * 6 + j].re;
            m[k++] = H[i * 6 + j].im;
        }
}

__global__ void k_clover_build(LinkView L, double csw, double2 *ce, double2 *co)
{
    const Geom &g = L.g;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    int c[4];
    long long q = i;
    c[1] = (int)(q % g.Lx);
    q /= g.Lx;
    c[2] = (int)(q % g.Ly);
    q /= g.Ly;
    c[3] = (int)(q % g.Lz);
    c[0] = (int)(q / g.Lz);
    const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
    const long long s = i >> 1;

    M3 F0[4], B[4];  // F0[l] = Fhat_0l, B[l] as above (index 1..3)
    for (int l = 1; l <= 3; l++) F0[l] = field_strength(L, c, 0, l);
    {
        M3 f23 = field_strength(L, c, 2, 3);
        M3 f13 = field_strength(L, c, 1, 3);
        M3 f12 = field_strength(L, c, 1, 2);
        B[1] = f23;
        for (int k = 0; k < 9; k++) B[2].a[k] = -f13.a[k];  // Fhat_31 = -Fhat_13
        B[3] = f12;
    }
    double2 *out = (par ? co : ce) + s;
    for (int blk = 0; blk < 2; blk++) {
        M3 Z[3];
        const double sg = blk == 0 ? 1.0 : -1.0;
        for (int l = 1; l <= 3; l++)
            for (int k = 0; k < 9; k++) {
                // upper: c (i/2)(F0l - Bl); lower: -c (i/2)(F0l + Bl)
                const C d = blk == 0 ? F0[l].a[k] - B[l].a[k] : F0[l].a[k] + B[l].a[k];
                Z[l - 1].a[k] = scale(sg * 0.5 * csw, mul_i(d));
            }
        double m[36];
        pack_block(Z, m);
        for (int k = 0; k < 18; k++) out[(long long)(blk * 18 + k) * g.Vh] = make_double2(m[2 * k], m[2 * k + 1]);
    }
}

// inverse of (diag + H) for one packed Hermitian block, by Gauss-Jordan with
// partial pivoting on the full complex 6x6 matrix; returns false if singular
__device__ bool invert_block(const double *m, double diag, double *out)
{
    C A[36], X[36];
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) X[i * 6 + j] = {i == j ? 1.0 : 0.0, 0.0};
    for (int i = 0; i < 6; i++) A[i * 6 + i] = {m[i] + diag, 0.0};
    int k = 6;
    for (int i = 0; i < 6; i++)
        for (int j = i + 1; j < 6; j++) {
            A[i * 6 + j] = {m[k], m[k + 1]};
            A[j * 6 + i] = {m[k], -m[k + 1]};
            k += 2;
        }
    for (int col = 0; col < 6; col++) {
        int piv = col;
        double best = -1;
        for (int r = col; r < 6; r++) {
            const double a = A[r * 6 + col].re * A[r * 6 + col].re + A[r * 6 + col].im * A[r * 6 + col].im;
            if (a > best) {
                best = a;
                piv = r;
            }
        }
        if (!(best > 0) || !isfinite(best)) return false;
        if (piv != col)
            for (int j = 0; j < 6; j++) {
                C t = A[col * 6 + j];
                A[col * 6 + j] = A[piv * 6 + j];
                A[piv * 6 + j] = t;
                t = X[col * 6 + j];
                X[col * 6 + j] = X[piv * 6 + j];
                X[piv * 6 + j] = t;
            }
        const C p = A[col * 6 + col];
        const double den = p.re * p.re + p.im * p.im;
        const C pinv = {p.re / den, -p.im / den};
        for (int j = 0; j < 6; j++) {
            A[col * 6 + j] = cmul(pinv, A[col * 6 + j]);
            X[col * 6 + j] = cmul(pinv, X[col * 6 + j]);
        }
        for (int r = 0; r < 6; r++) {
            if (r == col) continue;
            const C f = A[r * 6 + col];
            for (int j = 0; j < 6; j++) {
                A[r * 6 + j] = A[r * 6 + j] - cmul(f, A[col * 6 + j]);
                X[r * 6 + j] = X[r * 6 + j] - cmul(f, X[col * 6 + j]);
            }
        }
    }
    // the inverse of a Hermitian matrix is Hermitian: pack it (symmetrised)
    for (int i = 0; i < 6; i++) out[i] = X[i * 6 + i].re;
    k = 6;
    for (int i = 0; i < 6; i++)
        for (int j = i + 1; j < 6; j++) {
            out[k++] = 0.5 * (X[i * 6 + j].re + X[j * 6 + i].re);
            out[k++] = 0.5 * (X[i * 6 + j].im - X[j * 6 + i].im);
        }
    for (int q = 0; q < 36; q++)
        if (!isfinite(out[q])) return false;
    return true;
}

__global__ void k_clover_invert(const double2 *cl, long long Vh, double diag, double2 *inv64,
                                float4 *inv32, int *flag)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * Vh) return;
    const int blk = (int)(t / Vh);
    const long long s = t - blk * Vh;
    double m[36], o[36];
    for (int k = 0; k < 18; k++) {
        double2 v = cl[(long long)(blk * 18 + k) * Vh + s];
        m[2 * k] = v.x;
        m[2 * k + 1] = v.y;
    }
    if (!invert_block(m, diag, o)) {
        atomicExch(flag, 1);
        for (int q = 0; q < 36; q++) o[q] = 0;
    }
    for (int k = 0; k < 18; k++) inv64[(long long)(blk * 18 + k) * Vh + s] = make_double2(o[2 * k], o[2 * k + 1]);
    for (int k = 0; k < 9; k++)
        inv32[(long long)(blk * 9 + k) * Vh + s] =
            make_float4((float)o[4 * k], (float)o[4 * k + 1], (float)o[4 * k + 2], (float)o[4 * k + 3]);
}

// out = (diag_g + C_g) in with the packed clover matrix of the RHS's group
// (FP64 spinors, one thread per (site, RHS))
__global__ void k_clover_apply64(const CloverApplyParams p)
{
    const int n = p.nrhs;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long s = gid / n;
    if (s >= p.Vh) return;
    const int r = (int)(gid - s * n);
    const int ms = p.mask_stride > 1 ? p.mask_stride : 1;
    if (p.mask && !p.mask[r * ms]) return;
    const int grp = p.grp_of[r];
    const long long cs = p.Vh * n;
    Cx<double> v[12], w[12];
    load_spinor(static_cast<const double2 *>(p.in) + gid, cs, v);
#pragma unroll
    for (int blk = 0; blk < 2; blk++) {
        double m[36];
        load_clover_block(static_cast<const double2 *>(p.mat[grp]), p.Vh, s, blk, m);
#pragma unroll
        for (int i = 0; i < 6; i++) m[i] += p.diag[grp];
        herm6_apply(m, v + 6 * blk, w + 6 * blk);
    }
    if (p.g5)
#pragma unroll
        for (int j = 6; j < 12; j++) w[j] = -w[j];
    store_spinor(static_cast<double2 *>(p.out) + gid, cs, w);
}

// FP32 spinors on the paired layout, one thread per (site, RHS pair); the
// two RHS of a pair share their group (pairs never straddle a 12-RHS group)
__global__ void k_clover_apply32(const CloverApplyParams p)
{
    const int P = p.nrhs / 2;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long s = gid / P;
    if (s >= p.Vh) return;
    const int q = (int)(gid - s * P);
    const int ms = p.mask_stride > 1 ? p.mask_stride : 1;
    if (p.mask && !p.mask[2 * q * ms] && !p.mask[(2 * q + 1) * ms]) return;
    const int grp = p.grp_of[2 * q];
    const long long cs = p.Vh * P;
    C2 v[12], w[12];
    load_pair(static_cast<const float4 *>(p.in) + gid, cs, v);
#pragma unroll
    for (int blk = 0; blk < 2; blk++) {
        float m[36];
        load_clover_block(static_cast<const float4 *>(p.mat[grp]), p.Vh, s, blk, m);
#pragma unroll
        for (int i = 0; i < 6; i++) m[i] += (float)p.diag[grp];
        herm6_pair(m, v + 6 * blk, w + 6 * blk);
    }
    if (p.g5)
#pragma unroll
        for (int j = 6; j < 12; j++) w[j] = {fneg2(w[j].re), fneg2(w[j].im)};
    store_pair(static_cast<float4 *>(p.out) + gid, cs, w);
}

// The FP64 apply restricted to each RHS's own source site: for a point
// source (mat + diag) in vanishes elsewhere.  One thread per RHS; the caller
// zeroes `out` of the masked RHS beforehand (in and out may alias).
__global__ void k_clover_point64(const CloverApplyParams p, Geom g, const SlotInfo *slots,
                                 int parity)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= p.nrhs) return;
    if (p.mask && !p.mask[r]) return;
    const SlotInfo sl = slots[r];
    if (((sl.t + sl.x + sl.y + sl.z) & 1) != parity) return;
    const long long s = ((((long long)sl.t * g.Lz + sl.z) * g.Ly + sl.y) * g.Lx + sl.x) >> 1;
    const int n = p.nrhs, grp = p.grp_of[r];
    const long long cs = p.Vh * n, me = s * n + r;
    Cx<double> v[12], w[12];
    load_spinor(static_cast<const double2 *>(p.in) + me, cs, v);
#pragma unroll
    for (int blk = 0; blk < 2; blk++) {
        double m[36];
        load_clover_block(static_cast<const double2 *>(p.mat[grp]), p.Vh, s, blk, m);
#pragma unroll
        for (int i = 0; i < 6; i++) m[i] += p.diag[grp];
        herm6_apply(m, v + 6 * blk, w + 6 * blk);
    }
    store_spinor(static_cast<double2 *>(p.out) + me, cs, w);
}

// Per-RHS |(mat + diag) in|^2 of an FP64 spinor with an FP32 clover (mat),
// the product formed in FP32 and the squares summed in FP64: a residual
// report needs a few digits only.  Block = lanes x n RHS (reduce.cuh).
__global__ void __launch_bounds__(kMaxBlock)
    k_clover_norm(Cfg c, const CloverApplyParams p, double *out, double *partials,
                  unsigned int *counter)
{
    const int n = p.nrhs;
    const int r = threadIdx.x % n, lane = threadIdx.x / n;
    const long long cs = p.Vh * n;
    double acc[1] = {0};
    const bool act = !p.mask || p.mask[r];
    const int grp = p.grp_of[r];
    const float dg = (float)p.diag[grp];
    for (long long s = (long long)blockIdx.x * c.lanes + lane; act && s < p.Vh;
         s += (long long)gridDim.x * c.lanes) {
        Cx<double> v[12];
        load_spinor(static_cast<const double2 *>(p.in) + s * n + r, cs, v);
        Cx<float> vf[12], w[12];
#pragma unroll
        for (int k = 0; k < 12; k++) vf[k] = {(float)v[k].re, (float)v[k].im};
#pragma unroll
        for (int blk = 0; blk < 2; blk++) {
            float m[36];
            load_clover_block(static_cast<const float4 *>(p.mat[grp]), p.Vh, s, blk, m);
#pragma unroll
            for (int i = 0; i < 6; i++) m[i] += dg;
            herm6_apply(m, vf + 6 * blk, w + 6 * blk);
        }
        float ss = 0;
#pragma unroll
        for (int k = 0; k < 12; k++) ss = fmx(w[k].re, w[k].re, fmx(w[k].im, w[k].im, ss));
        acc[0] += (double)ss;
    }
    if (!reduce_last<1, 1>(acc, c, partials, counter, n)) return;
    out[r] = acc[0];
}

// FP64 [36 double2][Vh] -> FP32 [18 float4][Vh], same order of the 72 reals
__global__ void k_clover_to_f32(const double2 *in, float4 *out, long long Vh)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= Vh) return;
#pragma unroll
    for (int k = 0; k < 18; k++) {
        const double2 a = in[(long long)(2 * k) * Vh + s], b = in[(long long)(2 * k + 1) * Vh + s];
        out[(long long)k * Vh + s] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
    }
}

}  // namespace

cudaError_t launch_clover_to_f32(const double2 *in, float4 *out, long long Vh, cudaStream_t st)
{
    k_clover_to_f32<<<(unsigned)((Vh + 127) / 128), 128, 0, st>>>(in, out, Vh);
    return cudaGetLastError();
}

cudaError_t launch_clover_build(const double2 *links64_e, const double2 *links64_o,
                                const Geom &g, double csw, double2 *clov_e, double2 *clov_o,
                                cudaStream_t st)
{
    LinkView L;
    L.l[0] = links64_e;
    L.l[1] = links64_o;
    L.g = g;
    const int block = 128;
    k_clover_build<<<(unsigned)((g.V + block - 1) / block), block, 0, st>>>(L, csw, clov_e, clov_o);
    return cudaGetLastError();
}

cudaError_t launch_clover_invert(const double2 *clov, long long Vh, double M, double2 *inv64,
                                 float4 *inv32, int *flag, cudaStream_t st)
{
    const int block = 128;
    k_clover_invert<<<(unsigned)((2 * Vh + block - 1) / block), block, 0, st>>>(clov, Vh, 4.0 + M,
                                                                               inv64, inv32, flag);
    return cudaGetLastError();
}

cudaError_t launch_clover_point(const CloverApplyParams &p, const Geom &g, const SlotInfo *slots,
                                int parity, cudaStream_t st)
{
    k_clover_point64<<<1, kMaxRhs, 0, st>>>(p, g, slots, parity);
    return cudaGetLastError();
}

cudaError_t launch_clover_norm(BlasCtx &bc, const CloverApplyParams &p, double *out_dev,
                               cudaStream_t st)
{
    const Cfg c = cfg_wave(bc, k_clover_norm, p.Vh, p.nrhs);
    k_clover_norm<<<c.grid, c.block, 0, st>>>(c, p, out_dev, bc.partials, bc.counter);
    return cudaGetLastError();
}

cudaError_t launch_clover_apply(const CloverApplyParams &p, int prec, cudaStream_t st)
{
    const int block = 128;
    if (prec == 0) {
        const unsigned grid = (unsigned)((p.Vh * p.nrhs + block - 1) / block);
        k_clover_apply64<<<grid, block, 0, st>>>(p);
    } else {
        if (p.nrhs % 2) return cudaErrorInvalidValue;
        const unsigned grid = (unsigned)((p.Vh * (p.nrhs / 2) + block - 1) / block);
        k_clover_apply32<<<grid, block, 0, st>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace dp
