// Gauge-field packing, spinor packing, the point source and the
// restore-and-contract step of the method.
//
//  * links: lexicographic complex128 -> even-odd site-blocked SoA per parity
//    and direction, FP64 (18 reals), FP32 (18 reals) and FP32 12-real (rows 0
//    and 1 only; row 2 is rebuilt in the dslash from unitarity).
//  * point source (Sec. I, eq. linsysunprec with a source on one time slice;
//    Sec. II eq. redeft): eta' = alpha_B(x_src) delta_{x,x_src} e_k.
//  * restore and contract (Sec. II eq. backcorrection, Sec. III): S = S'/alpha_B
//    per site, C_PP(y0) = -sum_{y vec} sum_k |S_k(y)|^2, y0 relative to the
//    source, reduced per time slice in a fixed order (deterministic).
#include "cplx.cuh"
#include "dp_internal.h"

namespace dp {
namespace {

__device__ __forceinline__ void coords_full(const Geom &g, long long i, int &t, int &x, int &y,
                                            int &z)
{
    x = (int)(i % g.Lx);
    i /= g.Lx;
    y = (int)(i % g.Ly);
    i /= g.Ly;
    z = (int)(i % g.Lz);
    t = (int)(i / g.Lz);
}

__global__ void k_pack_links(const double2 *lex, Geom g, double2 *l64e, double2 *l64o,
                             float2 *l32fe, float2 *l32fo, float4 *l32ce, float4 *l32co)
{
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= g.V * 4) return;
    const long long i = gid >> 2;
    const int mu = (int)(gid & 3);
    int t, x, y, z;
    coords_full(g, i, t, x, y, z);
    const int par = (t + x + y + z) & 1;
    const long long s = i >> 1;
    const double2 *u = lex + (i * 4 + mu) * 9;
    double2 *o64 = (par ? l64o : l64e) + (long long)mu * 9 * g.Vh + s;
    // FP32 18-real: entries 0-7 as float4 [mu][4][s], entry 8 as float2 [mu][s]
    float4 *o32 = reinterpret_cast<float4 *>(par ? l32fo : l32fe) + (long long)mu * 4 * g.Vh + s;
    float2 *o32t = reinterpret_cast<float2 *>(reinterpret_cast<float4 *>(par ? l32fo : l32fe) + 16 * g.Vh) +
                   (long long)mu * g.Vh + s;
    float4 *oc = (par ? l32co : l32ce) + (long long)mu * 3 * g.Vh + s;
    double2 v[9];
#pragma unroll
    for (int k = 0; k < 9; k++) v[k] = u[k];
#pragma unroll
    for (int k = 0; k < 9; k++) o64[k * g.Vh] = v[k];
#pragma unroll
    for (int k = 0; k < 4; k++)
        o32[k * g.Vh] = make_float4((float)v[2 * k].x, (float)v[2 * k].y, (float)v[2 * k + 1].x,
                                    (float)v[2 * k + 1].y);
    o32t[0] = make_float2((float)v[8].x, (float)v[8].y);
#pragma unroll
    for (int k = 0; k < 3; k++)
        oc[k * g.Vh] = make_float4((float)v[2 * k].x, (float)v[2 * k].y, (float)v[2 * k + 1].x,
                                   (float)v[2 * k + 1].y);
}

// FP64 links of one parity -> rows 0, 1 in 16-bit with one FP32 scale per link
template <typename H2>
__device__ __forceinline__ unsigned f2h(float a, float b);
template <>
__device__ __forceinline__ unsigned f2h<__half2>(float a, float b)
{
    const __half2 h = __floats2half2_rn(a, b);
    unsigned v;
    memcpy(&v, &h, 4);
    return v;
}
template <>
__device__ __forceinline__ unsigned f2h<__nv_bfloat162>(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    unsigned v;
    memcpy(&v, &h, 4);
    return v;
}

template <typename H2>
__global__ void k_pack_links16(const double2 *l64, long long Vh, void *out)
{
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= Vh * 4) return;
    const int mu = (int)(gid / Vh);
    const long long s = gid - (long long)mu * Vh;
    double2 v[6];
    double mx = 0;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        v[k] = l64[((long long)mu * 9 + k) * Vh + s];
        mx = fmax(mx, fmax(fabs(v[k].x), fabs(v[k].y)));
    }
    const float sc = mx > 0 ? (float)mx : 1.0f;
    const double inv = 1.0 / sc;
    uint2 *o = static_cast<uint2 *>(out) + (long long)mu * 3 * Vh + s;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const double2 a = v[2 * k], b = v[2 * k + 1];
        o[k * Vh] = make_uint2(f2h<H2>((float)(a.x * inv), (float)(a.y * inv)),
                               f2h<H2>((float)(b.x * inv), (float)(b.y * inv)));
    }
    reinterpret_cast<float *>(static_cast<uint2 *>(out) + 12 * Vh)[(long long)mu * Vh + s] = sc;
}

// one thread per (full site, rhs)
__global__ void k_pack_spinor(const double2 *lex, Geom g, int n, int prec, void *ev, void *od)
{
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= g.V * n) return;
    const long long i = gid % g.V;
    const int r = (int)(gid / g.V);
    int t, x, y, z;
    coords_full(g, i, t, x, y, z);
    const int par = (t + x + y + z) & 1;
    const long long s = i >> 1;
    const double2 *src = lex + ((long long)r * g.V + i) * 12;
    const long long cs = g.Vh * n, me = s * n + r;
    if (prec == 0) {
        double2 *o = static_cast<double2 *>(par ? od : ev) + me;
#pragma unroll
        for (int k = 0; k < 12; k++) o[k * cs] = src[k];
    } else {
        // paired FP32 layout: float4 (re_2q, re_2q+1, im_2q, im_2q+1) at (k*Vh + s)*n/2 + q
        float *o = reinterpret_cast<float *>(static_cast<float4 *>(par ? od : ev));
        const int P = n / 2, q = r >> 1, L = r & 1;
        const long long csp = g.Vh * P;
#pragma unroll
        for (int k = 0; k < 12; k++) {
            float *f = o + 4 * (k * csp + s * P + q);
            f[L] = (float)src[k].x;
            f[2 + L] = (float)src[k].y;
        }
    }
}

__global__ void k_unpack_spinor(const void *ev, const void *od, Geom g, int n, int prec,
                                double2 *lex)
{
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= g.V * n) return;
    const long long i = gid % g.V;
    const int r = (int)(gid / g.V);
    int t, x, y, z;
    coords_full(g, i, t, x, y, z);
    const int par = (t + x + y + z) & 1;
    const long long s = i >> 1;
    double2 *dst = lex + ((long long)r * g.V + i) * 12;
    const long long cs = g.Vh * n, me = s * n + r;
    if (prec == 0) {
        const double2 *o = static_cast<const double2 *>(par ? od : ev) + me;
#pragma unroll
        for (int k = 0; k < 12; k++) dst[k] = o[k * cs];
    } else {
        const float *o = reinterpret_cast<const float *>(static_cast<const float4 *>(par ? od : ev));
        const int P = n / 2, q = r >> 1, L = r & 1;
        const long long csp = g.Vh * P;
#pragma unroll
        for (int k = 0; k < 12; k++) {
            const float *f = o + 4 * (k * csp + s * P + q);
            dst[k] = make_double2(f[L], f[2 + L]);
        }
    }
}

__global__ void k_point_source(Geom g, const SlotInfo *slots, int n, const int *mask, double2 *ev,
                               double2 *od)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    if (mask && !mask[k]) return;
    const SlotInfo sl = slots[k];
    const int par = (sl.t + sl.x + sl.y + sl.z) & 1;
    const long long s = ((((long long)sl.t * g.Lz + sl.z) * g.Ly + sl.y) * g.Lx + sl.x) >> 1;
    double2 *b = par ? od : ev;
    b[((long long)sl.comp * g.Vh + s) * n + k] = make_double2(sl.scale, 0.0);
}

constexpr int kContractBlock = 256;

// grid (P, T): block (p, t) sums |S'|^2/alpha_B^2 over its share of slice t,
// per group; partials[(t*P + p)*ng + grp].  With `ap`, also the gamma_0
// bilinear tr[gamma_0 S S^dag] (chiral basis: gamma_0 = -1 between spins 0,2
// and 1,3, i.e. -2 Re sum_c [S(0,c) S(2,c)* + S(1,c) S(3,c)*] per RHS) into
// partials[T*P*ng + (t*P + p)*ng + grp]
__global__ void __launch_bounds__(kContractBlock)
    k_contract(const double2 *xe, const double2 *xo, Geom g, int n, const double *alpha,
               const SlotInfo *slots, const int *mask, int ng, double *partials, double2 *prop,
               int ap)
{
    const int P = gridDim.x, p = blockIdx.x, t = blockIdx.y;
    const long long Vs = g.Vh / g.T;  // half-sites per slice per parity
    const long long chunk = (Vs + P - 1) / P;
    const long long j0 = p * chunk, j1 = min(Vs, j0 + chunk);
    const int nm = ng;
    const long long cs = g.Vh * n;
    double loc[kMaxGroups], lap[kMaxGroups];
    for (int m = 0; m < kMaxGroups; m++) loc[m] = lap[m] = 0;
    const long long work = (j1 > j0 ? j1 - j0 : 0) * n;
    for (long long e = threadIdx.x; e < work; e += blockDim.x) {
        const long long s = (long long)t * Vs + j0 + e / n;
        const int r = (int)(e % n);
        if (mask && !mask[r]) continue;
        const int xh = (int)(s % g.Lxh);
        long long q = s / g.Lxh;
        const int y = (int)(q % g.Ly);
        q /= g.Ly;
        const int z = (int)(q % g.Lz);
        const int grp = slots[r].group;
        const double *al = alpha + (long long)grp * 4 * g.Lmax;
        const double base = al[0 * g.Lmax + t] * al[2 * g.Lmax + y] * al[3 * g.Lmax + z];
        double acc = 0, acc_ap = 0;
        for (int par = 0; par < 2; par++) {
            const int x = 2 * xh + ((t + y + z + par) & 1);
            const double inv = 1.0 / (base * al[1 * g.Lmax + x]);
            const double2 *v = (par ? xo : xe) + s * n + r;
            double2 *pd = prop ? prop + ((long long)r * g.V + 2 * s + (x & 1)) * 12 : nullptr;
            double sp = 0;
            double2 c[12];
            for (int k = 0; k < 12; k++) {
                c[k] = v[k * cs];
                c[k].x *= inv;
                c[k].y *= inv;
                sp = fmx(c[k].x, c[k].x, sp);
                sp = fmx(c[k].y, c[k].y, sp);
                if (pd) pd[k] = c[k];
            }
            acc += sp;
            if (ap) {
                double b = 0;  // Re sum_c [S(0,c) S(2,c)* + S(1,c) S(3,c)*]
                for (int k = 0; k < 6; k++) {
                    b = fmx(c[k].x, c[k + 6].x, b);
                    b = fmx(c[k].y, c[k + 6].y, b);
                }
                acc_ap -= 2.0 * b;
            }
        }
#pragma unroll
        for (int m = 0; m < kMaxGroups; m++)
            if (m == grp) {
                loc[m] += acc;
                lap[m] += acc_ap;
            }
    }
    __shared__ double sh[kContractBlock];
    for (int m = 0; m < nm; m++) {
        sh[threadIdx.x] = loc[m];
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) partials[((long long)t * P + p) * nm + m] = sh[0];
        __syncthreads();
        if (!ap) continue;
        sh[threadIdx.x] = lap[m];
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0)
            partials[(long long)g.T * P * nm + ((long long)t * P + p) * nm + m] = sh[0];
        __syncthreads();
    }
}

// cpp[m][(t - t_src[m]) mod T] = -sum_p partials[t][p][m], summed in p order;
// cap (if non-null) from the second half of partials, with a + sign
__global__ void k_contract_final(const double *partials, int P, int T, int nm, const int *t_src,
                                 double *cpp, double *cap)
{
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= T * nm) return;
    const int t = id / nm, m = id % nm;
    double s = 0;
    for (int p = 0; p < P; p++) s += partials[((long long)t * P + p) * nm + m];
    const int rel = ((t - t_src[m]) % T + T) % T;
    cpp[m * T + rel] = -s;
    if (cap) {
        const double *pa = partials + (long long)T * P * nm;
        double a = 0;
        for (int p = 0; p < P; p++) a += pa[((long long)t * P + p) * nm + m];
        cap[m * T + rel] = a;
    }
}

// grid (P, T): the heavy-light bilinear sum_{k, j} S_h(k, j) conj(S_l(k, j))
// over block p's share of slice t (j: the 12 source components, k: sink spin
// and colour), each propagator restored by its own group's profile;
// partials[((t*P + p)) * 2 + {0: re, 1: im}]
__global__ void __launch_bounds__(kContractBlock)
    k_contract_hl(const double2 *xe, const double2 *xo, Geom g, int n, const double *alpha, int gh,
                  int gl, int sh, int sl, double *partials)
{
    const int P = gridDim.x, p = blockIdx.x, t = blockIdx.y;
    const long long Vs = g.Vh / g.T;
    const long long chunk = (Vs + P - 1) / P;
    const long long j0 = p * chunk, j1 = min(Vs, j0 + chunk);
    const long long cs = g.Vh * n;
    const double *ah = alpha + (long long)gh * 4 * g.Lmax, *al = alpha + (long long)gl * 4 * g.Lmax;
    double re = 0, im = 0;
    const long long work = (j1 > j0 ? j1 - j0 : 0) * 12;
    for (long long e = threadIdx.x; e < work; e += blockDim.x) {
        const long long s = (long long)t * Vs + j0 + e / 12;
        const int j = (int)(e % 12);
        const int xh = (int)(s % g.Lxh);
        long long q = s / g.Lxh;
        const int y = (int)(q % g.Ly);
        q /= g.Ly;
        const int z = (int)(q % g.Lz);
        const double bh = ah[0 * g.Lmax + t] * ah[2 * g.Lmax + y] * ah[3 * g.Lmax + z];
        const double bl = al[0 * g.Lmax + t] * al[2 * g.Lmax + y] * al[3 * g.Lmax + z];
        for (int par = 0; par < 2; par++) {
            const int x = 2 * xh + ((t + y + z + par) & 1);
            const double inv = 1.0 / (bh * ah[1 * g.Lmax + x] * bl * al[1 * g.Lmax + x]);
            const double2 *vh = (par ? xo : xe) + s * n + sh + j;
            const double2 *vl = (par ? xo : xe) + s * n + sl + j;
            double sr = 0, si = 0;
            for (int k = 0; k < 12; k++) {
                const double2 a = vh[k * cs], b = vl[k * cs];
                sr = fmx(a.x, b.x, fmx(a.y, b.y, sr));
                si = fmx(a.y, b.x, fmx(-a.x, b.y, si));
            }
            re += sr * inv;
            im += si * inv;
        }
    }
    __shared__ double sh_re[kContractBlock], sh_im[kContractBlock];
    sh_re[threadIdx.x] = re;
    sh_im[threadIdx.x] = im;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sh_re[threadIdx.x] += sh_re[threadIdx.x + w];
            sh_im[threadIdx.x] += sh_im[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[((long long)t * P + p) * 2] = sh_re[0];
        partials[((long long)t * P + p) * 2 + 1] = sh_im[0];
    }
}

// out[2 rel + {0, 1}] = -(re, im) summed over p in order, rel = (t - t_src) mod T
__global__ void k_contract_hl_final(const double *partials, int P, int T, int t_src, double *out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    double re = 0, im = 0;
    for (int p = 0; p < P; p++) {
        re += partials[((long long)t * P + p) * 2];
        im += partials[((long long)t * P + p) * 2 + 1];
    }
    const int rel = ((t - t_src) % T + T) % T;
    out[2 * rel] = -re;
    out[2 * rel + 1] = -im;
}

__global__ void k_cpp_commit(const double *src, double *dst, int T, int accumulate)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= T) return;
    dst[k] = accumulate ? dst[k] + src[k] : src[k];
}

}  // namespace

cudaError_t launch_pack_links(const double2 *lex, const Geom &g, double2 *l64[2], float2 *l32f[2],
                              float4 *l32c[2], cudaStream_t st)
{
    const int block = 128;
    const long long n = g.V * 4;
    k_pack_links<<<(unsigned)((n + block - 1) / block), block, 0, st>>>(
        lex, g, l64[0], l64[1], l32f[0], l32f[1], l32c[0], l32c[1]);
    return cudaGetLastError();
}

cudaError_t launch_pack_links16(const double2 *l64, long long Vh, int fmt, void *out,
                                cudaStream_t st)
{
    const int block = 128;
    const unsigned grid = (unsigned)((Vh * 4 + block - 1) / block);
    if (fmt == LINK_H16_12)
        k_pack_links16<__half2><<<grid, block, 0, st>>>(l64, Vh, out);
    else if (fmt == LINK_B16_12)
        k_pack_links16<__nv_bfloat162><<<grid, block, 0, st>>>(l64, Vh, out);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_pack_spinor(const double2 *lex, const Geom &g, int nrhs, int prec,
                               void *even, void *odd, cudaStream_t st)
{
    const int block = 128;
    const long long n = g.V * nrhs;
    k_pack_spinor<<<(unsigned)((n + block - 1) / block), block, 0, st>>>(lex, g, nrhs, prec, even,
                                                                         odd);
    return cudaGetLastError();
}

cudaError_t launch_unpack_spinor(const void *even, const void *odd, const Geom &g, int nrhs,
                                 int prec, double2 *lex, cudaStream_t st)
{
    const int block = 128;
    const long long n = g.V * nrhs;
    k_unpack_spinor<<<(unsigned)((n + block - 1) / block), block, 0, st>>>(even, odd, g, nrhs,
                                                                           prec, lex);
    return cudaGetLastError();
}

cudaError_t launch_point_source(const Geom &g, const SlotInfo *slots_dev, int nrhs,
                                const int *mask, double2 *even, double2 *odd, cudaStream_t st)
{
    k_point_source<<<1, kMaxRhs, 0, st>>>(g, slots_dev, nrhs, mask, even, odd);
    return cudaGetLastError();
}

cudaError_t launch_contract_hl(const double2 *xe, const double2 *xo, const Geom &g, int nrhs,
                               const double *alpha, int gh, int gl, int slot_h, int slot_l, int t_src,
                               double *partials, double *out_dev, cudaStream_t st)
{
    const int P = contract_blocks_per_slice(g);
    dim3 grid(P, g.T);
    k_contract_hl<<<grid, kContractBlock, 0, st>>>(xe, xo, g, nrhs, alpha, gh, gl, slot_h, slot_l,
                                                   partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_contract_hl_final<<<(g.T + 127) / 128, 128, 0, st>>>(partials, P, g.T, t_src, out_dev);
    return cudaGetLastError();
}

// partials must hold T * P * n_mass doubles, P = contract_blocks_per_slice(g)
int contract_blocks_per_slice(const Geom &g)
{
    const long long Vs = g.Vh / g.T;
    long long P = (Vs + 1023) / 1024;
    if (P < 1) P = 1;
    if (P > 64) P = 64;
    return (int)P;
}

cudaError_t launch_restore_contract(const double2 *xe, const double2 *xo, const Geom &g, int nrhs,
                                    const double *alpha, const SlotInfo *slots_dev, int ngroups,
                                    const int *t_src_dev, const int *mask, double *cpp_dev,
                                    double *partials, double2 *prop_lex, cudaStream_t st,
                                    double *cap_dev)
{
    if (ngroups < 1 || ngroups > kMaxGroups) return cudaErrorInvalidValue;
    const int P = contract_blocks_per_slice(g);
    dim3 grid(P, g.T);
    k_contract<<<grid, kContractBlock, 0, st>>>(xe, xo, g, nrhs, alpha, slots_dev, mask, ngroups,
                                                partials, prop_lex, cap_dev ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int tot = g.T * ngroups;
    k_contract_final<<<(tot + 127) / 128, 128, 0, st>>>(partials, P, g.T, ngroups, t_src_dev, cpp_dev,
                                                         cap_dev);
    return cudaGetLastError();
}

cudaError_t launch_cpp_commit(const double *src, double *dst, int T, int accumulate, cudaStream_t st)
{
    k_cpp_commit<<<(T + 127) / 128, 128, 0, st>>>(src, dst, T, accumulate);
    return cudaGetLastError();
}

// ---- allocation-free restore and contract -----------------------------------
//
// dp_restore_contract_noalloc runs the same two kernels as
// dp_restore_contract_dev, but its device scratch (profile tables, slot
// descriptors and the per-slice partial sums) lives in one file-scope device
// array instead of memory from the context allocator.  Layout of the array
// (256-byte aligned regions):
//   partials  kNaMaxT * kNaMaxP * kNaMaxGroups doubles   (1 MiB)
//   alpha     kNaMaxGroups * 4 * kMaxL doubles            (64 KiB)
//   slots     kMaxRhs SlotInfo
//   t_src     kNaMaxGroups ints
constexpr int kNaMaxT = kMaxL;
constexpr int kNaMaxP = 64;
constexpr int kNaMaxGroups = kMaxGroups;
constexpr size_t kNaAlign = 256;
constexpr size_t na_round(size_t b) { return (b + kNaAlign - 1) / kNaAlign * kNaAlign; }
constexpr size_t kNaPartOff = 0;
constexpr size_t kNaAlphaOff = kNaPartOff + na_round(sizeof(double) * kNaMaxT * kNaMaxP * kNaMaxGroups);
constexpr size_t kNaSlotOff = kNaAlphaOff + na_round(sizeof(double) * kNaMaxGroups * 4 * kMaxL);
constexpr size_t kNaTsrcOff = kNaSlotOff + na_round(sizeof(SlotInfo) * kMaxRhs);
constexpr size_t kNaBytes = kNaTsrcOff + na_round(sizeof(int) * kNaMaxGroups);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

size_t noalloc_scratch_bytes() { return kNaBytes; }

}  // namespace dp

#include <mutex>

#include "ctx.h"

namespace {
// Device address of g_noalloc_scratch per device.  In host code the array's
// name only stands in for the symbol; the address a kernel may use is looked
// up once per device with that device current.  A device reset destroys the
// module that holds the array, so the address is forgotten whenever a context
// is created on that device (every context there is invalid after a reset and
// has to be created again) and looked up anew on the next call.
constexpr int kNaMaxDevices = 64;
std::mutex g_na_mu;
void *g_na_addr[kNaMaxDevices] = {};

// host-side tables of one call: per thread, outside the caller's stack
// (about 82 KiB), allocated once per thread by the loader, not per call
thread_local double t_na_alpha[dp::kMaxGroups * 4 * dp::kMaxL];
thread_local double t_na_hop[8 * dp::kMaxL];
thread_local dp::SlotInfo t_na_slots[dp::kMaxRhs];

dp_status noalloc_scratch_address(int device, unsigned char **out)
{
    if (device < 0 || device >= kNaMaxDevices) {
        dp::set_error("device index %d beyond the %d supported", device, kNaMaxDevices);
        return DP_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, dp::g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            dp::set_error("cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
            return DP_ERR_CUDA;
        }
        g_na_addr[device] = p;
    }
    *out = static_cast<unsigned char *>(g_na_addr[device]);
    return DP_OK;
}
}  // namespace

namespace dp {
void noalloc_forget_address(int device)
{
    if (device < 0 || device >= kNaMaxDevices) return;
    std::lock_guard<std::mutex> lk(g_na_mu);
    g_na_addr[device] = nullptr;
}
}  // namespace dp

extern "C" dp_status dp_restore_contract_noalloc(dp_ctx *ctx, dp_field field, int n_groups,
                                                 const dp_profile *profiles, const int *src,
                                                 const double *xe, const double *xo,
                                                 double *cpp_dev)
{
    using namespace dp;
    if (!ctx) {
        set_error("null context");
        return DP_ERR_INVALID_ARG;
    }
    Ctx &c = ctx->c;
    if (cudaSetDevice(c.device) != cudaSuccess) {
        set_error("cudaSetDevice(%d) failed", c.device);
        return DP_ERR_CUDA;
    }
    auto fp = find_field(&c, field);
    if (!fp) {
        set_error("unknown field");
        return DP_ERR_NOT_FOUND;
    }
    constexpr int kNaGroupsMax = kMaxRhs / 12 < kNaMaxGroups ? kMaxRhs / 12 : kNaMaxGroups;
    if (n_groups < 1 || n_groups > kNaGroupsMax || !profiles || !src || !xe || !xo || !cpp_dev) {
        set_error("dp_restore_contract_noalloc: invalid argument (n_groups in [1, %d]: %d RHS "
                  "slots of 12, scratch for %d groups; non-null pointers)",
                  kNaGroupsMax, kMaxRhs, kNaMaxGroups);
        return DP_ERR_INVALID_ARG;
    }
    const Geom &g = fp->g;
    const int P = contract_blocks_per_slice(g);
    if (g.T > kNaMaxT || P > kNaMaxP || g.Lmax > kMaxL) {
        set_error("lattice beyond the fixed scratch of dp_restore_contract_noalloc "
                  "(T <= %d, %d partial sums per slice, extents <= %d)", kNaMaxT, kNaMaxP, kMaxL);
        return DP_ERR_INVALID_ARG;
    }
    unsigned char *base = nullptr;
    dp_status s = noalloc_scratch_address(c.device, &base);
    if (s != DP_OK) return s;
    double *alpha = t_na_alpha, *hop = t_na_hop;
    SlotInfo *slots = t_na_slots;
    int tsrc[kNaMaxGroups] = {};
    const int Lm = g.Lmax, n = 12 * n_groups;
    const int L[4] = {g.T, g.Lx, g.Ly, g.Lz};
    for (int k = 0; k < n_groups; k++) {
        for (int mu = 0; mu < 4; mu++)
            if (src[4 * k + mu] < 0 || src[4 * k + mu] >= L[mu]) {
                set_error("source coordinate out of range");
                return DP_ERR_INVALID_ARG;
            }
        s = profile_tables(profiles[k], g, fp->bc_t, src + 4 * k, alpha + (size_t)k * 4 * Lm, hop);
        if (s != DP_OK) return s;
        tsrc[k] = src[4 * k];
        for (int j = 0; j < 12; j++) {
            SlotInfo &sl = slots[12 * k + j];
            sl.group = k;
            sl.comp = j;
            sl.t = src[4 * k];
            sl.x = src[4 * k + 1];
            sl.y = src[4 * k + 2];
            sl.z = src[4 * k + 3];
            sl.scale = 1.0;
        }
    }
    double *part_d = reinterpret_cast<double *>(base + kNaPartOff);
    double *alpha_d = reinterpret_cast<double *>(base + kNaAlphaOff);
    SlotInfo *slots_d = reinterpret_cast<SlotInfo *>(base + kNaSlotOff);
    int *tsrc_d = reinterpret_cast<int *>(base + kNaTsrcOff);
    // every partial sum the final kernel reads is written earlier in the same
    // call, so nothing in the shared array has to be cleared first
    cudaError_t e = cudaMemcpyAsync(alpha_d, alpha, sizeof(double) * n_groups * 4 * Lm,
                                    cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(slots_d, slots, sizeof(SlotInfo) * n, cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tsrc_d, tsrc, sizeof(int) * n_groups, cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) {
        dim3 grid(P, g.T);
        k_contract<<<grid, kContractBlock, 0, c.stream>>>((const double2 *)xe, (const double2 *)xo, g, n,
                                                          alpha_d, slots_d, nullptr, n_groups, part_d,
                                                          nullptr, 0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const int tot = g.T * n_groups;
        k_contract_final<<<(tot + 127) / 128, 128, 0, c.stream>>>(part_d, P, g.T, n_groups, tsrc_d, cpp_dev,
                                                                   nullptr);
        e = cudaGetLastError();
    }
    // the host tables are reused by this thread's next call: wait for the
    // copies (and the kernels) before returning
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) {
        set_error("restore/contract (no-alloc): %s", cudaGetErrorString(e));
        return DP_ERR_CUDA;
    }
    c.launches += 2;
    return DP_OK;
}
