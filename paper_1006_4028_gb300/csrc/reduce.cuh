// Deterministic per-RHS grid reductions shared by the BLAS-1 kernels.
//
// A block is `lanes` sites x `units` threads, thread t = lane*units + unit;
// a unit is one RHS (FP64) or one RHS pair (FP32 paired layout, LANES = 2).
// Each thread passes per-RHS partial sums (FP64); the block sums them over
// its lanes in a fixed tree, writes one partial per RHS to global scratch,
// and the last block to finish (atomic ticket) sums the block partials in a
// fixed order.  The result for an RHS never depends on the other RHS.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>

#include "dp_internal.h"

namespace dp {

constexpr int kMaxBlock = 512;

struct Cfg {
    int lanes, block, grid;
};

inline Cfg cfg_for(long long Vh, int units, int max_grid)
{
    Cfg c;
    c.lanes = 256;
    while (c.lanes * units > kMaxBlock && c.lanes > 1) c.lanes >>= 1;
    c.block = c.lanes * units;
    long long g = (Vh + c.lanes - 1) / c.lanes;
    if (g > max_grid) g = max_grid;
    if (g < 1) g = 1;
    c.grid = (int)g;
    return c;
}

// Grid of a grid-stride reduction: one full wave (resident blocks per SM x
// SMs, from the occupancy calculator), so no partial second wave idles the
// machine at the end; never more blocks than the scratch holds.
template <typename K>
inline int one_wave(K kernel, int block, int cap)
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

template <typename K>
inline Cfg cfg_wave(const BlasCtx &bc, K kernel, long long Vh, int units)
{
    Cfg c = cfg_for(Vh, units, bc.blocks);
    c.grid = std::min(c.grid, one_wave(kernel, c.block, bc.blocks));
    return c;
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

// ---- per-RHS BiCGStab scalar recurrences, applied by the last block ----------

// alpha = rho / <rhat, v>
__device__ __forceinline__ void finish_alpha(RhsState &S, double re, double im)
{
    if (!S.active) return;
    const double2 rv = make_double2(re, im);
    if (!zfinite(rv)) {
        S.status = 3;
        S.active = 0;
    } else if (rv.x == 0.0 && rv.y == 0.0) {
        S.status = 2;
        S.active = 0;
    } else {
        S.alpha = zdiv(S.rho, rv);
    }
}

// omega = <t, s> / <t, t>
__device__ __forceinline__ void finish_omega(RhsState &S, double re, double im, double tt)
{
    if (!S.active) return;
    if (!(isfinite(re) && isfinite(im) && isfinite(tt))) {
        S.status = 3;
        S.active = 0;
        return;
    }
    S.omega = tt > 0 ? make_double2(re / tt, im / tt) : make_double2(0.0, 0.0);
}

// FP32 BiCGStab with the shadow image rhat' = Mhat^dag rhat: the s pass keeps
// <rhat, s> and <rhat', s> (= <rhat, t>) for the omega step
__device__ __forceinline__ void finish_s_dots(RhsState &S, double rs_re, double rs_im, double rt_re,
                                              double rt_im)
{
    if (!S.active) return;
    S.rs = make_double2(rs_re, rs_im);
    S.rt = make_double2(rt_re, rt_im);
    if (!(zfinite(S.rs) && zfinite(S.rt))) {
        S.status = 3;
        S.active = 0;
    }
}

// omega = <t, s>/|t|^2 from the x - A^-1 D epilogue's sums, rho' = <rhat, s> -
// omega <rhat', s>, beta = (rho'/rho)(alpha/omega); a breakdown is flagged
// for the update pass (finish_update_rr)
__device__ __forceinline__ void finish_omega_shadow(RhsState &S, double ts_re, double ts_im, double tt)
{
    if (!S.active) return;
    if (!(isfinite(ts_re) && isfinite(ts_im) && isfinite(tt))) {
        S.status = 3;
        S.active = 0;
        return;
    }
    S.omega = tt > 0 ? make_double2(ts_re / tt, ts_im / tt) : make_double2(0.0, 0.0);
    const double2 wrt = zmul(S.omega, S.rt);
    const double2 rho_new = make_double2(S.rs.x - wrt.x, S.rs.y - wrt.y);
    if ((S.omega.x == 0.0 && S.omega.y == 0.0) || (rho_new.x == 0.0 && rho_new.y == 0.0)) {
        S.brk = 1;
        S.beta = make_double2(0.0, 0.0);
    } else {
        S.beta = zmul(zdiv(rho_new, S.rho), zdiv(S.alpha, S.omega));
        S.rho = rho_new;
    }
}

// iteration count, convergence, cap, breakdown; beta = (rho'/rho)(alpha/omega)
__device__ __forceinline__ void finish_update(RhsState &S, double re, double im, double rr,
                                              int max_iter)
{
    if (!S.active) return;
    S.iters++;
    const double2 rho_new = make_double2(re, im);
    S.rr = rr;
    if (!(zfinite(rho_new) && isfinite(rr))) {
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

// iteration count, convergence, cap, and a breakdown flagged by
// finish_omega_shadow
__device__ __forceinline__ void finish_update_rr(RhsState &S, double rr, int max_iter)
{
    if (!S.active) return;
    S.iters++;
    S.rr = rr;
    if (!isfinite(rr)) {
        S.status = 3;
        S.active = 0;
    } else if (S.rr <= S.tol2) {
        S.status = 1;
        S.active = 0;
    } else if (S.iters >= max_iter) {
        S.status = 4;
        S.active = 0;
    } else if (S.brk) {
        S.status = 2;
        S.active = 0;
    }
}

// start of an inner solve: rho = |r|^2, tol2 (tol^2 on entry) *= |r|^2
__device__ __forceinline__ void finish_init(RhsState &S, double bb)
{
    if (!S.active) return;
    S.rr = bb;
    S.bb = bb;
    S.tol2 = S.tol2 * bb;
    S.rho = make_double2(bb, 0.0);
    S.alpha = make_double2(1.0, 0.0);
    S.omega = make_double2(1.0, 0.0);
    S.beta = make_double2(0.0, 0.0);
    S.iters = 0;
    S.brk = 0;
    if (!isfinite(bb)) {
        S.status = 3;
        S.active = 0;
    } else if (bb <= S.tol2) {
        S.status = 1;
        S.active = 0;
    }
}

// ---- per-RHS CGNE scalar recurrences (real, in the .x parts) ----------------

// rho' = |Mhat^dag r|^2; beta = rho'/rho (first iteration: 0)
__device__ __forceinline__ void finish_cg_gamma(RhsState &S, double zz, int first)
{
    if (!S.active) return;
    if (!isfinite(zz)) {
        S.status = 3;
        S.active = 0;
    } else if (zz == 0.0) {  // Mhat^dag r = 0 with r != 0: singular operator
        S.status = 2;
        S.active = 0;
    } else {
        S.beta = make_double2(first ? 0.0 : zz / S.rho.x, 0.0);
        S.rho = make_double2(zz, 0.0);
    }
}

// alpha = rho / |Mhat p|^2
__device__ __forceinline__ void finish_cg_alpha(RhsState &S, double ww)
{
    if (!S.active) return;
    if (!isfinite(ww)) {
        S.status = 3;
        S.active = 0;
    } else if (ww == 0.0) {
        S.status = 2;
        S.active = 0;
    } else {
        S.alpha = make_double2(S.rho.x / ww, 0.0);
    }
}

// iteration count and the stop rules on |r|^2 (the Mhat residual)
__device__ __forceinline__ void finish_cg_update(RhsState &S, double rr, int max_iter)
{
    if (!S.active) return;
    S.iters++;
    S.rr = rr;
    if (!isfinite(rr)) {
        S.status = 3;
        S.active = 0;
    } else if (rr <= S.tol2) {
        S.status = 1;
        S.active = 0;
    } else if (S.iters >= max_iter) {
        S.status = 4;
        S.active = 0;
    }
}

// Block + grid reduction of NV doubles per RHS for LANES RHS per thread
// (v[L*NV + k] belongs to RHS LANES*unit + L).  Returns true in exactly one
// thread per unit (lane 0 of the last block), with the totals in v.  The
// block tree runs kRedChunk values at a time through shared memory; each
// value's summation order is the same fixed tree whatever NV is.
constexpr int kRedChunk = 4;

template <int W>
__device__ __forceinline__ void block_tree(double v[W], double *sh, const Cfg c, int t, int units,
                                           int lane)
{
#pragma unroll
    for (int k0 = 0; k0 < W; k0 += kRedChunk) {
#pragma unroll
        for (int k = 0; k < kRedChunk; k++)
            if (k0 + k < W) sh[t * kRedChunk + k] = v[k0 + k];
        __syncthreads();
        for (int w = c.lanes / 2; w > 0; w >>= 1) {
            if (lane < w)
#pragma unroll
                for (int k = 0; k < kRedChunk; k++)
                    if (k0 + k < W) sh[t * kRedChunk + k] += sh[(t + w * units) * kRedChunk + k];
            __syncthreads();
        }
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < kRedChunk; k++)
                if (k0 + k < W) v[k0 + k] = sh[t * kRedChunk + k];
        __syncthreads();
    }
}

template <int NV, int LANES>
__device__ bool reduce_last(double v[LANES * NV], const Cfg c, double *partials,
                            unsigned int *counter, int units)
{
    static_assert(NV <= kRedWidth, "per-RHS partials hold kRedWidth values");
    constexpr int W = LANES * NV;
    __shared__ double sh[kMaxBlock * kRedChunk];
    __shared__ bool last;
    const int t = threadIdx.x, u = t % units, lane = t / units;
    block_tree<W>(v, sh, c, t, units, lane);
    if (lane == 0)
#pragma unroll
        for (int L = 0; L < LANES; L++)
#pragma unroll
            for (int k = 0; k < NV; k++)
                partials[((long long)blockIdx.x * kMaxRhs + LANES * u + L) * kRedWidth + k] = v[L * NV + k];
    __threadfence();
    __syncthreads();
    if (t == 0) last = (atomicAdd(counter, 1u) == (unsigned)(gridDim.x - 1));
    __syncthreads();
    if (!last) return false;
    __threadfence();
    // last block: lane l sums blocks l, l+lanes, ... in order, then a fixed tree
    double acc[W];
#pragma unroll
    for (int k = 0; k < W; k++) acc[k] = 0;
    for (int b = lane; b < (int)gridDim.x; b += c.lanes)
#pragma unroll
        for (int L = 0; L < LANES; L++)
#pragma unroll
            for (int k = 0; k < NV; k++)
                acc[L * NV + k] += __ldcg(partials + ((long long)b * kMaxRhs + LANES * u + L) * kRedWidth + k);
    block_tree<W>(acc, sh, c, t, units, lane);
    if (t == 0) *counter = 0u;
    if (lane != 0) return false;
#pragma unroll
    for (int k = 0; k < W; k++) v[k] = acc[k];
    return true;
}

}  // namespace dp
