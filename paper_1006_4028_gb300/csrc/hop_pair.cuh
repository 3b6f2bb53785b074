// The spin projection, link multiplication and accumulation of one hop on
// the paired FP32 layout (two RHS per 64-bit register lane pair), shared by
// the dslash kernels and the Schwarz block solver.  Chiral gamma basis (see
// dp_internal.h); component index 3*spin + colour.
#pragma once

#include "cplx.cuh"
#include "pair.cuh"

namespace dp {

// upper two spins of (1 + SG*gamma_mu) psi for one colour, from its 4 spins
template <int MU, int SG>
__device__ __forceinline__ void project_pair(const C2 p0, const C2 p1, const C2 p2, const C2 p3,
                                             C2 &h0, C2 &h1)
{
    if (MU == 0) {
        h0 = SG < 0 ? c2_add(p0, p2) : c2_sub(p0, p2);
        h1 = SG < 0 ? c2_add(p1, p3) : c2_sub(p1, p3);
    } else if (MU == 1) {
        h0 = SG < 0 ? c2_addi(p0, p3) : c2_subi(p0, p3);
        h1 = SG < 0 ? c2_addi(p1, p2) : c2_subi(p1, p2);
    } else if (MU == 2) {
        h0 = SG < 0 ? c2_add(p0, p3) : c2_sub(p0, p3);
        h1 = SG < 0 ? c2_sub(p1, p2) : c2_add(p1, p2);
    } else {
        h0 = SG < 0 ? c2_addi(p0, p2) : c2_subi(p0, p2);
        h1 = SG < 0 ? c2_subi(p1, p3) : c2_addi(p1, p3);
    }
}

// acc += c t, acc += c (i t), acc += c (-i t); C = (c, c), MC = (-c, -c)
__device__ __forceinline__ void acc1(C2 &acc, f2 C, C2 t)
{
    acc.re = ffma2(C, t.re, acc.re);
    acc.im = ffma2(C, t.im, acc.im);
}
__device__ __forceinline__ void acc_i(C2 &acc, f2 C, f2 MC, C2 t)
{
    acc.re = ffma2(MC, t.im, acc.re);
    acc.im = ffma2(C, t.re, acc.im);
}
__device__ __forceinline__ void acc_mi(C2 &acc, f2 C, f2 MC, C2 t)
{
    acc.re = ffma2(C, t.im, acc.re);
    acc.im = ffma2(MC, t.re, acc.im);
}

// acc += c (1 + SG*gamma_mu) psi, colour a, given t0, t1 = (U h)_a of spins 0, 1
template <int MU, int SG>
__device__ __forceinline__ void accumulate_pair(C2 acc[12], int a, f2 C, f2 MC, C2 t0, C2 t1)
{
    acc1(acc[a], C, t0);
    acc1(acc[3 + a], C, t1);
    if (MU == 0) {
        acc1(acc[6 + a], SG < 0 ? C : MC, t0);
        acc1(acc[9 + a], SG < 0 ? C : MC, t1);
    } else if (MU == 1) {
        if (SG < 0) {
            acc_mi(acc[6 + a], C, MC, t1);
            acc_mi(acc[9 + a], C, MC, t0);
        } else {
            acc_i(acc[6 + a], C, MC, t1);
            acc_i(acc[9 + a], C, MC, t0);
        }
    } else if (MU == 2) {
        acc1(acc[6 + a], SG < 0 ? MC : C, t1);
        acc1(acc[9 + a], SG < 0 ? C : MC, t0);
    } else {
        if (SG < 0) {
            acc_mi(acc[6 + a], C, MC, t0);
            acc_i(acc[9 + a], C, MC, t1);
        } else {
            acc_i(acc[6 + a], C, MC, t0);
            acc_mi(acc[9 + a], C, MC, t1);
        }
    }
}

// acc += c (1 + SG*gamma_mu) U psi (forward) or c (1 + SG*gamma_mu) U^dag psi
// (backward) from the projected half spinor h (spins 0, 1 of colours 0-2)
template <int MU, int SG>
__device__ __forceinline__ void hop_apply(C2 (&acc)[12], const C2 (&h)[6], const Cx<float> (&u)[9],
                                          f2 C, f2 MC)
{
#pragma unroll
    for (int a = 0; a < 3; a++) {
        C2 t0, t1;
        // forward: (U h)_a = sum_b U_ab h_b; backward: (U^dag h)_a = sum_b conj(U_ba) h_b
        const Cx<float> e0 = SG < 0 ? u[3 * a] : u[a];
        const Cx<float> e1 = SG < 0 ? u[3 * a + 1] : u[3 + a];
        const Cx<float> e2 = SG < 0 ? u[3 * a + 2] : u[6 + a];
        const B2 b0 = bcast(e0.re, e0.im), b1 = bcast(e1.re, e1.im), b2 = bcast(e2.re, e2.im);
        if (SG < 0) {
            t0 = c2_mul(b0, h[0]);
            t1 = c2_mul(b0, h[3]);
            t0 = c2_fma(b1, h[1], t0);
            t1 = c2_fma(b1, h[4], t1);
            t0 = c2_fma(b2, h[2], t0);
            t1 = c2_fma(b2, h[5], t1);
        } else {
            t0 = c2_cjmul(b0, h[0]);
            t1 = c2_cjmul(b0, h[3]);
            t0 = c2_cjfma(b1, h[1], t0);
            t1 = c2_cjfma(b1, h[4], t1);
            t0 = c2_cjfma(b2, h[2], t0);
            t1 = c2_cjfma(b2, h[5], t1);
        }
        accumulate_pair<MU, SG>(acc, a, C, MC, t0, t1);
    }
}

}  // namespace dp
