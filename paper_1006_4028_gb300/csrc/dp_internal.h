// Internal definitions shared by the library's translation units.
//
// Device data layout (even-odd, site-blocked SoA; V/2 = Vh sites per parity):
//   half-site index s of a site of parity p = (t+x+y+z)&1 is i>>1 with
//   i = ((t*Lz + z)*Ly + y)*Lx + x (Lx even, so each x-row holds Lx/2 sites of
//   each parity).
//   spinor field of one parity, n RHS: [chunk][s][rhs] with chunk = float4
//     (6 per spinor, FP32) or double2 (12 per spinor, FP64); the 24 reals of a
//     spinor are (spin, colour, re/im) in that order, spin-major.
//   links of one parity: [mu][chunk][s]; FP64: 9 double2 (18 reals);
//     FP32: 18 reals as 4 float4 per link ([mu][4][s], entries 0-7) followed by
//     a float2 [mu][s] (entry 8), or 12 reals as 3 float4 (rows 0 and 1).
//   clover (and its inverse) of one parity: [slot][chunk][s]; 72 reals per
//     site = two Hermitian 6x6 chiral blocks (spins 0,1 and spins 2,3), each
//     packed as 6 real diagonal entries then the 15 upper-triangle entries
//     (i<j, row-major) as (re, im); FP64: 36 double2, FP32: 18 float4.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dp {

constexpr int kMaxRhs = 64;
constexpr int kMaxL = 256;

struct Geom {
    int T, Lx, Ly, Lz, Lxh, Lmax;
    long long V, Vh;
};

// dslash epilogues: D = hopping term D_{p,1-p}, A = clover(+mass) of parity p
enum Epi {
    EPI_HOP = 0,      // out = D in
    EPI_AINV = 1,     // out = A^-1 D in
    EPI_XMY_AINV = 2, // out = x - A^-1 D in
    EPI_AINV_XMY = 3, // out = A^-1 (x - D in)
    EPI_XPY = 4,      // out = x + D in
    EPI_XMY_G5 = 5    // out = x - gamma5 D in (last step of the adjoint Schur operator)
};

// link storage formats; the 16-bit ones hold rows 0 and 1 as FP16 or BF16
// values divided by one FP32 scale per link (max |element| of the two rows):
// [mu][3][s] uint2 (four 16-bit values each), then [mu][s] float scales
enum LinkFmt {
    LINK_F64_18 = 0,
    LINK_F32_18 = 1,
    LINK_F32_12 = 2,
    LINK_H16_12 = 3,
    LINK_B16_12 = 4,
    LINK_DF_18 = 5  // double-float (two FP32 per real), 18 reals: float4 [4][9][Vh]
};

// quantise FP64 links of one parity ([mu][9 double2][Vh]) into a 16-bit format
cudaError_t launch_pack_links16(const double2 *l64, long long Vh, int fmt, void *out,
                                cudaStream_t st);
inline size_t links16_bytes(long long Vh) { return (size_t)Vh * 4 * (3 * 8 + 4); }

constexpr int kMaxGroups = 8;  // point-source groups (12 RHS each) per batch

// per-RHS slot of a batch: which group (mass/profile/source) it belongs to and
// which spin-colour component of the point source it carries
struct SlotInfo {
    int group;      // index into the per-group arrays
    int comp;       // source component k = 3*spin + colour
    int t, x, y, z; // source site
    double scale;   // alpha_B(x_src): the source scaling eta' = alpha_B eta
};

struct DslashParams {
    const void *in;         // spinor, parity 1-p
    void *out;              // spinor, parity p
    const void *x;          // spinor, parity p (epilogues 2-4)
    const void *links[2];   // by parity
    const void *clov[kMaxGroups]; // parity p clover inverse per group
    const void *hop;        // [group][mu][2][Lmax] hop factors incl. the -1/2
    const int *active;      // NULL or per-RHS flags at active[r * active_stride]
    int active_stride;
    Geom g;
    int parity;             // output parity
    int nrhs;
    int8_t grp_of[kMaxRhs]; // RHS -> group
    // NULL, or (FP32, x - A^-1 D epilogue) per-site partial sums of the
    // BiCGStab omega: f2 (one lane per RHS of a pair) [3][Vh][nrhs/2] holding
    // Re <out, x>, Im <out, x> and |out|^2 over the 12 components of a site
    void *dots;
};

// ---- launch wrappers (dslash.cu) ----
// prec: 0 = FP64 (links LINK_F64_18), 1 = FP32 (links LINK_F32_18 / _F32_12
// / _H16_12 / _B16_12).  rpt: RHS per thread (FP64 1; FP32 2 = one RHS pair,
// 4 = two pairs, only for the A^-1 and x - A^-1 D epilogues).  stages > 0
// (FP32 one pair per thread, 12-real or 16-bit links, the A^-1 and
// x - A^-1 D epilogues, 64, 96 or 128 threads per block) selects the kernel
// that stages neighbour spinors and links through shared memory: 2-3 =
// that many directions in flight; 4 = 2 in flight, one persistent wave of
// blocks whose threads walk several sites; 5 = direct loads with an L1
// prefetch 2 directions ahead (any block size); 6 = the spinor alone staged
// (2 in flight), the link prefetched into L1, 16 warps per SM; 0 = direct
// loads
cudaError_t launch_dslash(const DslashParams &p, int prec, int link_fmt, int epi, int block,
                          int rpt, cudaStream_t st, int stages = 0);
bool dslash_rpt_ok(int nrhs, int rpt, int prec, int epi);
bool dslash_staged_ok(int prec, int link_fmt, int epi, int rpt, int stages, int block);
// double-float Schur launches of the outer loop (dslash_df.cu): EPI_AINV
// writes double-float, EPI_XMY_AINV reads x as double-float and writes FP64;
// links LINK_DF_18, clover inverse float4 [36][Vh], hops float2 [grp][8][Lmax]
cudaError_t launch_dslash_df(const DslashParams &p, int epi, int block, cudaStream_t st);
// FP64 <-> double-float, element-wise over `count` complex numbers; with a
// mask only the elements of RHS r with mask[r * mask_stride] != 0 (element
// i belongs to RHS i % n)
cudaError_t launch_to_df(const double2 *in, float4 *out, long long count, const int *mask, int n,
                         int mask_stride, cudaStream_t st);
cudaError_t launch_from_df(const float4 *in, double2 *out, long long count, const int *mask, int n,
                           int mask_stride, cudaStream_t st);

// launch shape of the Schur dslash launches (tuner result or default)
struct Shape {
    int block = 64;
    int rpt = 1;
    int stages = 0;
};

// ---- clover (clover.cu) ----
// clover term (no mass) for all sites of both parities, FP64, layout above
cudaError_t launch_clover_build(const double2 *links64_e, const double2 *links64_o,
                                const Geom &g, double csw, double2 *clov_e, double2 *clov_o,
                                cudaStream_t st);
// inverse of (4+M) + clover for one parity; writes FP64 and FP32 copies;
// flag[0] set to 1 if a block is singular or non-finite
cudaError_t launch_clover_invert(const double2 *clov, long long Vh, double M, double2 *inv64,
                                 float4 *inv32, int *flag, cudaStream_t st);
cudaError_t launch_clover_to_f32(const double2 *in, float4 *out, long long Vh, cudaStream_t st);
// out = (diag_g + C_g) in per RHS group g, one parity: C_g a packed clover
// matrix (clover term, or an inverse with diag_g = 0), FP64 or FP32 spinors
struct CloverApplyParams {
    const void *mat[kMaxGroups];
    double diag[kMaxGroups];
    int8_t grp_of[kMaxRhs];
    const int *mask;  // NULL or per-RHS flags: RHS with mask[r * stride] == 0 are skipped
    int mask_stride;  // 0 or 1: consecutive ints; else the stride in ints (RhsState rows)
    int g5;           // 1: out = gamma5 (mat + diag) in (sign flip of chiral block 1)
    const void *in;
    void *out;        // may alias `in`
    long long Vh;
    int nrhs;
};
cudaError_t launch_clover_apply(const CloverApplyParams &p, int prec, cudaStream_t st);
// FP64 apply at each masked RHS's source site only (point sources: zero
// elsewhere; the caller zeroes `out` of those RHS first); parity: that of p.in
cudaError_t launch_clover_point(const CloverApplyParams &p, const Geom &g, const SlotInfo *slots,
                                int parity, cudaStream_t st);
// per-RHS |(mat + diag) in|^2 into out_dev[nrhs]: FP64 spinor, FP32 clover
// (p.mat), FP32 products, FP64 sums
struct BlasCtx;
cudaError_t launch_clover_norm(BlasCtx &bc, const CloverApplyParams &p, double *out_dev,
                               cudaStream_t st);

// ---- field packing, sources, restore/contract (field.cu) ----
cudaError_t launch_pack_links(const double2 *lex, const Geom &g, double2 *l64[2], float2 *l32f[2],
                              float4 *l32c[2], cudaStream_t st);
// lexicographic complex128 spinors [nrhs][V][12] <-> packed parity halves
cudaError_t launch_pack_spinor(const double2 *lex, const Geom &g, int nrhs, int prec,
                               void *even, void *odd, cudaStream_t st);
cudaError_t launch_unpack_spinor(const void *even, const void *odd, const Geom &g, int nrhs,
                                 int prec, double2 *lex, cudaStream_t st);
// point source for every slot: RHS k = slots[k].scale at its source site for
// component slots[k].comp, FP64, both parities (zeroed by the caller)
cudaError_t launch_point_source(const Geom &g, const SlotInfo *slots_dev, int nrhs,
                                const int *mask, double2 *even, double2 *odd, cudaStream_t st);
// restore S = S'/alpha_B per site and contract C_PP per group:
// cpp[group][(t - t_src[group]) mod T] (+)= -sum_{slice t} |S|^2.
// alpha: [group][mu][Lmax] FP64 alpha_B per coordinate; partials: T*P*ngroups
// doubles with P = contract_blocks_per_slice(g); prop_lex: NULL or
// [nrhs][V][12] complex128 of the restored propagator
int contract_blocks_per_slice(const Geom &g);
// only RHS with mask[r] != 0 contribute (mask NULL: all)
// cap_dev (optional): C_AP(y0) = sum tr[gamma_0 S S^dag] per group, same
// layout as cpp_dev; partials then needs 2 * T * P * n_mass doubles
cudaError_t launch_restore_contract(const double2 *xe, const double2 *xo, const Geom &g, int nrhs,
                                    const double *alpha, const SlotInfo *slots_dev, int ngroups,
                                    const int *t_src_dev, const int *mask, double *cpp_dev,
                                    double *partials, double2 *prop_lex, cudaStream_t st,
                                    double *cap_dev = nullptr);
// heavy-light C(y0) = -sum_{y vec} tr[S_h S_l^dag] of two groups' propagators
// (slots slot_h.. and slot_l.., 12 each, groups gh, gl for their profiles);
// out_dev [T][2] (re, im), y0 relative to t_src; partials: 2 * T * P doubles
cudaError_t launch_contract_hl(const double2 *xe, const double2 *xo, const Geom &g, int nrhs,
                               const double *alpha, int gh, int gl, int slot_h, int slot_l, int t_src,
                               double *partials, double *out_dev, cudaStream_t st);
// dst[k] (+)= src[k], k < T (accumulate != 0: add)
cudaError_t launch_cpp_commit(const double *src, double *dst, int T, int accumulate, cudaStream_t st);

// ---- BLAS-1 and reductions (blas.cu) ----
struct RhsState {        // per RHS, device resident
    double2 rho, alpha, omega, beta;
    double rr, bb, tol2;  // |r|^2, |b|^2, stop threshold on |r|^2
    double scale;         // FP64 outer loop: |r| used to normalise the inner source
    int active;           // 1 while iterating
    int iters;
    int status;           // 0 running, 1 converged, 2 breakdown, 3 non-finite, 4 max-iter
    int fresh;            // 1: x = 0, next residual call sets |b|^2 and tol2
    int brk;              // FP32 BiCGStab: breakdown found by the omega reduction
    int refine;           // FP64 outer loop: per-slice refinement (the inner solve runs in
                          // another profile's metric; the global test does not stop it)
    double2 rs, rt;       // FP32 BiCGStab: <rhat, s> and <rhat', s> = <rhat, Mhat s>
};

constexpr int kRedWidth = 8;  // values per RHS in a block's reduction partials

struct BlasCtx {
    double *partials;     // [max_blocks][kMaxRhs][kRedWidth]
    unsigned int *counter;
    int *n_active;        // device counter of active RHS
    int blocks;
};

// all vectors one parity, n RHS, layout above; prec 0 = FP64, 1 = FP32
cudaError_t blas_bicg_init(BlasCtx &bc, int prec, const void *b, void *r, void *rhat, void *p,
                           void *v, void *x, long long Vh, int nrhs, RhsState *st, double tol,
                           cudaStream_t s);
// p, s, omega and update: FP64 only (the FP32 solver uses blas32_s_dots,
// blas32_omega_dots and blas32_update_pa, which carry the p update); alpha:
// both precisions
cudaError_t blas_bicg_p(BlasCtx &bc, int prec, const void *r, void *p, const void *v,
                        long long Vh, int nrhs, const RhsState *st, int first, cudaStream_t s);
cudaError_t blas_bicg_alpha(BlasCtx &bc, int prec, const void *rhat, const void *v,
                            long long Vh, int nrhs, RhsState *st, cudaStream_t s);
cudaError_t blas_bicg_s(BlasCtx &bc, int prec, const void *r, const void *v, void *sv,
                        long long Vh, int nrhs, const RhsState *st, cudaStream_t s);
cudaError_t blas_bicg_omega(BlasCtx &bc, int prec, const void *t, const void *sv,
                            long long Vh, int nrhs, RhsState *st, cudaStream_t s);
cudaError_t blas_bicg_update(BlasCtx &bc, int prec, void *x, void *r, const void *p,
                             const void *sv, const void *t, const void *rhat, long long Vh,
                             int nrhs, RhsState *st, int max_iter, cudaStream_t s);
// FP32 inner solver on the paired layout (blas32.cu); nrhs even
cudaError_t blas32_init(BlasCtx &bc, const void *b, void *r, void *rh, long long Vh, int nrhs,
                        RhsState *st, cudaStream_t s, void *p = nullptr);
cudaError_t blas32_alpha(BlasCtx &bc, const void *rh, const void *v, long long Vh, int nrhs,
                         RhsState *st, cudaStream_t s);
// BiCGStab with the shadow image rhat' = Mhat^dag rhat (formed once per
// inner solve), so that <rhat, v> = <rhat', p> and <rhat, t> = <rhat', s>
// ride in passes that already read p and s, and <t, s>, |t|^2 in the
// x - A^-1 D launch that forms t (DslashParams::dots).  Init: blas32_init,
// rhat' = Mhat^dag rhat, alpha = rho / <rhat', p> (blas32_alpha).  Per
// iteration: v = Mhat p; s_dots (s = r - alpha v, <rhat, s>, <rhat', s>);
// t = Mhat s with the dots; omega_dots (omega, rho' = <rhat, s> -
// omega <rhat', s>, beta); update_pa (x += alpha p + omega s, r = s - omega t,
// p = r + beta (p - omega v), |r|^2 decides convergence, next alpha =
// rho' / <rhat', p>): 14 vector streams and 7 launches per iteration
cudaError_t blas32_s_dots(BlasCtx &bc, const void *r, const void *v, void *sv, const void *rh,
                          const void *rh2, long long Vh, int nrhs, RhsState *st, cudaStream_t s);
cudaError_t blas32_omega_dots(BlasCtx &bc, const void *dots, long long Vh, int nrhs, RhsState *st,
                              cudaStream_t s);
cudaError_t blas32_update_pa(BlasCtx &bc, void *x, void *r, void *p, const void *sv, const void *t,
                             const void *v, const void *rh2, long long Vh, int nrhs, RhsState *st,
                             int max_iter, cudaStream_t s);
// CGNE (CG on the normal equations Mhat^dag Mhat x = Mhat^dag b), per RHS,
// real scalars in the .x parts of rho / alpha / beta.  Init: blas_bicg_init
// (r = b, x = p = 0, |b|^2).  Per iteration, with z = Mhat^dag r and
// w = Mhat p:  gamma: rho' = |z|^2, beta = rho'/rho (0 when first);
// p = z + beta p;  alpha = rho / |w|^2;  x += alpha p, r -= alpha w, |r|^2
// decides convergence
cudaError_t blas_cg_gamma(BlasCtx &bc, int prec, const void *z, long long Vh, int nrhs,
                          RhsState *st, int first, cudaStream_t s);
cudaError_t blas_cg_p(BlasCtx &bc, int prec, const void *z, void *p, long long Vh, int nrhs,
                      const RhsState *st, cudaStream_t s);
cudaError_t blas_cg_alpha(BlasCtx &bc, int prec, const void *w, long long Vh, int nrhs,
                          RhsState *st, cudaStream_t s);
cudaError_t blas_cg_update(BlasCtx &bc, int prec, void *x, void *r, const void *p, const void *w,
                           long long Vh, int nrhs, RhsState *st, int max_iter, cudaStream_t s);
cudaError_t blas32_cg_gamma(BlasCtx &bc, const void *z, long long Vh, int nrhs, RhsState *st,
                            int first, cudaStream_t s);
cudaError_t blas32_cg_p(BlasCtx &bc, const void *z, void *p, long long Vh, int nrhs,
                        const RhsState *st, cudaStream_t s);
cudaError_t blas32_cg_alpha(BlasCtx &bc, const void *w, long long Vh, int nrhs, RhsState *st,
                            cudaStream_t s);
cudaError_t blas32_cg_update(BlasCtx &bc, void *x, void *r, const void *p, const void *w,
                             long long Vh, int nrhs, RhsState *st, int max_iter, cudaStream_t s);
// GCR on the paired FP32 layout (blas32.cu): per-RHS <a, b> and |a|^2 into
// device arrays; w -= c wi and z -= c zi; w, z /= |w|; x += a z, r -= a w
// with |r|^2 deciding convergence (finish_cg_update); out = a - b
cudaError_t blas32_dotv(BlasCtx &bc, const void *a, const void *b, long long Vh, int nrhs,
                        const RhsState *st, double2 *out, cudaStream_t s);
cudaError_t blas32_norm2v(BlasCtx &bc, const void *a, long long Vh, int nrhs, const RhsState *st,
                          double *out, cudaStream_t s);
cudaError_t blas32_mgs(BlasCtx &bc, void *w, void *z, const void *wi, const void *zi, long long Vh,
                       int nrhs, const RhsState *st, const double2 *cf, cudaStream_t s);
cudaError_t blas32_normalise(BlasCtx &bc, void *w, void *z, long long Vh, int nrhs,
                             const RhsState *st, const double *nrm, cudaStream_t s);
cudaError_t blas32_gcr_update(BlasCtx &bc, void *x, void *r, const void *z, const void *w,
                              long long Vh, int nrhs, RhsState *st, const double2 *cf, int max_iter,
                              cudaStream_t s);
cudaError_t blas32_xmy(const void *a, const void *b, void *out, long long Vh, int nrhs, cudaStream_t s);

// Schwarz block solves of SAP+GCR (sap.cu)
struct SapParams {
    const void *res;                  // global residual, parity `parity`, paired FP32
    void *z;                          // global correction, += the block solutions
    const void *links[2];             // per parity, FP32 or 16-bit format
    const void *clov[2][kMaxGroups];  // FP32 clover inverses per parity and group
    const void *hop;                  // FP32 hop tables [group][8][Lmax]
    int8_t grp_of[kMaxRhs];
    const int *active;                // RhsState rows (stride active_stride) or NULL
    int active_stride;
    Geom g;
    int parity;                       // the Schur parity p
    int nrhs;
    int bs[4], nb[4];                 // block extents and blocks per direction (t, x, y, z)
    int colour;                       // blocks with (bt + bx + by + bz) % 2 == colour
    int n_mr;                         // minimal-residual steps per block
};
// block extents: 4 where the extent allows, else 2; false if an extent is odd
bool sap_blocks(const Geom &g, int bs[4], int nb[4]);
cudaError_t launch_sap_block(const SapParams &p, int link_fmt, cudaStream_t st);

// ---- per-time-slice accuracy of the outer loop (slices.cu) ----
// Per group m and absolute time slice t, over the RHS with mask[r] != 0 on
// the Schur parity `parity`: out[(m*T + t)*2 + 0] = sum |x/alpha_B|^2,
// out[... + 1] = sum |r/alpha_B|^2 (alpha_B of the group, per site: the
// restored metric); summed in a fixed order.  partials: 2 * T * P * ngroups
// doubles, P = contract_blocks_per_slice(g).
cudaError_t launch_slice_norms(const double2 *x, const double2 *r, const Geom &g, int parity,
                               int nrhs, const double *alpha, const SlotInfo *slots_dev,
                               int ngroups, const int *mask, double *partials, double *out,
                               cudaStream_t st);
// Transfer of the outer residual into the inner solver's metric for RHS with
// st.active && st.refine: R(site) = alpha_in/alpha_out of the RHS's group
// (alpha tables [group][mu][Lmax]).  ratio_norm: st.scale = |R r| (FP64,
// deterministic); to_f32 / scale64: inner source R r / scale (paired FP32 or
// FP64 layout, only the refined RHS are written); acc: x += scale e / R.
cudaError_t blas_ratio_norm(BlasCtx &bc, const double2 *r64, const Geom &g, int parity, int nrhs,
                            const double *alpha_out, const double *alpha_in,
                            const SlotInfo *slots_dev, RhsState *st, cudaStream_t s);
cudaError_t blas_to_f32_ratio(const double2 *r64, float4 *r32, const Geom &g, int parity,
                              int nrhs, const double *alpha_out, const double *alpha_in,
                              const SlotInfo *slots_dev, const RhsState *st, cudaStream_t s);
cudaError_t blas_scale64_ratio(const double2 *r64, double2 *out, const Geom &g, int parity,
                               int nrhs, const double *alpha_out, const double *alpha_in,
                               const SlotInfo *slots_dev, const RhsState *st, cudaStream_t s);
cudaError_t blas_acc_f32_ratio(double2 *x64, const float4 *e32, const Geom &g, int parity,
                               int nrhs, const double *alpha_out, const double *alpha_in,
                               const SlotInfo *slots_dev, const RhsState *st, cudaStream_t s);
cudaError_t blas_acc64_ratio(double2 *x64, const double2 *e64, const Geom &g, int parity,
                             int nrhs, const double *alpha_out, const double *alpha_in,
                             const SlotInfo *slots_dev, const RhsState *st, cudaStream_t s);

// FP64 outer loop helpers
// r = b - y (r = b for `fresh` RHS); |r|^2 -> st.rr; st.scale = |r|;
// convergence vs st.tol2 -> active
// (mask: NULL or per-RHS flags restricting the update further)
cudaError_t blas_residual64(BlasCtx &bc, const double2 *b, const double2 *y, double2 *r,
                            long long Vh, int nrhs, RhsState *st, const int *mask,
                            cudaStream_t s);
// out = a - b (FP64) for the RHS with mask[r] != 0
cudaError_t blas_sub64_masked(const double2 *a, const double2 *b, double2 *out, long long Vh,
                              int nrhs, const int *mask, cudaStream_t s);
// zero the FP64 vector entries of the RHS with mask[r] != 0
cudaError_t blas_zero_masked(double2 *v, long long Vh, int nrhs, const int *mask, cudaStream_t s);
// r32 = r64 / scale (active RHS); zero for inactive
cudaError_t blas_to_f32_scaled(const double2 *r64, float4 *r32, long long Vh, int nrhs,
                               const RhsState *st, cudaStream_t s);
// x64 += scale * e32 (active RHS)
cudaError_t blas_acc_f32(double2 *x64, const float4 *e32, long long Vh, int nrhs,
                         const RhsState *st, cudaStream_t s);
cudaError_t blas_zero(void *v, size_t bytes, cudaStream_t s);
// per-RHS squared norms (FP64 accumulate) into out_dev[nrhs]
cudaError_t blas_norm2(BlasCtx &bc, int prec, const void *v, long long Vh, int nrhs,
                       double *out_dev, cudaStream_t s);
// inner-solve state from the outer one: same active set; per-RHS inner
// tolerance max(inner_tol, 0.5 target |b|/|r|) (squared into tol2)
cudaError_t blas_inner_setup(const RhsState *outer, RhsState *inner, int nrhs,
                             double inner_tol, double target, cudaStream_t s);
// FP64 normalised copy out = v / scale (active RHS, zero otherwise)
cudaError_t blas_scale64(const double2 *v, double2 *out, long long Vh, int nrhs,
                         const RhsState *st, cudaStream_t s);
// x64 += scale * e64 (active RHS)
cudaError_t blas_acc64(double2 *x64, const double2 *e64, long long Vh, int nrhs,
                       const RhsState *st, cudaStream_t s);
// per-RHS |a - b|^2 (FP64) into out_dev[nrhs]
cudaError_t blas_diff_norm2(BlasCtx &bc, const double2 *a, const double2 *b, long long Vh,
                            int nrhs, double *out_dev, cudaStream_t s);
// count active RHS into bc.n_active
cudaError_t blas_count_active(BlasCtx &bc, const RhsState *st, int nrhs, cudaStream_t s);

}  // namespace dp
