/*
 * dpre -- distance-preconditioned O(a)-improved Wilson-clover solves on one
 * NVIDIA GB300 GPU (sm_103a).  C ABI of libdpre.so.
 *
 * The method (de Divitiis, Petronzio, Tantalo, arXiv 1006.4028):
 *   Sec. I, eq. (linsysunprec): solve sum_y (D[U]+M)_{x,y} S(y) = eta(x) for a
 *     source on one time slice, to a global residue r (eq. stopping).
 *   Sec. II, eq. (redeft): factor a profile out of the propagator.  This
 *     library takes the profile in the reciprocal orientation alpha_B = 1/alpha:
 *     S'(y) = alpha_B(y) S(y), eta'(y) = alpha_B(y) eta(y), and solves
 *     (D'+M) S' = eta' (eq. linsysprec) with D'+M = A (D+M) A^-1, A = diag(alpha_B).
 *     Only the hopping terms change: the coefficient of U_mu(x) S'(x+mu) becomes
 *     alpha_B(x_mu)/alpha_B(x_mu+1) and that of U_mu(x-mu)^dag S'(x-mu) becomes
 *     alpha_B(x_mu)/alpha_B(x_mu-1) (Sec. II modified derivatives; Sec. III,
 *     eq. redefcovs, for all four directions), with the antiperiodic time sign on
 *     the hops across t = T-1 <-> 0 (eq. redeftbc).
 *   Sec. II, eq. (backcorrection) and Sec. III: restore S = S'/alpha_B per site
 *     before contracting C_PP(y0) = -sum_{y vec} tr[S^dag(y) S(y)].
 *
 * Operator convention (the paper names the O(a)-improved Wilson operator of
 * Sec. II without writing it out; this is the standard form with r = 1):
 *   (D+M) psi(x) = (4+M) psi(x)
 *      - 1/2 sum_mu [ (1-gamma_mu) U_mu(x) psi(x+mu) + (1+gamma_mu) U_mu(x-mu)^dag psi(x-mu) ]
 *      + c_sw (i/4) sum_{mu,nu} sigma_{mu nu} Fhat_{mu nu}(x) psi(x),
 *   sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu], Fhat = (Q - Q^dag)/8 (4-leaf clover).
 *   Chiral gamma basis: gamma_mu = [[0, e_mu], [e_mu^dag, 0]], e_0 = -1,
 *   e_k = -i sigma_k, gamma_5 = gamma_0 gamma_1 gamma_2 gamma_3 = diag(1,1,-1,-1).
 *
 * Host data layouts (all complex128 = two doubles, re then im):
 *   dims = {T, Lx, Ly, Lz}; site index i = ((t*Lz + z)*Ly + y)*Lx + x;
 *   direction mu = 0 (t), 1 (x), 2 (y), 3 (z).
 *   links:   [V][4][3][3]       U_mu(x), row a, column b.
 *   spinor:  [nrhs][V][4][3]    spin, colour.
 *   prop:    [n_mass][12][V][4][3]  restored S for the 12 source components
 *            k = 3*spin + colour (solution for source component k).
 *   cpp:     [n_mass][T]        C_PP(y0), y0 = (t - t_src) mod T.
 *
 * Ownership: the caller owns every pointer it passes; the library copies what
 * it needs during the call and keeps no caller pointer.  Handles (dp_ctx,
 * dp_field, dp_ticket) belong to the library until released.
 *
 * Errors: every entry point returns a dp_status; nothing aborts or throws
 * across the ABI.  dp_last_error() gives a thread-local message for the last
 * failing call on the calling thread.  NaN/Inf inputs give DP_ERR_INVALID_ARG.
 * Every extent must be even (the even-odd split needs neighbours across the
 * periodic seams to have opposite parity), >= 2 and <= 256.
 *
 * Threading: a dp_ctx is used by one thread at a time, except dp_submit,
 * dp_wait and dp_serve_stats, which may be called from any thread.
 */
#ifndef DPRE_H
#define DPRE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dp_ctx dp_ctx;
typedef uint64_t dp_field;
typedef uint64_t dp_ticket;

typedef enum {
    DP_OK = 0,
    DP_ERR_INVALID_ARG = 1,
    DP_ERR_OOM = 2,
    DP_ERR_NOT_CONVERGED = 3,
    DP_ERR_BREAKDOWN = 4,
    DP_ERR_NONFINITE = 5,
    DP_ERR_TIMEOUT = 6,
    DP_ERR_REJECTED = 7,
    DP_ERR_CUDA = 8,
    DP_ERR_NOT_FOUND = 9
} dp_status;

/* Profile kinds, all in the alpha_B orientation, coordinates relative to the
 * source, rel_mu = (x_mu - src_mu) mod L_mu:
 *   NONE     alpha_B = 1 (unpreconditioned)
 *   EXP_T    alpha_B = exp(+alpha0 rel_t)                   (Sec. II, SF profile)
 *   COSH_T   alpha_B = 1/cosh[alpha0 (rel_t - T/2)]          (Sec. II, eq. pbcalpha)
 *   COSH_4D  alpha_B = prod_mu cosh[alpha0 (rel_mu - L_mu/2)] (Sec. III, eq. betaa)
 *   TABLE    alpha_B = prod_mu table[mu][x_mu] (absolute coordinates, > 0)   */
typedef enum {
    DP_PROF_NONE = 0,
    DP_PROF_EXP_T = 1,
    DP_PROF_COSH_T = 2,
    DP_PROF_COSH_4D = 3,
    DP_PROF_TABLE = 4
} dp_prof_kind;

typedef struct {
    int kind;               /* dp_prof_kind */
    double alpha0;
    const double *table[4]; /* TABLE only: alpha_B,mu per coordinate, length L_mu */
} dp_profile;

typedef enum {
    DP_PREC_FP64 = 0,       /* FP64 Krylov solve ("FP64 plain" when unbatched)   */
    DP_PREC_MIXED_FP32 = 1, /* FP32 inner BiCGStab, FP32 links, FP64 outer loop  */
    DP_PREC_MIXED_FP16 = 2, /* FP32 inner with FP16 links (per-link scale)       */
    DP_PREC_MIXED_BF16 = 3  /* FP32 inner with BF16 links (per-link scale)       */
} dp_prec;

/* BiCGStab on Mhat x = b (Sec. I, eqs. linsysunprec/linsysprec solved
 * iteratively), CG on the normal equations Mhat^dag Mhat x = Mhat^dag b
 * (CGNE), or GCR preconditioned by the Schwarz alternating procedure
 * (SAP+GCR, the solver of the paper's Table I, Sec. III; mixed precisions
 * only), all stopping on |b - Mhat x| / |b|. */
typedef enum { DP_SOLVER_BICGSTAB = 0, DP_SOLVER_CGNE = 1, DP_SOLVER_SAP_GCR = 2 } dp_solver;

typedef struct {
    int max_iter;     /* total inner iterations allowed (0: 20000)                  */
    int solver;       /* dp_solver                                                 */
    int prec;         /* dp_prec                                                   */
    int compress12;   /* FP32 links stored as 12 reals (row 2 rebuilt); 16-bit
                         links always are                                           */
    double inner_tol; /* relative reduction per inner solve (0: 1e-6 mixed)         */
    int batched;      /* 1: all RHS in one multi-RHS solve; 0: one RHS at a time    */
    int use_graph;    /* capture one solver iteration as a CUDA graph               */
    int check_every;  /* iterations between convergence reads (0: automatic)        */
    int sap_ncy;      /* SAP+GCR: Schwarz cycles per preconditioning (0: 4)          */
    int sap_nmr;      /* SAP+GCR: minimal-residual steps per block solve (0: 4)      */
    int gcr_nkv;      /* SAP+GCR: Krylov vectors before a GCR restart (0: 8)         */
    int outer_df;     /* mixed precisions: 1 = the outer loop's Schur operator in
                         double-float arithmetic (two FP32 per real, ~48-bit
                         significands, ~1e-14 relative; for r >= 1e-12) on the
                         FP32 units instead of FP64; 0 = FP64                       */
    double slice_tol; /* per-time-slice accuracy target: 0 = max(10 r, 1e-8) (default),
                         > 0 as given, < 0 off (the paper's global test alone).
                         See below. */
} dp_solve_opts;

/* Per-time-slice accuracy.  The residue r of the paper's stopping rule (Sec.
 * I, eq. stopping) bounds the residual summed over the lattice, which leaves
 * the far time slices, where the propagator is exponentially small, wrong
 * unless the profile makes the preconditioned solution roughly flat (Sec. II;
 * the light-quark profile of Sec. III steepens it instead).  So after the
 * global test passes, the FP64 outer loop measures per time slice t
 *   rho_t = |r_t / alpha_B| / |x_t / alpha_B|
 * (r the FP64 true residual of the even-odd Schur system, x the solution, both
 * on the Schur parity, restored by the profile per site, summed over the 12
 * components of the point source).  While max_t rho_t > slice_tol it runs more
 * defect-correction rounds whose inner solve uses a time profile built from
 * the measured slice norms (an exact change of the correction equation's
 * preconditioning, Sec. II).  If that stops improving, the solve returns
 * DP_ERR_NOT_CONVERGED (results still written) instead of DP_OK.
 * dp_solve_info.slice_residue reports the final max_t rho_t.  The default
 * target holds every slice to 10 r, but never below 1e-8: a per-slice residual
 * of 1e-8 keeps C_PP(y0) well inside 1e-6 on the workloads tested (the
 * 48x24^3 heavy quark at r = 1e-11 ends at 6e-10 from the oracle's C_PP with
 * no refinement), and refining further buys the correlator nothing. */

typedef struct {
    int iters_inner;         /* inner Krylov iterations (max over RHS)          */
    int iters_outer;         /* FP64 true-residual corrections                  */
    double true_rel_residue; /* max over RHS of |eta'-(D'+M)S'|/|eta'|, FP64, full lattice */
    double seconds;          /* wall time of the call                           */
    int n_rhs;               /* right-hand sides solved                         */
    int status;              /* dp_status of this solve                         */
    double slice_residue;    /* max over time slices of rho_t (see above); 0 when
                                the per-slice check is off                       */
    int refine_rounds;       /* outer rounds spent on per-slice refinement       */
} dp_solve_info;

/* Optional device allocator.  alloc returns device memory of >= bytes, 256-byte
 * aligned, usable on `stream`; free releases it.  NULL hooks: stream-ordered
 * allocation from a memory pool the context owns, which keeps memory freed
 * inside the context reserved for reuse (a solve's work vectors are
 * allocated and freed per call: re-mapping gigabytes each time would leave
 * the GPU idle) until dp_trim or dp_destroy. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*free)(void *ptr, size_t bytes, void *stream, void *user);
    void *user;
} dp_alloc_hooks;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  `stream` is a cudaStream_t to run
 * on (NULL: the library creates its own non-blocking stream). */
dp_status dp_create(dp_ctx **out, int device, const dp_alloc_hooks *hooks, void *stream);
void dp_destroy(dp_ctx *ctx);
const char *dp_last_error(void);
/* Device memory the library holds for this context, in bytes (memory the
 * context's pool keeps reserved after a free is not counted). */
size_t dp_device_bytes(dp_ctx *ctx);
/* Return the memory the context's pool keeps reserved to the device (waits
 * for the context stream first).  No effect with allocation hooks. */
dp_status dp_trim(dp_ctx *ctx);

/* ---- gauge fields (Sec. I: D[U]; Sec. II: O(a)-improved operator) -------- */

/* Upload and pack a gauge field: lexicographic complex128 links (layout above)
 * to even-odd, site-blocked SoA on the device in FP64 (18 reals) and FP32 (12
 * and 18 reals) copies.  The 16-bit copies (rows 0 and 1 as FP16 or BF16
 * times one FP32 scale per link, the largest modulus of those six entries)
 * are made from the FP64 links the first time a DP_PREC_MIXED_FP16 / _BF16
 * call needs them.
 * bc_t = -1 antiperiodic time (the paper's case, Sec. II), +1 periodic, 0
 * Dirichlet: no quark hop across t = T-1 <-> 0, the boundary of the
 * Schroedinger-functional setting the paper recommends the method for (end of
 * Sec. II; profile exp: alpha_B = exp(+alpha0 y0)).  Only the quark field sees
 * the boundary: the clover term is built from the given (periodic) links, and
 * there are no boundary fields or boundary improvement terms. */
dp_status dp_field_load(dp_ctx *ctx, const double *links, const int dims[4], int bc_t,
                        dp_field *out);
/* Build the clover term c_sw (i/4) sigma.Fhat for this field (FP64, two
 * Hermitian 6x6 chiral blocks per site). */
dp_status dp_field_set_csw(dp_ctx *ctx, dp_field field, double csw);
dp_status dp_field_free(dp_ctx *ctx, dp_field field);

/* ---- solves (Sec. I-III: source scaling, solve, restore, contract) ------- */

/* Point source at src = {t, x, y, z} for all 12 spin-colour components, one
 * mass M and profile.  Scales the source by alpha_B(x_src), solves the
 * even-odd Schur system of (D'+M) to relative residue r (stopping on the
 * preconditioned system, Sec. II), reconstructs the odd sites, restores
 * S = S'/alpha_B per site and contracts C_PP.  cpp_out: host [T]; prop_out:
 * NULL or host [12][V][4][3] restored propagator; info may be NULL.
 * Returns DP_ERR_NOT_CONVERGED if max_iter ran out (results still written). */
dp_status dp_solve_point(dp_ctx *ctx, dp_field field, double M, const dp_profile *profile,
                         const int src[4], double r, const dp_solve_opts *opts,
                         double *cpp_out, double *prop_out, dp_solve_info *info);

/* Several masses, each with its own profile, sharing one point source: all
 * 12 x n_mass RHS run in one multi-RHS solve.  cpp_out: host [n_mass][T];
 * prop_out NULL or host [n_mass][12][V][4][3]; info NULL or [n_mass]. */
dp_status dp_solve_point_multi(dp_ctx *ctx, dp_field field, int n_mass, const double *M,
                               const dp_profile *profiles, const int src[4], double r,
                               const dp_solve_opts *opts, double *cpp_out, double *prop_out,
                               dp_solve_info *info);

/* dp_solve_point plus the axial-pseudoscalar correlator of the same pair of
 * degenerate quarks, from the same restored propagator:
 *   cap_out[y0] = C_AP(y0) = sum_{y vec} tr[gamma_0 S(y) S(y)^dag]
 * (= -tr[gamma_0 gamma_5 S(y,x) gamma_5 S(x,y)] by gamma_5-hermiticity), y0
 * relative to the source time, host [T], caller-owned, non-NULL.  The PCAC
 * mass the paper labels its quark masses with (Sec. II) is then
 * [C_AP(y0+1) - C_AP(y0-1)] / (4 C_PP(y0)).  Other arguments as
 * dp_solve_point (no propagator output). */
dp_status dp_solve_point_corr(dp_ctx *ctx, dp_field field, double M, const dp_profile *profile,
                              const int src[4], double r, const dp_solve_opts *opts, double *cpp_out,
                              double *cap_out, dp_solve_info *info);

/* A heavy and a light quark from the same point source, each with its own
 * mass and profile, in one batch; besides each one's C_PP (cpp_out
 * [2][T], heavy first) the heavy-light pseudoscalar correlator
 *   hl_out[2 y0 + {0, 1}] = (re, im) of -sum_{y vec} tr[S_h(y) S_l(y)^dag]
 * (= -tr[gamma_5 S_h(y,x) gamma_5 S_l(x,y)]), each propagator restored by its
 * own profile before the contraction (Sec. III); y0 relative to the source
 * time, host [T][2], caller-owned.  With equal masses and profiles it
 * equals C_PP.  info: [2].  Always one batched solve. */
dp_status dp_solve_point_hl(dp_ctx *ctx, dp_field field, double M_h, const dp_profile *profile_h,
                            double M_l, const dp_profile *profile_l, const int src[4], double r,
                            const dp_solve_opts *opts, double *cpp_out, double *hl_out,
                            dp_solve_info *info);

/* As dp_solve_point_multi, but cpp_out is DEVICE memory ([n_mass][T] doubles)
 * written on the context stream; nothing is copied to the host except the
 * convergence flags the iteration loop reads. */
dp_status dp_solve_point_dev(dp_ctx *ctx, dp_field field, int n_mass, const double *M,
                             const dp_profile *profiles, const int src[4], double r,
                             const dp_solve_opts *opts, double *cpp_out_dev,
                             dp_solve_info *info);

/* Restore and contract a preconditioned propagator already on the device
 * (Sec. II eq. backcorrection; Sec. III, restore before contracting):
 * S = S'/alpha_B per site, C_PP(y0) = -sum_{y vec} sum |S|^2 with
 * y0 = (t - src_t) mod T.  xe/xo: device FP64 S' of the even/odd sites in the
 * packed layout [12 components][V/2 sites][n_groups*12 RHS] of complex128
 * (site s of parity p is the half index i>>1 of a site with (t+x+y+z)&1 = p);
 * RHS 12g..12g+11 belong to group g, whose profile and source are
 * profiles[g] and src[4g..4g+3].  cpp_dev: device [n_groups][T].  Device
 * scratch (tables and per-slice partial sums, a few hundred KB) comes from the
 * context allocator.  Runs on the context stream; returns after the stream
 * work is queued. */
dp_status dp_restore_contract_dev(dp_ctx *ctx, dp_field field, int n_groups,
                                  const dp_profile *profiles, const int *src, const double *xe,
                                  const double *xo, double *cpp_dev);

/* The same restore and contraction as dp_restore_contract_dev, for callers
 * that must not allocate device memory: an application whose own allocator
 * already holds the free device memory (a cudaMalloc from the library would
 * fail or fragment it), or a latency-bound loop that cannot afford an
 * allocation or an out-of-memory failure in the middle of a run.  The paper
 * has no counterpart; it is an interface choice of this library.
 *
 * The device scratch is one fixed array inside the library (about 1.1 MB on
 * every GPU that loads the library, held until the process exits): profile
 * tables, slot descriptors and the per-slice partial sums, sized for T <= 256,
 * up to 64 partial sums per time slice (always the case for extents <= 256)
 * and n_groups <= 5 (the 64 RHS slots of a batch hold five 12-component
 * groups).  Larger requests return DP_ERR_INVALID_ARG.  No
 * cudaMalloc, cudaFree or other allocating call is made.
 *
 * The first call on a device looks up the array's device address (with that
 * device current) and keeps it; make that first call before any stream
 * capture.  A device reset (cudaDeviceReset) unloads the array with everything
 * else, and every dp_ctx on that device must then be destroyed and created
 * again: creating a context on a device forgets the kept address, so the next
 * call looks it up anew (make that call, too, before any stream capture).
 * The host-side tables of a call live in per-thread storage (about 82 KiB per
 * calling thread, set up by the loader), not on the caller's stack.  Every
 * call shares the one array and it keeps the last call's
 * contents (nothing needs clearing: each value read is written earlier in the
 * same call).  Calls that overlap on the GPU (other threads, other contexts on
 * the same device) race on the array: serialise them.  Arguments, layouts and
 * results are those of dp_restore_contract_dev; the call returns after its
 * work on the context stream has finished. */
dp_status dp_restore_contract_noalloc(dp_ctx *ctx, dp_field field, int n_groups,
                                      const dp_profile *profiles, const int *src, const double *xe,
                                      const double *xo, double *cpp_dev);

/* ---- operator application (host buffers; for checks and small jobs) ----- */

typedef enum {
    DP_APPLY_HOP = 0,       /* hopping part only (with profile factors)        */
    DP_APPLY_CLOVER = 1,    /* clover term c_sw (i/4) sigma.Fhat only            */
    DP_APPLY_FULL = 2,      /* (D'+M) psi                                        */
    DP_APPLY_CLOVER_INV = 3 /* (4 + M + clover)^-1 psi                           */
} dp_apply_kind;

/* out = op(in) for nrhs host spinors [nrhs][V][4][3] (complex128), computed
 * in precision `prec` (DP_PREC_FP64; the mixed precisions: FP32 kernels with
 * FP32-rounded inputs and the links of that precision).  The profile is
 * placed relative to src (NULL src: the origin).  compress12 selects 12-real
 * FP32 links. */
dp_status dp_apply(dp_ctx *ctx, dp_field field, int kind, double M, const dp_profile *profile,
                   const int src[4], int prec, int compress12, const double *in, double *out,
                   int nrhs);

/* Host-only (no GPU needed): the profile factors and hop coefficients the
 * solver uses for this geometry, profile and source.  alpha_out: [4][Lmax]
 * alpha_B,mu(x_mu); hop_out: [4][2][Lmax], [mu][0][x] = -1/2 alpha_B(x)/
 * alpha_B(x+1) (forward), [mu][1][x] = -1/2 alpha_B(x)/alpha_B(x-1)
 * (backward), with bc_t on the hops across t = T-1 <-> 0 (Sec. II modified
 * derivatives, eq. redeftbc; Sec. III eq. redefcovs).  Lmax = max(dims);
 * entries beyond L_mu are 1 (alpha) and 0 (hop). */
dp_status dp_profile_tables(const int dims[4], int bc_t, const dp_profile *profile,
                            const int src[4], double *alpha_out, double *hop_out);

/* ---- correlator analysis (host only, no GPU) ------------------------------
 * The paper plots effective masses of C_PP (Sec. III, Figs. 1-2) without
 * writing a definition out.  c holds C(y0), y0 = 0..T-1 relative to the
 * source (the layout dp_solve_point returns); caller-owned, only read. */

/* Effective mass per y0 = 0..T-2 into m_out[T-1].  kind 0: the log ratio
 * ln[C(y0)/C(y0+1)].  kind 1: the cosh form for two-sided decay round the
 * periodic time direction, the m > 0 with C(y0)/C(y0+1) =
 * cosh[m (T/2 - y0)] / cosh[m (T/2 - y0 - 1)] (bisection on (0, 50]).  NaN
 * where the ratio is not positive or the form cannot reach it.  Errors:
 * null pointers, T < 2, another kind (DP_ERR_INVALID_ARG). */
dp_status dp_effective_mass(const double *c, int T, int kind, double *m_out);

/* PCAC mass from the two correlators dp_solve_point_corr returns (the paper
 * labels its quark masses by am_PCAC, Sec. II):
 *   m_out[y0] = [C_AP(y0+1) - C_AP(y0-1)] / (4 C_PP(y0)),  y0 = 1..T-2,
 * the symmetric lattice derivative of the local axial current over twice the
 * pseudoscalar density correlator, no O(a) improvement term (the paper names
 * none); m_out[0] = m_out[T-1] = NaN.  cpp, cap, m_out: [T], caller-owned.
 * Errors: null pointers, T < 3 (DP_ERR_INVALID_ARG). */
dp_status dp_pcac_mass(const double *cpp, const double *cap, int T, double *m_out);

/* Fit of C(y0) = A exp(-m y0) (kind 0) or A [exp(-m y0) + exp(-m (T - y0))]
 * (kind 1) over y0 = t0..t1 by least squares in the relative deviations
 * A f(y0)/C(y0) - 1 (one configuration: no statistical weights).  A takes
 * its closed-form minimum for each m; m is located by a log-spaced scan of
 * [1e-4, 20] and golden-section search.  Out: m, A (may be NULL) and the rms
 * relative deviation (may be NULL).  Errors: 0 <= t0 < t1 < T violated, a
 * zero, non-finite value or sign change in the window (DP_ERR_INVALID_ARG). */
dp_status dp_fit_correlator(const double *c, int T, int kind, int t0, int t1, double *m_out,
                            double *A_out, double *rms_out);

/* ---- device-resident operator for benchmarks and the autotuner ---------- */

/* One hopping application D_{p,1-p} with the fused clover-inverse epilogue
 * (out = A_pp^-1 D_{p,1-p} in), on packed even-odd device spinors of nrhs
 * right-hand sides.  FP64 layout: double2 [12 components][V/2][nrhs]
 * (component = 3*spin + colour).  FP32 layout (RHS pairs): float4
 * [12 components][V/2][nrhs/2] holding (re_2q, re_2q+1, im_2q, im_2q+1) of
 * pair q.  `in`/`out` are device pointers the caller allocated with
 * dp_spinor_bytes().  Launch shape from the tuner unless given:
 * block_threads > 0 sets the block; rhs_per_thread selects the RHS per
 * thread (FP64: 1; FP32: 2 or 4, i.e. one or two RHS pairs of the paired
 * layout, 4 needing nrhs % 4 == 0), 0 the tuned or default choice; stages
 * selects how neighbour spinors and links reach the thread: 0 direct loads,
 * 2-3 staged through shared memory with that many of the 8 directions in
 * flight, 4 staged (2 in flight) by one persistent wave of blocks whose
 * threads walk several sites (staging needs 64, 96 or 128 threads per
 * block), 5 direct loads with an L1 prefetch 2 directions ahead, 6 the
 * spinor alone staged (2 in flight) with the link read from L1, 16 warps
 * per SM (64, 96 or 128 threads per block); all of 2-6 need 2 RHS per
 * thread and FP32 or 16-bit 12-real links (6 also takes FP32 18-real
 * links).  -1: the tuned or default choice.
 * FP32 needs nrhs even.  iters launches back to back; if ms_out is non-NULL
 * it receives the average launch time measured with CUDA events on the
 * context stream. */
size_t dp_spinor_bytes(dp_ctx *ctx, dp_field field, int prec, int nrhs);
dp_status dp_dslash_dev(dp_ctx *ctx, dp_field field, double M, const dp_profile *profile,
                        int prec, int compress12, int out_parity, const void *in, void *out,
                        int nrhs, int block_threads, int rhs_per_thread, int stages, int iters,
                        float *ms_out);

/* The even-odd Schur operator of the preconditioned system (Sec. II, eq.
 * linsysprec, reduced to parity p = `parity`, q = 1 - p):
 *   dagger = 0:  out = Mhat in = in - A_pp^-1 D_pq A_qq^-1 D_qp in
 *   dagger = 1:  out = Mhat^dag in = in - g5 D~_pq A_qq^-1 D~_qp g5 A_pp^-1 in
 * with A = 4 + M + clover, D the hopping part with the profile placed at src
 * (NULL: origin) and D~ the hopping part of the reciprocal profile 1/alpha_B
 * (D(alpha_B)^dag = g5 D(1/alpha_B) g5).  These are the operators the BiCGStab
 * and CGNE solvers apply.  in/out: distinct device arrays of one parity in the
 * packed layout of `prec` (see dp_dslash_dev), caller-owned; scratch (two
 * spinor arrays, two hop tables) comes from the context allocator.  FP32 and
 * 16-bit precisions need nrhs even.  Returns after the stream work finished. */
dp_status dp_schur_dev(dp_ctx *ctx, dp_field field, double M, const dp_profile *profile,
                       const int src[4], int prec, int compress12, int parity, int dagger,
                       const void *in, void *out, int nrhs);

/* ---- autotuner ----------------------------------------------------------- */

/* Time candidate launch shapes of the multi-RHS dslash for this field,
 * precision and nrhs (64-256 threads per block x the RHS-per-thread and
 * staging choices of dp_dslash_dev), and keep the fastest for the solver's
 * later launches.  best_* may be NULL.  DP_ERR_INVALID_ARG if no shape serves
 * nrhs (FP32 with an odd count). */
dp_status dp_autotune(dp_ctx *ctx, dp_field field, int prec, int compress12, int nrhs,
                      int *best_block_threads, int *best_rhs_per_thread, int *best_stages,
                      float *best_ms);

/* Set the launch shape of the Schur dslash for (this field's volume, prec,
 * link format from compress12, nrhs) without timing, e.g. a shape an earlier
 * dp_autotune reported and the caller kept (a tune cache), so that a rerun
 * (under a profiler, say) launches the same kernels.  The shape is checked
 * as dp_dslash_dev checks an explicit one (stages 0 with rhs_per_thread 1, 2
 * or 4 by precision, 2-6 for FP32 pairs); DP_ERR_INVALID_ARG if it cannot
 * serve nrhs. */
dp_status dp_tune_set(dp_ctx *ctx, dp_field field, int prec, int compress12, int nrhs,
                      int block_threads, int rhs_per_thread, int stages);

/* ---- per-kernel timing (CUDA events on the context stream) ---------------- */

/* Enable (1) or disable (0) event timing around every kernel launch the
 * solvers make; statistics accumulate per kernel name until reset. */
dp_status dp_timing_enable(dp_ctx *ctx, int on);
dp_status dp_timing_reset(dp_ctx *ctx);
/* Statistics of kernel class `name`: launches and total milliseconds of
 * stream time while timing is on.  Classes: "dslash_fp32", "dslash_fp64",
 * "dslash_df" (operator launches), "clover_apply", "sap_block", the inner
 * solvers' BLAS passes ("blas_alpha", "blas_s", "blas_omega", "blas_update",
 * "blas_p"), "outer_blas", "slice_norms", and the solver phases "admit",
 * "round", "harvest".  Synchronises the stream. */
dp_status dp_timing_get(dp_ctx *ctx, const char *name, long *launches, double *total_ms);
/* Kernel launches made by this context since creation. */
long dp_launch_count(dp_ctx *ctx);

/* ---- serving: continuous batching over resident fields -------------------- */

typedef struct {
    dp_field field;
    double M;
    dp_profile profile;   /* TABLE pointers are copied at submit time */
    int src[4];
    double r;
    int prec;             /* dp_prec */
    double slice_tol;     /* as dp_solve_opts.slice_tol (0: max(10 r, 1e-8))  */
} dp_request;

typedef struct {
    long submitted, completed, rejected, in_flight;
    double p50_ms, p99_ms, mean_ms; /* submit -> completion latency */
    double solves_per_s;            /* completions / (last - first completion) */
    size_t hbm_budget, hbm_in_use;
    int max_concurrent_batches;     /* most field batches inside a round at once */
    long yields;                    /* inner solves ended at a convergence check to
                                       admit a waiting request                     */
} dp_serve_stats;

/* Start the scheduler.  One solver batch per field with work, each on a
 * CUDA stream of its own and driven by a host thread of its own, so rounds of
 * different fields run concurrently on the device; requests join their
 * field's batch between defect-correction rounds as slots free up.  When a
 * request arrives for a field whose batch has free slots while a round runs,
 * the inner solve ends at its next convergence check (after at least 8
 * iterations; the partial correction is a valid defect-correction step) and
 * the request is admitted at once instead of after the whole round.
 * hbm_budget: bytes of solver state the scheduler may hold for admitted
 * requests (0: 80% of free memory); max_slots: RHS slots per field batch
 * (multiple of 12, 0: 48).  Per-kernel timing (dp_timing_*) covers work on
 * the context stream only, not the scheduler's batches. */
dp_status dp_serve_start(dp_ctx *ctx, size_t hbm_budget, int max_slots);
/* Queue a request; the library copies it.  DP_ERR_REJECTED if it can never fit
 * the HBM budget or the scheduler is not running. */
dp_status dp_submit(dp_ctx *ctx, const dp_request *req, dp_ticket *ticket);
/* Wait up to timeout_s (< 0: forever) for a ticket; DP_ERR_TIMEOUT if not done.
 * cpp_out: host [T] of the request's field; info may be NULL. */
dp_status dp_wait(dp_ctx *ctx, dp_ticket ticket, double timeout_s, double *cpp_out,
                  dp_solve_info *info);
/* Cancel a queued (not yet admitted) request. */
dp_status dp_cancel(dp_ctx *ctx, dp_ticket ticket);
dp_status dp_serve_stats_get(dp_ctx *ctx, dp_serve_stats *out);
/* Stop the scheduler after draining (drain=1) or cancelling (drain=0) queued work. */
dp_status dp_serve_stop(dp_ctx *ctx, int drain);

#ifdef __cplusplus
}
#endif

#endif /* DPRE_H */
