// The method for point-source jobs on one gauge field, as a slot-based batch:
//
//   1. profile tables and source scaling eta' = alpha_B(x_src) eta
//      (Sec. II eq. redeft; Sec. III eq. redefa);
//   2. even-odd Schur form of (D'+M) S' = eta' (eq. linsysprec):
//        Mhat = 1 - A_ee^-1 D_eo A_oo^-1 D_oe,
//        bhat = A_ee^-1 (eta'_e - D_eo A_oo^-1 eta'_o);
//   3. Krylov solve of Mhat x_e = bhat to relative residue r (eq. stopping,
//      read as a relative L2 norm on the preconditioned system): an FP64
//      defect-correction loop (true Schur residual in FP64 every round) around
//      an inner solver in FP32 (mixed precision) or FP64 (plain): BiCGStab
//      (the FP32 one in shadow form: rhat' = Mhat^dag rhat once per inner
//      solve, so its inner products ride in the passes that form s and p and
//      in the dslash launch that forms t, and the p update in the x, r
//      pass), CG on the normal equations, or GCR preconditioned by the
//      Schwarz alternating procedure (sap.cu);
//   4. x_o = A_oo^-1 (eta'_o - D_oe x_e);
//   5. restore S = S'/alpha_B per site and contract C_PP(y0) (Sec. II eq.
//      backcorrection; Sec. III: restore before contracting).
//
// A batch holds n RHS slots.  A job (one mass, profile and source; 12
// spin-colour components, or one component for the unbatched FP64 baseline)
// occupies contiguous slots.  Jobs are admitted and completed between rounds,
// which is what the request scheduler uses for continuous batching.  Every
// decision (convergence, breakdown, iteration cap) is per RHS on the device
// and converged or empty slots are masked out of every kernel, so a job's
// arithmetic does not depend on the other slots.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "batch.h"

namespace dp {

#define CK(expr)                                                                 \
    do {                                                                         \
        cudaError_t e_ = (expr);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            set_error("%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return DP_ERR_CUDA;                                                  \
        }                                                                        \
    } while (0)

namespace {

// stream time of a scope under the context's kernel timing (a no-op when
// timing is off or while a graph is captured)
struct Timed {
    Ctx *c;
    const char *name;
    cudaEvent_t ev;
    cudaStream_t st;
    Timed(Ctx *c_, cudaStream_t s, const char *n) : c(c_), name(n), st(s) { c->time_begin(name, &ev, st); }
    ~Timed() { c->time_end(name, ev, st); }
};

dp_status dslash(Ctx *c, const Op &op, int parity, int epi, const void *in, void *out,
                 const void *x, const int *mask, int mask_stride, void *dots = nullptr)
{
    DslashParams P{};
    P.in = in;
    P.out = out;
    P.x = x;
    P.dots = dots;
    const Field &f = *op.f;
    P.links[0] = op.links[0];
    P.links[1] = op.links[1];
    for (int k = 0; k < kMaxGroups; k++) P.clov[k] = op.inv[parity][k];
    P.hop = op.hop;
    P.active = mask;
    P.active_stride = mask_stride;
    P.g = f.g;
    P.parity = parity;
    P.nrhs = op.nrhs;
    memcpy(P.grp_of, op.grp_of, sizeof P.grp_of);
    const char *name = op.pr == 0 ? "dslash_fp64" : "dslash_fp32";
    cudaEvent_t ev;
    c->time_begin(name, &ev, op.st);
    const bool schur = epi == EPI_AINV || epi == EPI_XMY_AINV;
    const int rpt = schur ? op.rpt : (op.pr == 0 ? 1 : 2);
    // the Schur launches take the tuned shape; the adjoint's x - g5 D launch
    // (CGNE) too when that shape is the spinor-staged kernel
    const bool shaped = schur || (epi == EPI_XMY_G5 && op.stages == 6);
    const int stages =
        shaped && dslash_staged_ok(op.pr, op.lf, epi, rpt, op.stages, op.block) ? op.stages : 0;
    CK(launch_dslash(P, op.pr, op.lf, epi, op.block, rpt, op.st, stages));
    c->time_end(name, ev, op.st);
    c->launches++;
    return DP_OK;
}

constexpr int kStateStride = (int)(sizeof(RhsState) / sizeof(int));

void set_shape(Op &op, const Shape &sh)
{
    op.block = sh.block;
    op.rpt = sh.rpt;
    op.stages = sh.stages;
}

const int *state_mask(const RhsState *st) { return st ? &st[0].active : nullptr; }

// Schur operator on parity p (q = 1 - p):
// y = Mhat x = x - A_pp^-1 D_pq A_qq^-1 D_qp x ; tmp (parity q) keeps A_qq^-1 D_qp x;
// dots (FP32, or NULL): the second launch also leaves the per-site sums of
// <y, x> and |y|^2 there (DslashParams::dots)
dp_status apply_mhat(Ctx *c, const Op &op, int p, const void *x, void *y, void *tmp,
                     const RhsState *mask, void *dots = nullptr)
{
    dp_status s = dslash(c, op, 1 - p, EPI_AINV, x, tmp, nullptr, state_mask(mask), kStateStride);
    if (s != DP_OK) return s;
    return dslash(c, op, p, EPI_XMY_AINV, tmp, y, x, state_mask(mask), kStateStride, dots);
}

// Adjoint Schur operator.  With the hopping part H(alpha_B) and the clover
// blocks A (Hermitian, commuting with gamma5), H(alpha_B)^dag =
// gamma5 H(1/alpha_B) gamma5, so
//   Mhat^dag y = y - gamma5 H~_pq A_qq^-1 H~_qp gamma5 A_pp^-1 y,
// H~ the hopping part with the reciprocal profile (op_adj's tables).
// tmp_p (parity p) and tmp_q (parity q) are scratch.
dp_status apply_mhat_dag(Ctx *c, const Op &op, const Op &op_adj, int p, const void *y, void *out,
                         void *tmp_p, void *tmp_q, const RhsState *mask)
{
    CloverApplyParams cp{};
    for (int k = 0; k < kMaxGroups; k++) cp.mat[k] = op.inv[p][k];
    memcpy(cp.grp_of, op.grp_of, sizeof cp.grp_of);
    cp.mask = state_mask(mask);
    cp.mask_stride = kStateStride;
    cp.g5 = 1;
    cp.in = y;
    cp.out = tmp_p;
    cp.Vh = op.f->g.Vh;
    cp.nrhs = op.nrhs;
    cudaEvent_t ev;
    c->time_begin("clover_apply", &ev, op.st);
    CK(launch_clover_apply(cp, op.pr, op.st));
    c->time_end("clover_apply", ev, op.st);
    c->launches++;
    dp_status s = dslash(c, op_adj, 1 - p, EPI_AINV, tmp_p, tmp_q, nullptr, state_mask(mask), kStateStride);
    if (s != DP_OK) return s;
    return dslash(c, op_adj, p, EPI_XMY_G5, tmp_q, out, y, state_mask(mask), kStateStride);
}

}  // namespace

Batch::Batch(Ctx *cc, std::shared_ptr<Field> ff, int nslots, const dp_solve_opts &o, int round_cap,
             int schur_parity, bool own_stream)
    : c(cc), f(std::move(ff)), own_stream_(own_stream), n(nslots), opts(o), round_iters(round_cap),
      sp(schur_parity & 1)
{
    st_ = c->stream;
    bc_ = c->bc;
    hnact_ = c->h_nactive;
}

Batch::~Batch()
{
    if (own_stream_ && st_) cudaStreamSynchronize(st_);  // the memory below is in use there
    if (graph) cudaGraphExecDestroy(graph);
    for (void *p : owned) c->release(p);
    if (own_stream_) {
        if (st_) cudaStreamDestroy(st_);
        if (hnact_) cudaFreeHost(hnact_);
    }
}

void *Batch::get(size_t bytes)
{
    void *p = c->alloc(bytes);
    // pool memory is usable on another stream once the context stream has
    // reached its allocation
    if (p && own_stream_ && cudaStreamSynchronize(c->stream) != cudaSuccess) p = nullptr;
    if (p) {
        owned.push_back(p);
        total_bytes += bytes;
    }
    return p;
}

size_t Batch::bytes_needed(const Geom &g, int nslots, int prec)
{
    const size_t v64 = (size_t)g.Vh * nslots * 24 * sizeof(double);
    const size_t vin = (size_t)g.Vh * nslots * 24 * (prec == DP_PREC_FP64 ? 8 : 4);
    // FP32 BiCGStab: rhat' and the omega sums (vin / 8) besides the 8 vectors
    const size_t shadow = prec == DP_PREC_FP64 ? 0 : vin + vin / 8;
    return 6 * v64 + 8 * vin + shadow + ((size_t)1 << 20);
}

dp_status Batch::init()
{
    const Geom &g = f->g;
    if (own_stream_) {
        st_ = nullptr;
        hnact_ = nullptr;
        CK(cudaStreamCreateWithFlags(&st_, cudaStreamNonBlocking));
        CK(cudaMallocHost(&hnact_, sizeof(int)));
        bc_ = BlasCtx{};
        bc_.blocks = c->bc.blocks;
        bc_.partials = (double *)get((size_t)bc_.blocks * kMaxRhs * kRedWidth * sizeof(double));
        bc_.counter = (unsigned int *)get(256);
        bc_.n_active = (int *)get(256);
        if (!bc_.partials || !bc_.counter || !bc_.n_active) {
            set_error("out of device memory for a solver batch's reduction scratch");
            return DP_ERR_OOM;
        }
    }
    mixed = opts.prec != DP_PREC_FP64;
    ipr = mixed ? 1 : 0;
    ilf = inner_link_format(opts.prec, opts.compress12);
    const long long Vh = g.Vh;
    const int Lm = g.Lmax;
    v64 = (size_t)Vh * n * 24 * sizeof(double);
    vin = (size_t)Vh * n * 24 * (ipr == 0 ? 8 : 4);
    bh = (double2 *)get(v64);
    x = (double2 *)get(v64);
    r64 = (double2 *)get(v64);
    y64 = (double2 *)get(v64);
    to64 = (double2 *)get(v64);
    t64 = (double2 *)get(v64);
    bool ok = bh && x && r64 && y64 && to64 && t64;
    void **iv[8] = {&in.r, &in.rh, &in.p, &in.v, &in.s, &in.t, &in.x, &in.to};
    for (auto pp : iv) {
        *pp = get(vin);
        ok = ok && *pp;
    }
    if (mixed && opts.solver == DP_SOLVER_BICGSTAB) {
        in.rh2 = get(vin);
        in.dots = get(vin / 8);
        ok = ok && in.rh2 && in.dots;
    }
    outer = (RhsState *)get(sizeof(RhsState) * kMaxRhs);
    inner = (RhsState *)get(sizeof(RhsState) * kMaxRhs);
    alpha_d = (double *)get(sizeof(double) * kMaxGroups * 4 * Lm);
    hop64_d = (double *)get(sizeof(double) * kMaxGroups * 8 * Lm);
    hop32_d = (float *)get(sizeof(float) * kMaxGroups * 8 * Lm);
    hopadj64_d = (double *)get(sizeof(double) * kMaxGroups * 8 * Lm);
    hopadj32_d = (float *)get(sizeof(float) * kMaxGroups * 8 * Lm);
    alpha_in_d = (double *)get(sizeof(double) * kMaxGroups * 4 * Lm);
    if (ipr == 0) hopin64_d = (double *)get(sizeof(double) * kMaxGroups * 8 * Lm);
    slice_d = (double *)get(sizeof(double) * kMaxGroups * 2 * g.T);
    slots_d = (SlotInfo *)get(sizeof(SlotInfo) * kMaxRhs);
    tsrc_d = (int *)get(sizeof(int) * kMaxGroups);
    mask_d = (int *)get(sizeof(int) * kMaxRhs);
    cpp_d = (double *)get(sizeof(double) * kMaxGroups * g.T);
    cap_d = (double *)get(sizeof(double) * kMaxGroups * g.T);
    cpart = (double *)get(sizeof(double) * 2 * (size_t)g.T * contract_blocks_per_slice(g) * kMaxGroups);
    nrm_d = (double *)get(sizeof(double) * kMaxRhs);
    ok = ok && outer && inner && alpha_d && hop64_d && hop32_d && hopadj64_d && hopadj32_d &&
         alpha_in_d && (ipr != 0 || hopin64_d) && slice_d && slots_d && tsrc_d && mask_d &&
         cpp_d && cap_d && cpart && nrm_d;
    if (!ok) {
        set_error("out of device memory for a %d-slot solver batch (%zu bytes per FP64 vector)", n, v64);
        return DP_ERR_OOM;
    }
    hs.assign(kMaxRhs, RhsState{});
    hin.assign(kMaxRhs, RhsState{});
    slot_job.assign(n, nullptr);
    slot_inner.assign(n, 0);
    slot_outer.assign(n, 0);
    slot_rr_prev.assign(n, 0.0);
    slot_stall.assign(n, 0);
    slots.assign(kMaxRhs, SlotInfo{});
    CK(cudaMemsetAsync(outer, 0, sizeof(RhsState) * kMaxRhs, st_));
    CK(cudaMemsetAsync(inner, 0, sizeof(RhsState) * kMaxRhs, st_));
    CK(cudaMemsetAsync(alpha_d, 0, sizeof(double) * kMaxGroups * 4 * Lm, st_));
    CK(cudaMemsetAsync(alpha_in_d, 0, sizeof(double) * kMaxGroups * 4 * Lm, st_));
    if (hopin64_d) CK(cudaMemsetAsync(hopin64_d, 0, sizeof(double) * kMaxGroups * 8 * Lm, st_));
    slice_h.assign((size_t)kMaxGroups * 2 * g.T, 0.0);
    CK(cudaMemsetAsync(hop64_d, 0, sizeof(double) * kMaxGroups * 8 * Lm, st_));
    CK(cudaMemsetAsync(hop32_d, 0, sizeof(float) * kMaxGroups * 8 * Lm, st_));
    CK(cudaMemsetAsync(hopadj64_d, 0, sizeof(double) * kMaxGroups * 8 * Lm, st_));
    CK(cudaMemsetAsync(hopadj32_d, 0, sizeof(float) * kMaxGroups * 8 * Lm, st_));

    op64 = Op{};
    op64.f = f.get();
    op64.st = st_;
    op64.pr = 0;
    op64.lf = LINK_F64_18;
    op64.links[0] = f->l64[0];
    op64.links[1] = f->l64[1];
    op64.hop = hop64_d;
    op64.nrhs = n;
    set_shape(op64, c->launch_shape(Vh, 0, LINK_F64_18, n));
    opin = op64;
    opin.pr = ipr;
    opin.lf = ilf;
    for (int p = 0; p < 2; p++) {
        dp_status e = field_links(c, *f, ilf, p, &opin.links[p]);
        if (e != DP_OK) return e;
    }
    // the inner solver's own hop tables: a job under per-slice refinement
    // solves its corrections in another profile's metric (slices.cu)
    opin.hop = ipr == 0 ? (const void *)hopin64_d : (const void *)hop32_d;
    set_shape(opin, c->launch_shape(Vh, ipr, ilf, n));
    opin_adj = opin;
    opin_adj.hop = ipr == 0 ? (const void *)hopadj64_d : (const void *)hopadj32_d;
    if (mixed && opts.solver == DP_SOLVER_SAP_GCR) {
        if (!sap_blocks(g, sap_bs, sap_nb)) {
            set_error("SAP+GCR needs even lattice extents");
            return DP_ERR_INVALID_ARG;
        }
        for (int k = 0; k < opts.gcr_nkv; k++) {
            zk[k] = get(vin);
            wk[k] = get(vin);
            if (!zk[k] || !wk[k]) {
                set_error("out of device memory for the GCR Krylov vectors");
                return DP_ERR_OOM;
            }
        }
        coef_d = (double2 *)get(sizeof(double2) * kMaxRhs);
        nrm2_d = (double *)get(sizeof(double) * kMaxRhs);
        if (!coef_d || !nrm2_d) {
            set_error("out of device memory");
            return DP_ERR_OOM;
        }
    }
    if (mixed && opts.outer_df) {
        xdf = (float4 *)get(v64);
        tdf = (float4 *)get(v64);
        hopdf_d = (float2 *)get(sizeof(float2) * kMaxGroups * 8 * Lm);
        if (!xdf || !tdf || !hopdf_d) {
            set_error("out of device memory for the double-float outer operator");
            return DP_ERR_OOM;
        }
        CK(cudaMemsetAsync(hopdf_d, 0, sizeof(float2) * kMaxGroups * 8 * Lm, st_));
        opdf = op64;
        opdf.lf = LINK_DF_18;
        for (int p = 0; p < 2; p++) {
            dp_status e = field_links(c, *f, LINK_DF_18, p, &opdf.links[p]);
            if (e != DP_OK) return e;
        }
        opdf.hop = hopdf_d;
    }
    check_every = opts.check_every > 0 ? opts.check_every : (Vh * n >= (1 << 20) ? 2 : 8);
    if (own_stream_) {
        // memory from the context's stream-ordered pool becomes usable on
        // this batch's stream once the context stream has reached it
        CK(cudaMemsetAsync(bc_.counter, 0, 256, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    CK(cudaStreamSynchronize(st_));
    return DP_OK;
}

int Batch::active_jobs() const
{
    int k = 0;
    for (auto *j : jobs)
        if (j) k++;
    return k;
}

bool Batch::can_admit(int ncomp) const
{
    if (max_jobs > 0 && active_jobs() >= max_jobs) return false;
    int free_tab = -1;
    for (int k = 0; k < kMaxGroups; k++)
        if (!jobs[k]) {
            free_tab = k;
            break;
        }
    if (free_tab < 0) return false;
    for (int s0 = 0; s0 + ncomp <= n; s0 += ncomp) {
        bool fr = true;
        for (int k = 0; k < ncomp; k++)
            if (slot_job[s0 + k]) fr = false;
        if (fr) return true;
    }
    return false;
}

dp_status Batch::upload_mask(const std::vector<int> &m)
{
    CK(cudaMemcpyAsync(mask_d, m.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st_));
    // the host vector may go away: make the copy complete before returning
    CK(cudaStreamSynchronize(st_));
    return DP_OK;
}

dp_status Batch::admit(Job *j)
{
    Timed tm(c, st_, "admit");
    const Geom &g = f->g;
    const int Lm = g.Lmax;
    int tab = -1, s0 = -1;
    for (int k = 0; k < kMaxGroups; k++)
        if (!jobs[k]) {
            tab = k;
            break;
        }
    for (int b = 0; b + j->ncomp <= n && tab >= 0; b += j->ncomp) {
        bool fr = true;
        for (int k = 0; k < j->ncomp; k++)
            if (slot_job[b + k]) fr = false;
        if (fr) {
            s0 = b;
            break;
        }
    }
    if (tab < 0 || s0 < 0) {
        set_error("no free slots in the batch");
        return DP_ERR_REJECTED;
    }
    // tables and clover inverse of the job
    std::vector<double> alpha(4 * Lm), hop(8 * Lm);
    dp_profile pf = j->grp.prof;
    for (int mu = 0; mu < 4; mu++)
        if (pf.kind == DP_PROF_TABLE) pf.table[mu] = j->grp.table[mu].data();
    dp_status s = profile_tables(pf, g, f->bc_t, j->grp.src, alpha.data(), hop.data());
    if (s != DP_OK) return s;
    double scale = 1.0;
    for (int mu = 0; mu < 4; mu++) scale *= alpha[mu * Lm + j->grp.src[mu]];
    std::shared_ptr<CloverInv> ci;
    s = get_clover_inv(c, *f, j->grp.M, &ci);
    if (s != DP_OK) return s;
    std::vector<float> hopf(hop.begin(), hop.end());
    // reciprocal profile: each hop factor -1/2 s alpha(x)/alpha(y) (s = +-1)
    // becomes -1/2 s alpha(y)/alpha(x) = (1/4) / (its original)
    std::vector<double> hopa(hop.size());
    for (size_t k = 0; k < hop.size(); k++) hopa[k] = hop[k] != 0.0 ? 0.25 / hop[k] : 0.0;
    std::vector<float> hopaf(hopa.begin(), hopa.end());
    CK(cudaMemcpyAsync(hopadj64_d + (size_t)tab * 8 * Lm, hopa.data(), sizeof(double) * 8 * Lm, cudaMemcpyHostToDevice, st_));
    CK(cudaMemcpyAsync(hopadj32_d + (size_t)tab * 8 * Lm, hopaf.data(), sizeof(float) * 8 * Lm, cudaMemcpyHostToDevice, st_));
    if (hopdf_d) {
        // double-float hop factors: nearest float, then the nearest float of the rest
        std::vector<float2> hd(hop.size());
        for (size_t k = 0; k < hop.size(); k++) {
            const float hi = (float)hop[k];
            hd[k] = make_float2(hi, (float)(hop[k] - (double)hi));
        }
        CK(cudaMemcpyAsync(hopdf_d + (size_t)tab * 8 * Lm, hd.data(), sizeof(float2) * 8 * Lm,
                           cudaMemcpyHostToDevice, st_));
        s = clover_inv_df(c, *f, *ci);
        if (s != DP_OK) return s;
        for (int p = 0; p < 2; p++) opdf.inv[p][tab] = ci->invdf[p];
    }
    CK(cudaMemcpyAsync(alpha_d + (size_t)tab * 4 * Lm, alpha.data(), sizeof(double) * 4 * Lm, cudaMemcpyHostToDevice, st_));
    CK(cudaMemcpyAsync(alpha_in_d + (size_t)tab * 4 * Lm, alpha.data(), sizeof(double) * 4 * Lm, cudaMemcpyHostToDevice, st_));
    if (hopin64_d)
        CK(cudaMemcpyAsync(hopin64_d + (size_t)tab * 8 * Lm, hop.data(), sizeof(double) * 8 * Lm, cudaMemcpyHostToDevice, st_));
    CK(cudaMemcpyAsync(hop64_d + (size_t)tab * 8 * Lm, hop.data(), sizeof(double) * 8 * Lm, cudaMemcpyHostToDevice, st_));
    CK(cudaMemcpyAsync(hop32_d + (size_t)tab * 8 * Lm, hopf.data(), sizeof(float) * 8 * Lm, cudaMemcpyHostToDevice, st_));
    const int ts = j->grp.src[0];
    CK(cudaMemcpyAsync(tsrc_d + tab, &ts, sizeof(int), cudaMemcpyHostToDevice, st_));
    invs[tab] = ci;
    for (int p = 0; p < 2; p++) {
        op64.inv[p][tab] = ci->inv64[p];
        opin.inv[p][tab] = ipr == 0 ? (const void *)ci->inv64[p] : (const void *)ci->inv32[p];
        opin_adj.inv[p][tab] = opin.inv[p][tab];
    }
    for (int k = 0; k < j->ncomp; k++) {
        SlotInfo &sl = slots[s0 + k];
        sl.group = tab;
        sl.comp = j->comp0 + k;
        sl.t = j->grp.src[0];
        sl.x = j->grp.src[1];
        sl.y = j->grp.src[2];
        sl.z = j->grp.src[3];
        sl.scale = scale;
        op64.grp_of[s0 + k] = opin.grp_of[s0 + k] = opin_adj.grp_of[s0 + k] = opdf.grp_of[s0 + k] =
            (int8_t)tab;
        slot_job[s0 + k] = j;
        slot_inner[s0 + k] = 0;
        slot_outer[s0 + k] = 0;
        slot_rr_prev[s0 + k] = 0;
        slot_stall[s0 + k] = 0;
    }
    CK(cudaMemcpyAsync(slots_d + s0, &slots[s0], sizeof(SlotInfo) * j->ncomp, cudaMemcpyHostToDevice, st_));
    j->tab = tab;
    j->slot0 = s0;
    j->src_scale = scale;
    j->slice_ok = j->refining = false;
    j->refine_rounds = j->slice_stall = 0;
    j->slice_best = j->slice_res = 0;
    jobs[tab] = j;
    if (graph) {  // kernel parameters (clover pointers, groups) changed
        cudaGraphExecDestroy(graph);
        graph = nullptr;
    }
    std::vector<int> m(n, 0);
    for (int k = 0; k < j->ncomp; k++) m[s0 + k] = 1;
    s = upload_mask(m);
    if (s != DP_OK) return s;
    const long long Vh = g.Vh;
    // eta'_p -> y64, eta'_q -> to64 (p = Schur parity; only this job's slots
    // are non-zero)
    CK(cudaMemsetAsync(y64, 0, v64, st_));
    CK(cudaMemsetAsync(to64, 0, v64, st_));
    CK(launch_point_source(g, slots_d, n, mask_d, sp == 0 ? y64 : to64, sp == 0 ? to64 : y64,
                           st_));
    CloverApplyParams cp{};
    memcpy(cp.grp_of, op64.grp_of, sizeof cp.grp_of);
    cp.mask = mask_d;
    cp.Vh = Vh;
    cp.nrhs = n;
    const int src_par = (j->grp.src[0] + j->grp.src[1] + j->grp.src[2] + j->grp.src[3]) & 1;
    if (src_par == sp) {
        // point source on the Schur parity: eta'_q = 0, bhat = A_pp^-1 eta'_p,
        // non-zero at the source site only
        for (int k = 0; k < kMaxGroups; k++) cp.mat[k] = op64.inv[sp][k];
        cp.in = y64;
        cp.out = bh;
        CK(blas_zero_masked(bh, Vh, n, mask_d, st_));
        CK(launch_clover_point(cp, g, slots_d, sp, st_));
    } else {
        // to64 <- A_qq^-1 eta'_q (in place, at the source site), bhat =
        // A_pp^-1 (eta'_p - D_pq to64)
        for (int k = 0; k < kMaxGroups; k++) cp.mat[k] = op64.inv[1 - sp][k];
        cp.in = to64;
        cp.out = to64;
        CK(launch_clover_point(cp, g, slots_d, 1 - sp, st_));
        s = dslash(c, op64, sp, EPI_AINV_XMY, to64, bh, y64, mask_d, 1);
        if (s != DP_OK) return s;
    }
    CK(blas_zero_masked(x, Vh, n, mask_d, st_));
    CK(blas_zero_masked(t64, Vh, n, mask_d, st_));
    // outer state rows: active, fresh (r = bhat, |bhat|^2 sets the threshold)
    for (int k = 0; k < j->ncomp; k++) {
        RhsState st{};
        st.active = 1;
        st.fresh = 1;
        st.tol2 = j->r * j->r;
        hs[s0 + k] = st;
    }
    CK(cudaMemcpyAsync(outer + s0, &hs[s0], sizeof(RhsState) * j->ncomp, cudaMemcpyHostToDevice, st_));
    CK(blas_residual64(bc_, bh, y64, r64, Vh, n, outer, mask_d, st_));
    c->launches += 5;
    CK(cudaStreamSynchronize(st_));
    return DP_OK;
}

dp_status Batch::bicgstab(int max_iter, int *iters_done)
{
    BlasCtx &bc = bc_;
    const int pr = opin.pr;
    const long long Vh = f->g.Vh;
    // FP32: the shadow form (blas32_s_dots / omega_dots / update_pa), with the
    // p update in the x, r update pass and rhat' = Mhat^dag rhat
    const bool fused = pr == 1;
    if (fused) {
        CK(cudaMemsetAsync(in.x, 0, vin, st_));
        CK(cudaMemsetAsync(in.v, 0, vin, st_));
        CK(blas32_init(bc, in.rh, in.r, in.rh, Vh, n, inner, st_, in.p));
        dp_status s = apply_mhat_dag(c, opin, opin_adj, sp, in.rh, in.rh2, in.s, in.to, inner);
        if (s != DP_OK) return s;
        CK(blas32_alpha(bc, in.rh2, in.p, Vh, n, inner, st_));
        CK(blas_count_active(bc, inner, n, st_));
        c->launches += 1;
    } else {
        CK(blas_bicg_init(bc, pr, in.rh, in.r, in.rh, in.p, in.v, in.x, Vh, n, inner, 0.0, st_));
    }
    c->launches += 2;
    CK(cudaMemcpyAsync(hnact_, bc.n_active, sizeof(int), cudaMemcpyDeviceToHost, st_));
    CK(cudaStreamSynchronize(st_));
    int it = 0;
    if (*hnact_ == 0) {
        *iters_done = 0;
        return DP_OK;
    }
    auto body_fused = [&]() -> dp_status {
        dp_status s = apply_mhat(c, opin, sp, in.p, in.v, in.to, inner);
        if (s != DP_OK) return s;
        {
            Timed tm(c, st_, "blas_s");
            CK(blas32_s_dots(bc, in.r, in.v, in.s, in.rh, in.rh2, Vh, n, inner, st_));
        }
        s = apply_mhat(c, opin, sp, in.s, in.t, in.to, inner, in.dots);
        if (s != DP_OK) return s;
        {
            Timed tm(c, st_, "blas_omega");
            CK(blas32_omega_dots(bc, in.dots, Vh, n, inner, st_));
        }
        {
            Timed tm(c, st_, "blas_update");
            CK(blas32_update_pa(bc, in.x, in.r, in.p, in.s, in.t, in.v, in.rh2, Vh, n, inner,
                                max_iter, st_));
        }
        c->launches += 4;
        return DP_OK;
    };
    auto body = [&](int first) -> dp_status {
        if (fused) return body_fused();
        {
            Timed tm(c, st_, "blas_p");
            CK(blas_bicg_p(bc, pr, in.r, in.p, in.v, Vh, n, inner, first, st_));
        }
        dp_status s = apply_mhat(c, opin, sp, in.p, in.v, in.to, inner);
        if (s != DP_OK) return s;
        {
            Timed tm(c, st_, "blas_alpha");
            CK(blas_bicg_alpha(bc, pr, in.rh, in.v, Vh, n, inner, st_));
        }
        {
            Timed tm(c, st_, "blas_s");
            CK(blas_bicg_s(bc, pr, in.r, in.v, in.s, Vh, n, inner, st_));
        }
        s = apply_mhat(c, opin, sp, in.s, in.t, in.to, inner);
        if (s != DP_OK) return s;
        {
            Timed tm(c, st_, "blas_omega");
            CK(blas_bicg_omega(bc, pr, in.t, in.s, Vh, n, inner, st_));
        }
        {
            Timed tm(c, st_, "blas_update");
            CK(blas_bicg_update(bc, pr, in.x, in.r, in.p, in.s, in.t, in.rh, Vh, n, inner, max_iter,
                                st_));
        }
        c->launches += 6;
        return DP_OK;
    };
    const bool graphs = opts.use_graph && !c->timing;
    while (true) {
        if (it == 0 || !graphs) {
            dp_status s = body(it == 0);
            if (s != DP_OK) return s;
        } else {
            if (!graph) {
                cudaGraph_t gr;
                CK(cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal));
                const long before = c->launches.load();
                dp_status s = body(0);
                cudaError_t ce = cudaStreamEndCapture(st_, &gr);
                c->launches = before;
                if (s != DP_OK) return s;
                CK(ce);
                CK(cudaGraphInstantiate(&graph, gr, 0));
                cudaGraphDestroy(gr);
                graph_max_iter = max_iter;
            }
            CK(cudaGraphLaunch(graph, st_));
            c->launches += fused ? 8 : 10;
        }
        it++;
        if (it >= max_iter) break;
        if (it % check_every == 0) {
            CK(cudaMemcpyAsync(hnact_, bc.n_active, sizeof(int), cudaMemcpyDeviceToHost, st_));
            CK(cudaStreamSynchronize(st_));
            if (*hnact_ == 0) break;
            if (yield_check && it >= yield_min && yield_check()) break;
        }
    }
    *iters_done = it;
    return DP_OK;
}

dp_status Batch::sap(const void *r, void *z)
{
    const long long Vh = f->g.Vh;
    CK(cudaMemsetAsync(z, 0, vin, st_));
    CK(cudaMemcpyAsync(in.s, r, vin, cudaMemcpyDeviceToDevice, st_));
    SapParams P{};
    P.res = in.s;
    P.z = z;
    P.links[0] = opin.links[0];
    P.links[1] = opin.links[1];
    for (int p = 0; p < 2; p++)
        for (int k = 0; k < kMaxGroups; k++) P.clov[p][k] = opin.inv[p][k];
    P.hop = opin.hop;
    memcpy(P.grp_of, opin.grp_of, sizeof P.grp_of);
    P.active = state_mask(inner);
    P.active_stride = kStateStride;
    P.g = f->g;
    P.parity = sp;
    P.nrhs = n;
    for (int mu = 0; mu < 4; mu++) {
        P.bs[mu] = sap_bs[mu];
        P.nb[mu] = sap_nb[mu];
    }
    P.n_mr = opts.sap_nmr;
    for (int cyc = 0; cyc < opts.sap_ncy; cyc++)
        for (int colour = 0; colour < 2; colour++) {
            P.colour = colour;
            cudaEvent_t ev;
            c->time_begin("sap_block", &ev);
            CK(launch_sap_block(P, opin.lf, st_));
            c->time_end("sap_block", ev);
            c->launches++;
            if (cyc == opts.sap_ncy - 1 && colour == 1) break;
            // global residual of the correction so far: res = r - Mhat z
            dp_status s = apply_mhat(c, opin, sp, z, in.v, in.to, inner);
            if (s != DP_OK) return s;
            CK(blas32_xmy(r, in.v, in.s, Vh, n, st_));
            c->launches++;
        }
    return DP_OK;
}

// GCR preconditioned by SAP, restarted every gcr_nkv directions; per RHS:
// z_k = SAP(r), w_k = Mhat z_k orthonormalised against w_0..w_{k-1} (the same
// combinations applied to z_k), then x += <w_k, r> z_k, r -= <w_k, r> w_k
dp_status Batch::sap_gcr(int max_iter, int *iters_done)
{
    BlasCtx &bc = bc_;
    const long long Vh = f->g.Vh;
    CK(blas_bicg_init(bc, 1, in.rh, in.r, in.rh, in.p, in.v, in.x, Vh, n, inner, 0.0, st_));
    c->launches += 2;
    CK(cudaMemcpyAsync(hnact_, bc.n_active, sizeof(int), cudaMemcpyDeviceToHost, st_));
    CK(cudaStreamSynchronize(st_));
    *iters_done = 0;
    if (*hnact_ == 0) return DP_OK;
    int it = 0;
    while (it < max_iter) {
        for (int k = 0; k < opts.gcr_nkv && it < max_iter; k++) {
            dp_status s = sap(in.r, zk[k]);
            if (s != DP_OK) return s;
            s = apply_mhat(c, opin, sp, zk[k], wk[k], in.to, inner);
            if (s != DP_OK) return s;
            for (int i = 0; i < k; i++) {
                CK(blas32_dotv(bc, wk[i], wk[k], Vh, n, inner, coef_d, st_));
                CK(blas32_mgs(bc, wk[k], zk[k], wk[i], zk[i], Vh, n, inner, coef_d, st_));
            }
            CK(blas32_norm2v(bc, wk[k], Vh, n, inner, nrm2_d, st_));
            CK(blas32_normalise(bc, wk[k], zk[k], Vh, n, inner, nrm2_d, st_));
            CK(blas32_dotv(bc, wk[k], in.r, Vh, n, inner, coef_d, st_));
            CK(blas32_gcr_update(bc, in.x, in.r, zk[k], wk[k], Vh, n, inner, coef_d, max_iter, st_));
            c->launches += 2 * k + 5;
            it++;
            CK(cudaMemcpyAsync(hnact_, bc.n_active, sizeof(int), cudaMemcpyDeviceToHost, st_));
            CK(cudaStreamSynchronize(st_));
            if (*hnact_ == 0 || (yield_check && it >= yield_min && yield_check())) {
                *iters_done = it;
                return DP_OK;
            }
        }
    }
    *iters_done = it;
    return DP_OK;
}

dp_status Batch::contract_hl(const Job &h, const Job &l, double *out_dev)
{
    if (h.slot0 < 0 || l.slot0 < 0 || h.ncomp != 12 || l.ncomp != 12) {
        set_error("heavy-light contraction needs two whole 12-RHS jobs of this batch");
        return DP_ERR_INVALID_ARG;
    }
    const Geom &g = f->g;
    CK(launch_contract_hl(sp == 0 ? x : y64, sp == 0 ? y64 : x, g, n, alpha_d, h.tab, l.tab, h.slot0,
                          l.slot0, h.grp.src[0], cpart, out_dev, st_));
    c->launches += 2;
    return DP_OK;
}

dp_status Batch::outer_mhat()
{
    if (!xdf) return apply_mhat(c, op64, sp, x, y64, t64, outer);
    // double-float: x -> xdf, tdf = A_qq^-1 D_qp xdf, y64 = x - A_pp^-1 D_pq tdf,
    // t64 <- tdf (reconstruction of the other parity)
    const Geom &g = f->g;
    const long long cnt = g.Vh * 12 * n;
    const int *mask = state_mask(outer);
    CK(launch_to_df(x, xdf, cnt, mask, n, kStateStride, st_));
    DslashParams P{};
    P.links[0] = opdf.links[0];
    P.links[1] = opdf.links[1];
    P.hop = opdf.hop;
    P.active = mask;
    P.active_stride = kStateStride;
    P.g = g;
    P.nrhs = n;
    memcpy(P.grp_of, opdf.grp_of, sizeof P.grp_of);
    cudaEvent_t ev;
    c->time_begin("dslash_df", &ev);
    P.parity = 1 - sp;
    for (int k = 0; k < kMaxGroups; k++) P.clov[k] = opdf.inv[1 - sp][k];
    P.in = xdf;
    P.out = tdf;
    CK(launch_dslash_df(P, EPI_AINV, 128, st_));
    P.parity = sp;
    for (int k = 0; k < kMaxGroups; k++) P.clov[k] = opdf.inv[sp][k];
    P.in = tdf;
    P.x = xdf;
    P.out = y64;
    CK(launch_dslash_df(P, EPI_XMY_AINV, 128, st_));
    c->time_end("dslash_df", ev);
    CK(launch_from_df(tdf, t64, cnt, mask, n, kStateStride, st_));
    c->launches += 4;
    return DP_OK;
}

// CG on the normal equations Mhat^dag Mhat x = Mhat^dag b, stopping on the
// residual of Mhat x = b itself (recursively updated r = b - Mhat x)
dp_status Batch::cgne(int max_iter, int *iters_done)
{
    BlasCtx &bc = bc_;
    const int pr = opin.pr;
    const long long Vh = f->g.Vh;
    CK(blas_bicg_init(bc, pr, in.rh, in.r, in.rh, in.p, in.v, in.x, Vh, n, inner, 0.0, st_));
    c->launches += 2;
    CK(cudaMemcpyAsync(hnact_, bc.n_active, sizeof(int), cudaMemcpyDeviceToHost, st_));
    CK(cudaStreamSynchronize(st_));
    int it = 0;
    if (*hnact_ == 0) {
        *iters_done = 0;
        return DP_OK;
    }
    // z -> in.s, w = Mhat p -> in.v; in.t and in.to are scratch
    auto body = [&](int first) -> dp_status {
        dp_status s = apply_mhat_dag(c, opin, opin_adj, sp, in.r, in.s, in.t, in.to, inner);
        if (s != DP_OK) return s;
        CK(blas_cg_gamma(bc, pr, in.s, Vh, n, inner, first, st_));
        CK(blas_cg_p(bc, pr, in.s, in.p, Vh, n, inner, st_));
        s = apply_mhat(c, opin, sp, in.p, in.v, in.to, inner);
        if (s != DP_OK) return s;
        CK(blas_cg_alpha(bc, pr, in.v, Vh, n, inner, st_));
        CK(blas_cg_update(bc, pr, in.x, in.r, in.p, in.v, Vh, n, inner, max_iter, st_));
        c->launches += 5;
        return DP_OK;
    };
    const bool graphs = opts.use_graph && !c->timing;
    while (true) {
        if (it == 0 || !graphs) {
            dp_status s = body(it == 0);
            if (s != DP_OK) return s;
        } else {
            if (!graph) {
                cudaGraph_t gr;
                CK(cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal));
                const long before = c->launches.load();
                dp_status s = body(0);
                cudaError_t ce = cudaStreamEndCapture(st_, &gr);
                c->launches = before;
                if (s != DP_OK) return s;
                CK(ce);
                CK(cudaGraphInstantiate(&graph, gr, 0));
                cudaGraphDestroy(gr);
                graph_max_iter = max_iter;
            }
            CK(cudaGraphLaunch(graph, st_));
            c->launches += 10;
        }
        it++;
        if (it >= max_iter) break;
        if (it % check_every == 0) {
            CK(cudaMemcpyAsync(hnact_, bc.n_active, sizeof(int), cudaMemcpyDeviceToHost, st_));
            CK(cudaStreamSynchronize(st_));
            if (*hnact_ == 0) break;
            if (yield_check && it >= yield_min && yield_check()) break;
        }
    }
    *iters_done = it;
    return DP_OK;
}

dp_status Batch::round()
{
    Timed tm(c, st_, "round");
    const long long Vh = f->g.Vh;
    const int max_outer = 200;
    // per-RHS stop rules on the host: stagnation of the true residual, round
    // and iteration caps
    CK(cudaMemcpyAsync(hs.data(), outer, sizeof(RhsState) * n, cudaMemcpyDeviceToHost, st_));
    CK(cudaStreamSynchronize(st_));
    int nact = 0;
    bool changed = false;
    for (int k = 0; k < n; k++) {
        if (!slot_job[k] || !hs[k].active) continue;
        // (a refined RHS is judged per slice in harvest, not by its global |r|)
        if (!hs[k].refine && slot_outer[k] > 0 && hs[k].rr >= slot_rr_prev[k]) slot_stall[k]++;
        else slot_stall[k] = 0;
        slot_rr_prev[k] = hs[k].rr;
        if (slot_stall[k] >= 3 || slot_outer[k] >= max_outer || slot_inner[k] >= opts.max_iter) {
            hs[k].active = 0;
            hs[k].status = 4;
            changed = true;
        } else {
            nact++;
        }
    }
    if (changed) CK(cudaMemcpyAsync(outer, hs.data(), sizeof(RhsState) * n, cudaMemcpyHostToDevice, st_));
    if (nact == 0) return DP_OK;
    for (int k = 0; k < n; k++)
        if (slot_job[k] && hs[k].active) slot_outer[k]++;
    const bool refine = any_refining();
    const Geom &g = f->g;
    {
        Timed tm(c, st_, "outer_blas");
        // refined RHS: |R r| in the inner solver's metric first (it may flag
        // a non-finite RHS before the inner state is set up)
        if (refine) {
            CK(blas_ratio_norm(bc_, r64, g, sp, n, alpha_d, alpha_in_d, slots_d, outer, st_));
            c->launches++;
        }
        CK(blas_inner_setup(outer, inner, n, opts.inner_tol, 0.0, st_));
        if (mixed)
            CK(blas_to_f32_scaled(r64, (float4 *)in.rh, Vh, n, outer, st_));
        else
            CK(blas_scale64(r64, (double2 *)in.rh, Vh, n, outer, st_));
        if (refine) {
            if (mixed)
                CK(blas_to_f32_ratio(r64, (float4 *)in.rh, g, sp, n, alpha_d, alpha_in_d, slots_d, outer,
                                     st_));
            else
                CK(blas_scale64_ratio(r64, (double2 *)in.rh, g, sp, n, alpha_d, alpha_in_d, slots_d,
                                      outer, st_));
            c->launches++;
        }
    }
    c->launches += 2;
    // inner budget of this round
    int budget = round_iters > 0 ? round_iters : opts.max_iter;
    int done = 0;
    dp_status s = opts.solver == DP_SOLVER_CGNE      ? cgne(budget, &done)
                  : opts.solver == DP_SOLVER_SAP_GCR ? sap_gcr(budget, &done)
                                                     : bicgstab(budget, &done);
    if (s != DP_OK) return s;
    CK(cudaMemcpyAsync(hin.data(), inner, sizeof(RhsState) * n, cudaMemcpyDeviceToHost, st_));
    CK(cudaStreamSynchronize(st_));
    bool bad = false;
    for (int k = 0; k < n; k++) {
        if (!slot_job[k] || !hs[k].active) continue;
        slot_inner[k] += hin[k].iters;
        if (hin[k].status == 3) {
            hs[k].active = 0;
            hs[k].status = 3;
            bad = true;
        }
    }
    if (bad) CK(cudaMemcpyAsync(outer, hs.data(), sizeof(RhsState) * n, cudaMemcpyHostToDevice, st_));
    {
        Timed tm(c, st_, "outer_blas");
        if (mixed)
            CK(blas_acc_f32(x, (const float4 *)in.x, Vh, n, outer, st_));
        else
            CK(blas_acc64(x, (const double2 *)in.x, Vh, n, outer, st_));
        if (refine) {
            if (mixed)
                CK(blas_acc_f32_ratio(x, (const float4 *)in.x, g, sp, n, alpha_d, alpha_in_d, slots_d,
                                      outer, st_));
            else
                CK(blas_acc64_ratio(x, (const double2 *)in.x, g, sp, n, alpha_d, alpha_in_d, slots_d,
                                    outer, st_));
            c->launches++;
        }
    }
    // t64 keeps A_qq^-1 D_qp x of this (final, once converged) x: the
    // reconstruction of the other parity reuses it
    s = outer_mhat();
    if (s != DP_OK) return s;
    {
        Timed tm(c, st_, "outer_blas");
        CK(blas_residual64(bc_, bh, y64, r64, Vh, n, outer, nullptr, st_));
    }
    c->launches += 3;
    return DP_OK;
}

bool Batch::any_refining() const
{
    for (const Job *j : jobs)
        if (j && j->refining) return true;
    return false;
}

dp_status Batch::set_inner_profile(const Job &j, const double *h)
{
    const Geom &g = f->g;
    const int Lm = g.Lmax, T = g.T, m = j.tab;
    // alpha_B,t(t) = |x_src|/|x_t| in the restored metric, times 1 in space,
    // walking away from the source.  Only slices the solution already resolves
    // (their own residual below a tenth of their norm) say how fast the
    // propagator falls; an unresolved slice holds noise (or nothing yet), so it
    // continues the slice-to-slice factor of the last resolved step (between
    // 1 and e^1.5).  No step exceeds e^{+-2}.
    constexpr double kStep = 7.389056098930650;   // e^2
    constexpr double kGrowMax = 4.481689070338065; // e^1.5
    std::vector<double> tt(T), one(Lm, 1.0);
    const int ts = j.grp.src[0];
    const double ref = h[2 * ts] > 0 && std::isfinite(h[2 * ts]) ? h[2 * ts] : 1.0;
    double prev = 1.0, growth = 1.0;
    for (int k = 0; k < T; k++) {
        const int t = (ts + k) % T;
        const double v = h[2 * t], rr = h[2 * t + 1];
        const bool resolved = v > 0 && std::isfinite(v) && std::isfinite(rr) && rr <= 0.01 * v;
        double a = resolved ? std::sqrt(ref / v) : prev * growth;
        if (!(a > 0) || !std::isfinite(a)) a = prev;
        if (k > 0) {
            a = std::min(std::max(a, prev / kStep), prev * kStep);
            if (resolved) growth = std::min(std::max(a / prev, 1.0), kGrowMax);
        }
        tt[t] = prev = a;
    }
    dp_profile pf{};
    pf.kind = DP_PROF_TABLE;
    pf.table[0] = tt.data();
    pf.table[1] = pf.table[2] = pf.table[3] = one.data();
    std::vector<double> alpha(4 * Lm), hop(8 * Lm), hopa(8 * Lm);
    dp_status s = profile_tables(pf, g, f->bc_t, j.grp.src, alpha.data(), hop.data());
    if (s != DP_OK) return s;
    for (size_t k = 0; k < hop.size(); k++) hopa[k] = hop[k] != 0.0 ? 0.25 / hop[k] : 0.0;
    CK(cudaMemcpyAsync(alpha_in_d + (size_t)m * 4 * Lm, alpha.data(), sizeof(double) * 4 * Lm,
                       cudaMemcpyHostToDevice, st_));
    if (ipr == 0) {
        CK(cudaMemcpyAsync(hopin64_d + (size_t)m * 8 * Lm, hop.data(), sizeof(double) * 8 * Lm,
                           cudaMemcpyHostToDevice, st_));
        CK(cudaMemcpyAsync(hopadj64_d + (size_t)m * 8 * Lm, hopa.data(), sizeof(double) * 8 * Lm,
                           cudaMemcpyHostToDevice, st_));
    } else {
        std::vector<float> hf(hop.begin(), hop.end()), haf(hopa.begin(), hopa.end());
        CK(cudaMemcpyAsync(hop32_d + (size_t)m * 8 * Lm, hf.data(), sizeof(float) * 8 * Lm,
                           cudaMemcpyHostToDevice, st_));
        CK(cudaMemcpyAsync(hopadj32_d + (size_t)m * 8 * Lm, haf.data(), sizeof(float) * 8 * Lm,
                           cudaMemcpyHostToDevice, st_));
        CK(cudaStreamSynchronize(st_));  // the float vectors go away
    }
    CK(cudaStreamSynchronize(st_));
    return DP_OK;
}

// Per-slice accuracy (slices.cu).  A job is checked when all its RHS passed
// the global test, and after every refinement round.  Refinement gives up
// (status 4: not converged) when two rounds in a row fail to halve the worst
// slice residual, or after kMaxRefine rounds.
dp_status Batch::slice_check(bool *changed)
{
    constexpr int kMaxRefine = 16;
    const Geom &g = f->g;
    const int T = g.T;
    std::vector<Job *> cand;
    int ng = 0;
    for (int tab = 0; tab < kMaxGroups; tab++) {
        Job *j = jobs[tab];
        if (!j || !(j->slice_tol > 0)) continue;
        bool any_active = false, all_ok = true;
        for (int k = 0; k < j->ncomp; k++) {
            const RhsState &st = hs[j->slot0 + k];
            if (st.active) any_active = true;
            else if (st.status != 1) all_ok = false;
        }
        const bool want = j->refining ? any_active : (!any_active && all_ok && !j->slice_ok);
        if (want) {
            cand.push_back(j);
            ng = std::max(ng, tab + 1);
        }
    }
    if (cand.empty()) return DP_OK;
    std::vector<int> m(n, 0);
    for (Job *j : cand)
        for (int k = 0; k < j->ncomp; k++) m[j->slot0 + k] = 1;
    dp_status s = upload_mask(m);
    if (s != DP_OK) return s;
    {
        Timed tm(c, st_, "slice_norms");
        CK(launch_slice_norms(x, r64, g, sp, n, alpha_d, slots_d, ng, mask_d, cpart, slice_d,
                              st_));
    }
    c->launches += 2;
    CK(cudaMemcpyAsync(slice_h.data(), slice_d, sizeof(double) * ng * T * 2, cudaMemcpyDeviceToHost,
                       st_));
    CK(cudaStreamSynchronize(st_));
    for (Job *j : cand) {
        const double *h = slice_h.data() + (size_t)j->tab * T * 2;
        double worst = 0;
        for (int t = 0; t < T; t++) {
            const double a = h[2 * t], b = h[2 * t + 1];
            // a slice the solution has not reached (zero norm, residual left)
            // counts as far from its target, not as a non-finite result
            const double rho = a > 0 ? std::sqrt(b / a) : (b > 0 ? 1e300 : 0.0);
            if (!(rho <= worst)) worst = rho;  // NaN propagates
        }
        j->slice_res = worst;
        // inner reduction of the next refinement round: a tenth of the factor
        // the worst slice still misses by (in the flattened metric the global
        // reduction is about the per-slice one), at least the inner solver's
        // own floor (the round's tolerance rides in the outer tol2, which the
        // global test ignores for a refined RHS)
        const double floor_tol = std::max(opts.inner_tol, 1e-12);
        const double want = std::min(0.5, std::max(floor_tol, 0.1 * j->slice_tol / worst));
        auto set_all = [&](int active, int status, int refine) {
            for (int k = 0; k < j->ncomp; k++) {
                RhsState &st = hs[j->slot0 + k];
                st.active = active;
                st.status = status;
                st.refine = refine;
                if (refine) st.tol2 = want * want;
                slot_stall[j->slot0 + k] = 0;
            }
            *changed = true;
        };
        if (j->refining) j->refine_rounds++;  // a refinement round has just finished
        if (worst <= j->slice_tol) {
            j->slice_ok = true;
            if (j->refining) set_all(0, 1, 0);
            j->refining = false;
        } else if (!j->refining) {
            if (!std::isfinite(worst)) {
                set_all(0, 3, 0);
                continue;
            }
            j->refining = true;
            j->refine_rounds = 0;
            j->slice_best = worst;
            j->slice_stall = 0;
            s = set_inner_profile(*j, h);
            if (s != DP_OK) return s;
            set_all(1, 0, 1);
        } else {
            if (worst < 0.5 * j->slice_best) {
                j->slice_best = worst;
                j->slice_stall = 0;
            } else {
                j->slice_stall++;
            }
            if (j->slice_stall >= 2 || j->refine_rounds >= kMaxRefine || !std::isfinite(worst)) {
                set_all(0, std::isfinite(worst) ? 4 : 3, 0);
                j->refining = false;
            } else {
                s = set_inner_profile(*j, h);
                if (s != DP_OK) return s;
                set_all(1, 0, 1);  // the next round's tolerance
            }
        }
    }
    return DP_OK;
}

dp_status Batch::harvest(std::vector<Job *> &finished)
{
    Timed tm(c, st_, "harvest");
    const Geom &g = f->g;
    const long long Vh = g.Vh;
    CK(cudaMemcpyAsync(hs.data(), outer, sizeof(RhsState) * n, cudaMemcpyDeviceToHost, st_));
    CK(cudaStreamSynchronize(st_));
    {
        bool changed = false;
        dp_status s = slice_check(&changed);
        if (s != DP_OK) return s;
        if (changed) {
            CK(cudaMemcpyAsync(outer, hs.data(), sizeof(RhsState) * n, cudaMemcpyHostToDevice, st_));
            CK(cudaStreamSynchronize(st_));
        }
    }
    for (int tab = 0; tab < kMaxGroups; tab++) {
        Job *j = jobs[tab];
        if (!j) continue;
        bool all = true;
        for (int k = 0; k < j->ncomp; k++)
            if (hs[j->slot0 + k].active) all = false;
        if (!all) continue;
        std::vector<int> m(n, 0);
        for (int k = 0; k < j->ncomp; k++) m[j->slot0 + k] = 1;
        dp_status s = upload_mask(m);
        if (s != DP_OK) return s;
        // other parity q = 1 - p: x_q = A_qq^-1 (eta'_q - D_qp x_p)
        //                           = A_qq^-1 eta'_q - t64, t64 = A_qq^-1 D_qp x_p
        // from the last FP64 Schur application (x_p final): no extra dslash
        // only this job's slots: the other parity of jobs finished earlier
        // stays in y64 (heavy-light contractions read it)
        CK(blas_zero_masked(y64, Vh, n, mask_d, st_));
        CK(blas_zero_masked(to64, Vh, n, mask_d, st_));
        CK(launch_point_source(g, slots_d, n, mask_d, sp == 0 ? y64 : to64, sp == 0 ? to64 : y64,
                               st_));
        CloverApplyParams cp{};
        memcpy(cp.grp_of, op64.grp_of, sizeof cp.grp_of);
        cp.mask = mask_d;
        cp.Vh = Vh;
        cp.nrhs = n;
        for (int k = 0; k < kMaxGroups; k++) cp.mat[k] = op64.inv[1 - sp][k];
        cp.in = to64;
        cp.out = to64;
        CK(launch_clover_point(cp, g, slots_d, 1 - sp, st_));
        CK(blas_sub64_masked(to64, t64, y64, Vh, n, mask_d, st_));
        // residual report: the full residual of (D'+M)S' = eta' is (A_pp rhat, 0)
        // with x_q rebuilt from x_p, so |A_pp rhat| / |eta'| (a few digits:
        // FP32 products, FP64 sums)
        for (int k = 0; k < kMaxGroups; k++) {
            cp.mat[k] = f->clov32[sp];
            cp.diag[k] = jobs[k] ? 4.0 + jobs[k]->grp.M : 0.0;
        }
        cp.in = r64;
        cp.out = nullptr;
        CK(launch_clover_norm(bc_, cp, nrm_d, st_));
        double2 *prop_d = nullptr;
        void *prop_tmp = nullptr;
        if (j->prop_host) {
            prop_tmp = c->alloc((size_t)g.V * 24 * sizeof(double) * n);
            if (prop_tmp && own_stream_) CK(cudaStreamSynchronize(c->stream));
            if (!prop_tmp) {
                set_error("out of device memory for the propagator");
                return DP_ERR_OOM;
            }
            prop_d = (double2 *)prop_tmp;
        }
        CK(launch_restore_contract(sp == 0 ? x : y64, sp == 0 ? y64 : x, g, n, alpha_d, slots_d,
                                   kMaxGroups, tsrc_d, mask_d, cpp_d, cpart, prop_d, st_,
                                   j->cap_dst ? cap_d : nullptr));
        if (j->cpp_dst) CK(launch_cpp_commit(cpp_d + (size_t)tab * g.T, j->cpp_dst, g.T, j->accumulate, st_));
        if (j->cap_dst) CK(launch_cpp_commit(cap_d + (size_t)tab * g.T, j->cap_dst, g.T, j->accumulate, st_));
        if (j->cpp_host) CK(cudaMemcpyAsync(j->cpp_host, cpp_d + (size_t)tab * g.T, sizeof(double) * g.T, cudaMemcpyDeviceToHost, st_));
        if (prop_d)
            CK(cudaMemcpyAsync(j->prop_host, prop_d + (size_t)j->slot0 * g.V * 12,
                               sizeof(double) * 24 * g.V * j->ncomp, cudaMemcpyDeviceToHost, st_));
        std::vector<double> nr(n);
        CK(cudaMemcpyAsync(nr.data(), nrm_d, sizeof(double) * n, cudaMemcpyDeviceToHost, st_));
        CK(cudaStreamSynchronize(st_));
        if (prop_tmp) c->release(prop_tmp);
        c->launches += 6;
        SolveResult &R = j->res;
        R = SolveResult{};
        R.status = DP_OK;
        R.slice_residue = j->slice_res;
        R.refine_rounds = j->refine_rounds;
        for (int k = 0; k < j->ncomp; k++) {
            const int sl = j->slot0 + k;
            R.iters_inner = std::max(R.iters_inner, slot_inner[sl]);
            R.iters_outer = std::max(R.iters_outer, slot_outer[sl]);
            R.true_rel_residue = std::max(R.true_rel_residue, std::sqrt(nr[sl]) / j->src_scale);
            const int st = hs[sl].status;
            if (st == 3) R.status = DP_ERR_NONFINITE;
            else if (st == 2 && R.status == DP_OK) R.status = DP_ERR_BREAKDOWN;
            else if (st != 1 && R.status == DP_OK) R.status = DP_ERR_NOT_CONVERGED;
            slot_job[sl] = nullptr;
        }
        jobs[tab] = nullptr;
        invs[tab].reset();
        j->done = true;
        finished.push_back(j);
    }
    return DP_OK;
}

dp_status solve_groups(Ctx *c, std::shared_ptr<Field> f, const std::vector<Group> &groups,
                       double r_target, const dp_solve_opts &o, double *cpp_dev, double *prop_host,
                       std::vector<SolveResult> &res, double *cap_dev, double *hl_dev)
{
    const Geom &g = f->g;
    const int ng = (int)groups.size();
    if (ng < 1 || 12 * ng > kMaxRhs) {
        set_error("between 1 and %d point-source groups per batch", kMaxRhs / 12);
        return DP_ERR_INVALID_ARG;
    }
    if (!(r_target > 0) || !(r_target < 1)) {
        set_error("residue r must be in (0, 1)");
        return DP_ERR_INVALID_ARG;
    }
    const int L[4] = {g.T, g.Lx, g.Ly, g.Lz};
    for (const Group &gr : groups) {
        if (!std::isfinite(gr.M)) {
            set_error("mass is not finite");
            return DP_ERR_INVALID_ARG;
        }
        for (int mu = 0; mu < 4; mu++)
            if (gr.src[mu] < 0 || gr.src[mu] >= L[mu]) {
                set_error("source coordinate %d out of range", mu);
                return DP_ERR_INVALID_ARG;
            }
    }
    res.assign(ng, SolveResult());
    const bool batched = o.batched != 0;
    // all groups share the source: solve on its parity
    const int sp = (groups[0].src[0] + groups[0].src[1] + groups[0].src[2] + groups[0].src[3]) & 1;
    // unbatched: one RHS at a time; the FP32 kernels work on RHS pairs, so the
    // mixed-precision unbatched batch has two slots and admits one job
    const bool mixed = o.prec != DP_PREC_FP64;
    Batch B(c, f, batched ? 12 * ng : (mixed ? 2 : 1), o, 0, sp);
    if (!batched) B.set_max_jobs(1);
    dp_status s = B.init();
    if (s != DP_OK) return s;
    std::vector<Job> jobs(batched ? ng : 12 * ng);
    for (size_t k = 0; k < jobs.size(); k++) {
        Job &j = jobs[k];
        const int gi = batched ? (int)k : (int)k / 12;
        j.grp = groups[gi];
        j.comp0 = batched ? 0 : (int)k % 12;
        j.ncomp = batched ? 12 : 1;
        j.r = r_target;
        j.slice_tol = slice_target(o.slice_tol, r_target);
        j.cpp_dst = cpp_dev + (size_t)gi * g.T;
        if (cap_dev) j.cap_dst = cap_dev + (size_t)gi * g.T;
        j.accumulate = batched ? 0 : (j.comp0 > 0);
        if (prop_host) j.prop_host = prop_host + ((size_t)gi * 12 + j.comp0) * g.V * 24;
    }
    // batched: all jobs at once; unbatched: one RHS after the other
    size_t next = 0;
    std::vector<Job *> fin;
    while (true) {
        while (next < jobs.size() && B.can_admit(jobs[next].ncomp)) {
            s = B.admit(&jobs[next]);
            if (s != DP_OK) return s;
            next++;
        }
        if (B.active_jobs() == 0) break;
        s = B.round();
        if (s != DP_OK) return s;
        s = B.harvest(fin);
        if (s != DP_OK) return s;
    }
    if (hl_dev) {
        if (!batched || ng != 2) {
            set_error("heavy-light contraction needs one batched solve of two masses");
            return DP_ERR_INVALID_ARG;
        }
        s = B.contract_hl(jobs[0], jobs[1], hl_dev);
        if (s != DP_OK) return s;
    }
    dp_status ret = DP_OK;
    for (int gi = 0; gi < ng; gi++) {
        SolveResult &R = res[gi];
        R.status = DP_OK;
        for (size_t k = 0; k < jobs.size(); k++) {
            const int jg = batched ? (int)k : (int)k / 12;
            if (jg != gi) continue;
            const SolveResult &J = jobs[k].res;
            if (batched) {
                R = J;
            } else {
                R.iters_inner = std::max(R.iters_inner, J.iters_inner);
                R.iters_outer = std::max(R.iters_outer, J.iters_outer);
                R.true_rel_residue = std::max(R.true_rel_residue, J.true_rel_residue);
                R.slice_residue = std::max(R.slice_residue, J.slice_residue);
                R.refine_rounds = std::max(R.refine_rounds, J.refine_rounds);
                if (J.status != DP_OK && R.status == DP_OK) R.status = J.status;
            }
        }
        if (R.status != DP_OK && ret == DP_OK) ret = (dp_status)R.status;
    }
    if (ret != DP_OK) set_error("solve finished with status %d (see per-mass info)", ret);
    return ret;
}

}  // namespace dp

using namespace dp;

static dp_status solve_common(dp_ctx *ctx, dp_field field, int n_mass, const double *M,
                              const dp_profile *profiles, const int src[4], double r,
                              const dp_solve_opts *opts, double *cpp_out, int cpp_on_device,
                              double *prop_out, dp_solve_info *info, double *cap_out = nullptr,
                              double *hl_out = nullptr)
{
    if (!ctx) {
        set_error("null context");
        return DP_ERR_INVALID_ARG;
    }
    auto t0 = std::chrono::steady_clock::now();
    Ctx &c = ctx->c;
    if (cudaSetDevice(c.device) != cudaSuccess) {
        set_error("cudaSetDevice failed");
        return DP_ERR_CUDA;
    }
    auto fp = find_field(&c, field);
    if (!fp) {
        set_error("unknown field");
        return DP_ERR_NOT_FOUND;
    }
    if (n_mass < 1 || n_mass > kMaxRhs / 12 || !M || !profiles || !src || !cpp_out) {
        set_error("invalid argument (n_mass in [1, %d], non-null M, profiles, src, cpp_out)", kMaxRhs / 12);
        return DP_ERR_INVALID_ARG;
    }
    dp_solve_opts o;
    dp_status s = check_opts(opts, &o);
    if (s != DP_OK) return s;
    if (!opts) o.batched = 1;
    const int L[4] = {fp->g.T, fp->g.Lx, fp->g.Ly, fp->g.Lz};
    std::vector<Group> groups(n_mass);
    for (int k = 0; k < n_mass; k++) {
        groups[k].M = M[k];
        groups[k].prof = profiles[k];
        for (int mu = 0; mu < 4; mu++) {
            groups[k].src[mu] = src[mu];
            if (profiles[k].kind == DP_PROF_TABLE) {
                if (!profiles[k].table[mu]) {
                    set_error("TABLE profile without table for direction %d", mu);
                    return DP_ERR_INVALID_ARG;
                }
                groups[k].table[mu].assign(profiles[k].table[mu], profiles[k].table[mu] + L[mu]);
            }
        }
    }
    fp->users++;
    double *cpp_dev = cpp_out;
    void *tmp = nullptr, *tmp_ap = nullptr;
    if (!cpp_on_device) {
        tmp = c.alloc(sizeof(double) * n_mass * fp->g.T);
        cpp_dev = (double *)tmp;
    }
    if (cap_out) tmp_ap = c.alloc(sizeof(double) * n_mass * fp->g.T);
    void *tmp_hl = hl_out ? c.alloc(sizeof(double) * 2 * fp->g.T) : nullptr;
    std::vector<SolveResult> res;
    if (!cpp_dev || (cap_out && !tmp_ap) || (hl_out && !tmp_hl)) {
        fp->users--;
        c.release(tmp);
        c.release(tmp_ap);
        c.release(tmp_hl);
        set_error("out of device memory");
        return DP_ERR_OOM;
    }
    s = solve_groups(&c, fp, groups, r, o, cpp_dev, prop_out, res, (double *)tmp_ap, (double *)tmp_hl);
    if (s == DP_OK || s == DP_ERR_NOT_CONVERGED || s == DP_ERR_BREAKDOWN) {
        if (!cpp_on_device)
            cudaMemcpyAsync(cpp_out, cpp_dev, sizeof(double) * n_mass * fp->g.T, cudaMemcpyDeviceToHost, c.stream);
        if (cap_out)
            cudaMemcpyAsync(cap_out, tmp_ap, sizeof(double) * n_mass * fp->g.T, cudaMemcpyDeviceToHost, c.stream);
        if (hl_out)
            cudaMemcpyAsync(hl_out, tmp_hl, sizeof(double) * 2 * fp->g.T, cudaMemcpyDeviceToHost, c.stream);
    }
    cudaStreamSynchronize(c.stream);
    if (tmp) c.release(tmp);
    if (tmp_ap) c.release(tmp_ap);
    if (tmp_hl) c.release(tmp_hl);
    fp->users--;
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info)
        for (int k = 0; k < n_mass; k++) {
            info[k] = dp_solve_info{};
            if (k < (int)res.size()) {
                info[k].iters_inner = res[k].iters_inner;
                info[k].iters_outer = res[k].iters_outer;
                info[k].true_rel_residue = res[k].true_rel_residue;
                info[k].status = res[k].status;
                info[k].slice_residue = res[k].slice_residue;
                info[k].refine_rounds = res[k].refine_rounds;
            } else {
                info[k].status = s;
            }
            info[k].seconds = secs;
            info[k].n_rhs = 12;
        }
    return s;
}

extern "C" {

dp_status dp_solve_point(dp_ctx *ctx, dp_field field, double M, const dp_profile *profile,
                         const int src[4], double r, const dp_solve_opts *opts, double *cpp_out,
                         double *prop_out, dp_solve_info *info)
{
    dp_profile none{};
    none.kind = DP_PROF_NONE;
    return solve_common(ctx, field, 1, &M, profile ? profile : &none, src, r, opts, cpp_out, 0,
                        prop_out, info);
}

dp_status dp_solve_point_multi(dp_ctx *ctx, dp_field field, int n_mass, const double *M,
                               const dp_profile *profiles, const int src[4], double r,
                               const dp_solve_opts *opts, double *cpp_out, double *prop_out,
                               dp_solve_info *info)
{
    return solve_common(ctx, field, n_mass, M, profiles, src, r, opts, cpp_out, 0, prop_out, info);
}

dp_status dp_solve_point_corr(dp_ctx *ctx, dp_field field, double M, const dp_profile *profile,
                              const int src[4], double r, const dp_solve_opts *opts, double *cpp_out,
                              double *cap_out, dp_solve_info *info)
{
    if (!cap_out) {
        set_error("dp_solve_point_corr: cap_out is NULL");
        return DP_ERR_INVALID_ARG;
    }
    dp_profile none{};
    none.kind = DP_PROF_NONE;
    return solve_common(ctx, field, 1, &M, profile ? profile : &none, src, r, opts, cpp_out, 0,
                        nullptr, info, cap_out);
}

dp_status dp_solve_point_hl(dp_ctx *ctx, dp_field field, double M_h, const dp_profile *profile_h,
                            double M_l, const dp_profile *profile_l, const int src[4], double r,
                            const dp_solve_opts *opts, double *cpp_out, double *hl_out,
                            dp_solve_info *info)
{
    if (!hl_out || !cpp_out) {
        set_error("dp_solve_point_hl: NULL output");
        return DP_ERR_INVALID_ARG;
    }
    dp_solve_opts o{};
    if (opts) o = *opts;
    o.batched = 1;  // both masses in one batch: the contraction reads both propagators
    const double M[2] = {M_h, M_l};
    dp_profile none{};
    none.kind = DP_PROF_NONE;
    const dp_profile prof[2] = {profile_h ? *profile_h : none, profile_l ? *profile_l : none};
    return solve_common(ctx, field, 2, M, prof, src, r, &o, cpp_out, 0, nullptr, info, nullptr,
                        hl_out);
}

dp_status dp_solve_point_dev(dp_ctx *ctx, dp_field field, int n_mass, const double *M,
                             const dp_profile *profiles, const int src[4], double r,
                             const dp_solve_opts *opts, double *cpp_out_dev, dp_solve_info *info)
{
    return solve_common(ctx, field, n_mass, M, profiles, src, r, opts, cpp_out_dev, 1, nullptr, info);
}

dp_status dp_schur_dev(dp_ctx *ctx, dp_field field, double M, const dp_profile *profile,
                       const int src[4], int prec, int compress12, int parity, int dagger,
                       const void *in, void *out, int nrhs)
{
    if (!ctx) {
        set_error("null context");
        return DP_ERR_INVALID_ARG;
    }
    Ctx &c = ctx->c;
    if (cudaSetDevice(c.device) != cudaSuccess) {
        set_error("cudaSetDevice failed");
        return DP_ERR_CUDA;
    }
    auto fp = find_field(&c, field);
    if (!fp) {
        set_error("unknown field");
        return DP_ERR_NOT_FOUND;
    }
    Field &f = *fp;
    const int pr = prec == DP_PREC_FP64 ? 0 : 1;
    if (!in || !out || in == out || nrhs < 1 || nrhs > kMaxRhs || (parity & ~1) ||
        (dagger != 0 && dagger != 1) || prec < DP_PREC_FP64 || prec > DP_PREC_MIXED_BF16 ||
        (pr == 1 && nrhs % 2) || !std::isfinite(M)) {
        set_error("dp_schur_dev: invalid argument");
        return DP_ERR_INVALID_ARG;
    }
    if (!f.has_clover) {
        set_error("clover term not built");
        return DP_ERR_INVALID_ARG;
    }
    const Geom &g = f.g;
    const int zero_src[4] = {0, 0, 0, 0};
    dp_profile none{};
    none.kind = DP_PROF_NONE;
    std::vector<double> alpha(4 * g.Lmax), hop(8 * g.Lmax), hopa(8 * g.Lmax);
    dp_status s = profile_tables(profile ? *profile : none, g, f.bc_t, src ? src : zero_src,
                                 alpha.data(), hop.data());
    if (s != DP_OK) return s;
    for (size_t k = 0; k < hop.size(); k++) hopa[k] = hop[k] != 0.0 ? 0.25 / hop[k] : 0.0;
    std::vector<float> hopf(hop.begin(), hop.end()), hopaf(hopa.begin(), hopa.end());
    const int lf = inner_link_format(prec, compress12);
    Op op{};
    op.f = &f;
    op.st = c.stream;
    op.pr = pr;
    op.lf = lf;
    op.nrhs = nrhs;
    for (int q = 0; q < 2; q++) {
        s = field_links(&c, f, lf, q, &op.links[q]);
        if (s != DP_OK) return s;
    }
    std::shared_ptr<CloverInv> ci;
    s = get_clover_inv(&c, f, M, &ci);
    if (s != DP_OK) return s;
    for (int q = 0; q < 2; q++) op.inv[q][0] = pr == 0 ? (const void *)ci->inv64[q] : (const void *)ci->inv32[q];
    set_shape(op, c.launch_shape(g.Vh, pr, lf, nrhs));
    if (!dslash_rpt_ok(nrhs, op.rpt, pr, EPI_AINV)) {
        op.rpt = pr == 0 ? 1 : 2;
        op.stages = 0;
    }
    const size_t tb = hop.size() * (pr == 0 ? sizeof(double) : sizeof(float));
    const size_t vb = (size_t)g.Vh * nrhs * 24 * (pr == 0 ? 8 : 4);
    void *hd = c.alloc(tb), *had = c.alloc(tb), *tp = c.alloc(vb), *tq = c.alloc(vb);
    auto run = [&]() -> dp_status {
        if (!hd || !had || !tp || !tq) {
            set_error("out of device memory (dp_schur_dev)");
            return DP_ERR_OOM;
        }
        CK(cudaMemcpyAsync(hd, pr == 0 ? (const void *)hop.data() : (const void *)hopf.data(), tb,
                           cudaMemcpyHostToDevice, c.stream));
        CK(cudaMemcpyAsync(had, pr == 0 ? (const void *)hopa.data() : (const void *)hopaf.data(), tb,
                           cudaMemcpyHostToDevice, c.stream));
        op.hop = hd;
        Op adj = op;
        adj.hop = had;
        dp_status e = dagger ? apply_mhat_dag(&c, op, adj, parity, in, out, tp, tq, nullptr)
                             : apply_mhat(&c, op, parity, in, out, tq, nullptr);
        if (e != DP_OK) return e;
        CK(cudaStreamSynchronize(c.stream));
        return DP_OK;
    };
    s = run();
    c.release(hd);
    c.release(had);
    c.release(tp);
    c.release(tq);
    return s;
}

}  // extern "C"
