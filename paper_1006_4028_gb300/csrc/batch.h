// Slot-based solver batch: see solver.cu.
#pragma once

#include <functional>
#include <memory>
#include <vector>

#include "ctx.h"

namespace dp {

// a point-source job: `ncomp` spin-colour components (from comp0) of one
// (mass, profile, source) group
struct Job {
    Group grp;
    int comp0 = 0, ncomp = 12;
    double r = 1e-10;
    double *cpp_dst = nullptr;   // device [T], written (or added to) on completion
    int accumulate = 0;
    double *cpp_host = nullptr;  // host [T], written on completion
    double *cap_dst = nullptr;   // device [T] C_AP, written (or added to) on completion, or NULL
    double *prop_host = nullptr; // host [ncomp][V][12] complex128 or NULL
    // per-slice accuracy target (0: not checked): the restored Schur residual
    // of every time slice relative to that slice's solution, see slices.cu
    double slice_tol = 0;
    SolveResult res;
    bool done = false;
    // per-slice check state (set by the batch)
    bool slice_ok = false, refining = false;
    int refine_rounds = 0, slice_stall = 0;
    double slice_best = 0, slice_res = 0;
    // set by the batch
    int tab = -1, slot0 = -1;
    double src_scale = 1.0;
    void *user = nullptr;
};

struct Op {
    const Field *f = nullptr;
    cudaStream_t st = nullptr;  // the stream its launches go to
    int pr = 0;  // 0 FP64, 1 FP32
    int lf = 0;  // link format
    const void *links[2] = {nullptr, nullptr};  // per parity, in format lf
    const void *hop = nullptr;
    const void *inv[2][kMaxGroups] = {};
    int8_t grp_of[kMaxRhs] = {};
    int nrhs = 0;
    int block = 128;
    int rpt = 1;     // RHS per thread of the Schur launches
    int stages = 0;  // shared-memory staging of the Schur launches (0: direct)
};

struct InnerVecs {
    void *r = nullptr, *rh = nullptr, *p = nullptr, *v = nullptr, *s = nullptr, *t = nullptr,
         *x = nullptr, *to = nullptr;
    // FP32 BiCGStab: rhat' = Mhat^dag rhat and the per-site omega sums
    void *rh2 = nullptr, *dots = nullptr;
};

class Batch {
  public:
    // schur_parity: the parity p whose Schur system is solved; a job whose
    // source sits on parity p needs no dslash to set up its right-hand side
    // own_stream: the batch runs on a stream of its own with its own reduction
    // scratch (the scheduler runs one batch per field concurrently); else on
    // the context stream with the context's scratch
    Batch(Ctx *c, std::shared_ptr<Field> f, int nslots, const dp_solve_opts &o, int round_cap,
          int schur_parity = 0, bool own_stream = false);
    ~Batch();
    Batch(const Batch &) = delete;
    Batch &operator=(const Batch &) = delete;

    static size_t bytes_needed(const Geom &g, int nslots, int prec);
    dp_status init();
    bool can_admit(int ncomp) const;
    // set up the job's source, Schur right-hand side and outer state
    dp_status admit(Job *j);
    // one FP64 defect-correction round for every active RHS
    dp_status round();
    // finish jobs whose RHS are all done: odd sites, residual, restore, C_PP
    dp_status harvest(std::vector<Job *> &finished);
    // after harvest: heavy-light correlator of two finished jobs of this
    // batch (both parities of their solutions stay in place until the next
    // admission): out_dev [T][2] (re, im)
    dp_status contract_hl(const Job &h, const Job &l, double *out_dev);
    int active_jobs() const;
    // at most this many jobs at once (0: as many as the slots hold)
    void set_max_jobs(int m) { max_jobs = m; }
    // called at the inner solver's convergence checks (after at least
    // min_iter iterations of the round's inner solve): returning true ends
    // the inner solve there, so the round closes early (the partial
    // correction is a valid defect-correction step) and a waiting request can
    // be admitted at once
    void set_yield(std::function<bool()> fn, int min_iter = 8)
    {
        yield_check = std::move(fn);
        yield_min = min_iter;
    }
    size_t bytes() const { return total_bytes; }
    const std::shared_ptr<Field> &field() const { return f; }

  private:
    void *get(size_t bytes);
    dp_status upload_mask(const std::vector<int> &m);
    // per-slice residuals of the jobs that finished globally or are refining;
    // starts, continues or ends their refinement (updates hs; sets *changed)
    dp_status slice_check(bool *changed);
    // inner solver's profile of a job: a time table that flattens the
    // restored per-slice norms of its current solution; h[2t] = |x_t|^2,
    // h[2t + 1] = |r_t|^2 (absolute t)
    dp_status set_inner_profile(const Job &j, const double *h);
    dp_status bicgstab(int max_iter, int *iters_done);
    dp_status cgne(int max_iter, int *iters_done);
    dp_status sap_gcr(int max_iter, int *iters_done);
    // z = SAP(r): the Schwarz alternating procedure as a preconditioner
    dp_status sap(const void *r, void *z);
    // y64 = Mhat x, t64 = A_qq^-1 D_qp x for the active outer RHS (FP64 or
    // double-float)
    dp_status outer_mhat();

    Ctx *c;
    std::shared_ptr<Field> f;
    bool own_stream_ = false;
    cudaStream_t st_ = nullptr;
    BlasCtx bc_{};
    int *hnact_ = nullptr;  // pinned
    int n;
    dp_solve_opts opts;
    int round_iters;
    int sp = 0;
    int max_jobs = 0;
    std::function<bool()> yield_check;
    int yield_min = 8;
    int mixed = 1, ipr = 1, ilf = LINK_F32_12;
    int check_every = 4;
    size_t v64 = 0, vin = 0, total_bytes = 0;
    std::vector<void *> owned;
    double2 *bh = nullptr, *x = nullptr, *r64 = nullptr, *y64 = nullptr, *to64 = nullptr,
            *t64 = nullptr;
    float4 *xdf = nullptr, *tdf = nullptr;  // double-float outer operator (opts.outer_df)
    static constexpr int kMaxNkv = 32;
    void *zk[kMaxNkv] = {}, *wk[kMaxNkv] = {};  // SAP+GCR directions and their images
    double2 *coef_d = nullptr;
    double *nrm2_d = nullptr;
    int sap_bs[4] = {0, 0, 0, 0}, sap_nb[4] = {0, 0, 0, 0};
    float2 *hopdf_d = nullptr;
    InnerVecs in;
    RhsState *outer = nullptr, *inner = nullptr;
    double *alpha_d = nullptr, *hop64_d = nullptr, *hopadj64_d = nullptr;
    // the inner solver's profile per group (equal to alpha_d until a job is
    // refined) and, for the FP64 inner solver, its own hop tables
    double *alpha_in_d = nullptr, *hopin64_d = nullptr;
    double *slice_d = nullptr;  // [kMaxGroups][T][2] per-slice norms
    std::vector<double> slice_h;
    bool any_refining() const;
    float *hop32_d = nullptr, *hopadj32_d = nullptr;  // adj: the reciprocal profile (CGNE)
    SlotInfo *slots_d = nullptr;
    int *tsrc_d = nullptr, *mask_d = nullptr;
    double *cpp_d = nullptr, *cap_d = nullptr, *cpart = nullptr, *nrm_d = nullptr;
    Op op64, opin, opin_adj, opdf;
    cudaGraphExec_t graph = nullptr;
    int graph_max_iter = 0;
    Job *jobs[kMaxGroups] = {};
    std::shared_ptr<CloverInv> invs[kMaxGroups];
    std::vector<Job *> slot_job;
    std::vector<int> slot_inner, slot_outer, slot_stall;
    std::vector<double> slot_rr_prev;
    std::vector<SlotInfo> slots;
    std::vector<RhsState> hs, hin;
};

}  // namespace dp
