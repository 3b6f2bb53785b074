// Request scheduler: continuous batching of point-source solves over the
// gauge fields resident in a context.
//
// A scheduler thread keeps one solver batch (see solver.cu) per field with
// queued or running work.  Between defect-correction rounds it completes the
// jobs whose RHS have all converged, frees their slots, and admits queued
// requests into free slots, so requests that arrive while others are on the
// GPU join the running batch.  A batch's device memory is counted against
// the HBM budget; a request whose field has no batch waits until a new batch
// fits the budget, and one that can never fit is rejected at submit time.
// Latency is measured from submit to completion on the host clock.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "batch.h"

namespace dp {

using Clock = std::chrono::steady_clock;

struct Request {
    dp_ticket id;
    dp_request req;
    Group grp;
    Job job;
    std::vector<double> cpp;
    Clock::time_point t_submit, t_done;
    bool admitted = false, done = false, cancelled = false;
    dp_status status = DP_OK;
    std::string err;  // message of a failed request (set on the scheduler thread)
    std::shared_ptr<Field> field;
};

struct Scheduler {
    Ctx *c;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<dp_ticket, std::shared_ptr<Request>> all;
    std::map<uint64_t, std::unique_ptr<Batch>> batches;  // by field id
    std::map<uint64_t, uint64_t> field_of_batch;
    bool stop = false, drain = true;
    size_t budget = 0, in_use = 0;
    int max_slots = 48;
    dp_ticket next = 1;
    long submitted = 0, completed = 0, rejected = 0;
    std::vector<double> lat_ms;
    Clock::time_point first_done, last_done;
    dp_solve_opts opts{};

    void run();
};

void SchedDeleter::operator()(Scheduler *s) const { delete s; }

void Scheduler::run()
{
    cudaSetDevice(c->device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        // admit queued requests into batches (FIFO per field)
        for (auto it = queue.begin(); it != queue.end();) {
            auto rq = *it;
            if (rq->cancelled) {
                it = queue.erase(it);
                continue;
            }
            const uint64_t fid = rq->req.field;
            auto bit = batches.find(fid);
            if (bit == batches.end()) {
                const size_t need = Batch::bytes_needed(rq->field->g, max_slots, rq->req.prec);
                if (in_use + need > budget) {
                    ++it;
                    continue;
                }
                auto b = std::make_unique<Batch>(c, rq->field, max_slots, opts, 200);
                lk.unlock();
                dp_status s = b->init();
                lk.lock();
                if (s != DP_OK) {
                    rq->status = s;
                    rq->err = dp_last_error();
                    rq->done = true;
                    rq->t_done = Clock::now();
                    rq->field->users--;
                    it = queue.erase(it);
                    done_cv.notify_all();
                    continue;
                }
                in_use += b->bytes();
                bit = batches.emplace(fid, std::move(b)).first;
            }
            Batch &B = *bit->second;
            if (!B.can_admit(12)) {
                ++it;
                continue;
            }
            lk.unlock();
            dp_status s = B.admit(&rq->job);
            lk.lock();
            if (s != DP_OK) {
                rq->status = s;
                rq->err = dp_last_error();
                rq->done = true;
                rq->t_done = Clock::now();
                rq->field->users--;
                it = queue.erase(it);
                done_cv.notify_all();
                continue;
            }
            rq->admitted = true;
            it = queue.erase(it);
        }
        // one round per batch with work, then complete finished jobs
        bool worked = false;
        for (auto &kv : batches) {
            Batch &B = *kv.second;
            if (B.active_jobs() == 0) continue;
            worked = true;
            lk.unlock();
            std::vector<Job *> fin;
            dp_status s = B.round();
            if (s == DP_OK) s = B.harvest(fin);
            lk.lock();
            for (Job *j : fin) {
                Request *rq = static_cast<Request *>(j->user);
                rq->status = (dp_status)j->res.status;
                if (rq->status != DP_OK)
                    rq->err = rq->status == DP_ERR_NOT_CONVERGED ? "solve did not reach the requested residue "
                                                                   "or per-slice accuracy"
                                                                 : "solve failed";
                rq->done = true;
                rq->t_done = Clock::now();
                rq->field->users--;
                completed++;
                lat_ms.push_back(std::chrono::duration<double, std::milli>(rq->t_done - rq->t_submit).count());
                if (completed == 1) first_done = rq->t_done;
                last_done = rq->t_done;
            }
            if (s != DP_OK) {
                // a failing batch fails its running jobs
                for (auto &ar : all)
                    if (ar.second->admitted && !ar.second->done &&
                        ar.second->req.field == kv.first) {
                        ar.second->status = s;
                        ar.second->err = dp_last_error();
                        ar.second->done = true;
                        ar.second->t_done = Clock::now();
                        ar.second->field->users--;
                    }
                kv.second.reset(new Batch(c, kv.second->field(), max_slots, opts, 200));
                lk.unlock();
                kv.second->init();
                lk.lock();
            }
            if (!fin.empty()) done_cv.notify_all();
        }
        // release idle batches when other fields wait for memory
        if (!queue.empty()) {
            for (auto it = batches.begin(); it != batches.end();) {
                bool waiting_here = false;
                for (auto &rq : queue)
                    if (rq->req.field == it->first) waiting_here = true;
                if (it->second->active_jobs() == 0 && !waiting_here) {
                    in_use -= it->second->bytes();
                    lk.unlock();
                    it->second.reset();
                    lk.lock();
                    it = batches.erase(it);
                } else {
                    ++it;
                }
            }
        }
        if (stop && (queue.empty() || !drain)) {
            bool running = false;
            for (auto &kv : batches)
                if (kv.second->active_jobs()) running = true;
            if (!running) break;
        }
        if (!worked) {
            if (stop && queue.empty()) break;
            cv.wait_for(lk, std::chrono::milliseconds(queue.empty() ? 50 : 2));
        }
    }
    // cancel what is left
    for (auto &rq : queue) {
        rq->status = DP_ERR_REJECTED;
        rq->done = true;
        rq->cancelled = true;
        rq->field->users--;
    }
    queue.clear();
    done_cv.notify_all();
    lk.unlock();
    for (auto &kv : batches) kv.second.reset();
    batches.clear();
    in_use = 0;
}

}  // namespace dp

using namespace dp;

extern "C" {

void dp_serve_shutdown(dp_ctx *ctx)
{
    if (!ctx || !ctx->c.sched) return;
    Scheduler &S = *ctx->c.sched;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        S.stop = true;
        S.drain = false;
    }
    S.cv.notify_all();
    if (S.th.joinable()) S.th.join();
    ctx->c.sched.reset();
}

dp_status dp_serve_start(dp_ctx *ctx, size_t hbm_budget, int max_slots)
{
    if (!ctx) {
        set_error("null context");
        return DP_ERR_INVALID_ARG;
    }
    Ctx &c = ctx->c;
    if (c.sched) {
        set_error("scheduler already running");
        return DP_ERR_INVALID_ARG;
    }
    if (max_slots == 0) max_slots = 48;
    if (max_slots < 12 || max_slots > kMaxRhs || max_slots % 12) {
        set_error("max_slots must be a multiple of 12 in [12, %d]", kMaxRhs / 12 * 12);
        return DP_ERR_INVALID_ARG;
    }
    if (cudaSetDevice(c.device) != cudaSuccess) {
        set_error("cudaSetDevice failed");
        return DP_ERR_CUDA;
    }
    if (hbm_budget == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        hbm_budget = (size_t)(0.8 * (double)fr);
    }
    auto S = std::make_unique<Scheduler>();
    S->c = &c;
    S->budget = hbm_budget;
    S->max_slots = max_slots;
    S->opts.prec = DP_PREC_MIXED_FP32;
    S->opts.compress12 = 1;
    S->opts.batched = 1;
    check_opts(&S->opts, &S->opts);
    c.sched.reset(S.release());
    Scheduler *sp = c.sched.get();
    sp->th = std::thread([sp] { sp->run(); });
    return DP_OK;
}

dp_status dp_submit(dp_ctx *ctx, const dp_request *req, dp_ticket *ticket)
{
    if (!ctx || !req || !ticket) {
        set_error("null argument");
        return DP_ERR_INVALID_ARG;
    }
    Ctx &c = ctx->c;
    if (!c.sched) {
        set_error("scheduler not running");
        return DP_ERR_REJECTED;
    }
    Scheduler &S = *c.sched;
    auto f = find_field(&c, req->field);
    if (!f) {
        set_error("unknown field");
        return DP_ERR_NOT_FOUND;
    }
    if (!f->has_clover) {
        set_error("clover term not built for this field");
        return DP_ERR_INVALID_ARG;
    }
    if (req->prec != DP_PREC_MIXED_FP32) {
        set_error("the scheduler serves mixed-precision FP32 requests");
        return DP_ERR_INVALID_ARG;
    }
    if (!std::isfinite(req->M) || !(req->r > 0 && req->r < 1) || !std::isfinite(req->slice_tol)) {
        set_error("invalid mass, residue or slice_tol");
        return DP_ERR_INVALID_ARG;
    }
    const int L[4] = {f->g.T, f->g.Lx, f->g.Ly, f->g.Lz};
    for (int mu = 0; mu < 4; mu++)
        if (req->src[mu] < 0 || req->src[mu] >= L[mu]) {
            set_error("source out of range");
            return DP_ERR_INVALID_ARG;
        }
    const size_t need = Batch::bytes_needed(f->g, S.max_slots, req->prec);
    auto rq = std::make_shared<Request>();
    rq->req = *req;
    rq->field = f;
    rq->grp.M = req->M;
    rq->grp.prof = req->profile;
    for (int mu = 0; mu < 4; mu++) {
        rq->grp.src[mu] = req->src[mu];
        if (req->profile.kind == DP_PROF_TABLE) {
            if (!req->profile.table[mu]) {
                set_error("TABLE profile without table");
                return DP_ERR_INVALID_ARG;
            }
            rq->grp.table[mu].assign(req->profile.table[mu], req->profile.table[mu] + L[mu]);
        }
    }
    rq->cpp.assign(f->g.T, 0.0);
    rq->job.grp = rq->grp;
    rq->job.r = req->r;
    rq->job.slice_tol = slice_target(req->slice_tol, req->r);
    rq->job.cpp_host = rq->cpp.data();
    rq->job.user = rq.get();
    rq->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S.mu);
        if (need > S.budget) {
            S.rejected++;
            set_error("request can never fit the HBM budget (%zu > %zu bytes)", need, S.budget);
            return DP_ERR_REJECTED;
        }
        if (S.stop) {
            set_error("scheduler stopping");
            return DP_ERR_REJECTED;
        }
        rq->id = S.next++;
        S.all[rq->id] = rq;
        S.queue.push_back(rq);
        S.submitted++;
        f->users++;
        *ticket = rq->id;
    }
    S.cv.notify_all();
    return DP_OK;
}

dp_status dp_wait(dp_ctx *ctx, dp_ticket ticket, double timeout_s, double *cpp_out,
                  dp_solve_info *info)
{
    if (!ctx || !ctx->c.sched) {
        set_error("scheduler not running");
        return DP_ERR_INVALID_ARG;
    }
    Scheduler &S = *ctx->c.sched;
    std::unique_lock<std::mutex> lk(S.mu);
    auto it = S.all.find(ticket);
    if (it == S.all.end()) {
        set_error("unknown ticket");
        return DP_ERR_NOT_FOUND;
    }
    auto rq = it->second;
    auto pred = [&] { return rq->done; };
    if (timeout_s < 0)
        S.done_cv.wait(lk, pred);
    else if (!S.done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) {
        set_error("request not finished within %.3f s", timeout_s);
        return DP_ERR_TIMEOUT;
    }
    if (cpp_out) std::copy(rq->cpp.begin(), rq->cpp.end(), cpp_out);
    if (info) {
        *info = dp_solve_info{};
        info->iters_inner = rq->job.res.iters_inner;
        info->iters_outer = rq->job.res.iters_outer;
        info->true_rel_residue = rq->job.res.true_rel_residue;
        info->slice_residue = rq->job.res.slice_residue;
        info->refine_rounds = rq->job.res.refine_rounds;
        info->seconds = std::chrono::duration<double>(rq->t_done - rq->t_submit).count();
        info->n_rhs = 12;
        info->status = rq->status;
    }
    S.all.erase(ticket);
    if (rq->status != DP_OK) set_error("%s", rq->err.empty() ? "request failed" : rq->err.c_str());
    return rq->status;
}

dp_status dp_cancel(dp_ctx *ctx, dp_ticket ticket)
{
    if (!ctx || !ctx->c.sched) {
        set_error("scheduler not running");
        return DP_ERR_INVALID_ARG;
    }
    Scheduler &S = *ctx->c.sched;
    std::lock_guard<std::mutex> lk(S.mu);
    auto it = S.all.find(ticket);
    if (it == S.all.end()) {
        set_error("unknown ticket");
        return DP_ERR_NOT_FOUND;
    }
    auto rq = it->second;
    if (rq->admitted || rq->done) {
        set_error("request already admitted");
        return DP_ERR_INVALID_ARG;
    }
    rq->cancelled = true;
    rq->done = true;
    rq->status = DP_ERR_REJECTED;
    rq->field->users--;
    S.done_cv.notify_all();
    return DP_OK;
}

dp_status dp_serve_stats_get(dp_ctx *ctx, dp_serve_stats *out)
{
    if (!ctx || !ctx->c.sched || !out) {
        set_error("scheduler not running");
        return DP_ERR_INVALID_ARG;
    }
    Scheduler &S = *ctx->c.sched;
    std::lock_guard<std::mutex> lk(S.mu);
    *out = dp_serve_stats{};
    out->submitted = S.submitted;
    out->completed = S.completed;
    out->rejected = S.rejected;
    long inflight = 0;
    for (auto &kv : S.all)
        if (!kv.second->done) inflight++;
    out->in_flight = inflight;
    if (!S.lat_ms.empty()) {
        std::vector<double> v = S.lat_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) {
            const double pos = q * (v.size() - 1);
            const size_t lo = (size_t)std::floor(pos), hi = std::min(v.size() - 1, lo + 1);
            return v[lo] + (pos - lo) * (v[hi] - v[lo]);
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        double s = 0;
        for (double x : v) s += x;
        out->mean_ms = s / v.size();
    }
    if (S.completed > 1) {
        const double span = std::chrono::duration<double>(S.last_done - S.first_done).count();
        if (span > 0) out->solves_per_s = (S.completed - 1) / span;
    }
    out->hbm_budget = S.budget;
    out->hbm_in_use = S.in_use;
    return DP_OK;
}

dp_status dp_serve_stop(dp_ctx *ctx, int drain)
{
    if (!ctx || !ctx->c.sched) {
        set_error("scheduler not running");
        return DP_ERR_INVALID_ARG;
    }
    Scheduler &S = *ctx->c.sched;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        S.stop = true;
        S.drain = drain != 0;
    }
    S.cv.notify_all();
    if (S.th.joinable()) S.th.join();
    ctx->c.sched.reset();
    return DP_OK;
}

}  // extern "C"
