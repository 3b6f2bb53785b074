// Request scheduler: continuous batching of point-source solves over the
// gauge fields resident in a context.
//
// One solver batch (see solver.cu) per field with queued or running work,
// each on a CUDA stream of its own and driven by a worker thread of its own,
// so the rounds of different fields (different lattice volumes) run
// concurrently on the device.  Between defect-correction rounds a worker
// completes the jobs whose RHS have all converged (and met their per-slice
// accuracy target), frees their slots, and admits its field's queued
// requests into free slots, so requests that arrive while others are on the
// GPU join the running batch.  A coordinator thread creates a field's batch
// when its device memory fits the HBM budget and retires idle batches when
// other fields wait for memory; a request that can never fit is rejected at
// submit time.  Latency is measured from submit to completion on the host
// clock.
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

struct Scheduler;

// one field's batch and the thread that runs its rounds
struct Worker {
    uint64_t fid = 0;
    std::shared_ptr<Field> field;
    std::unique_ptr<Batch> B;
    std::thread th;
    size_t bytes = 0;
    bool stop = false;     // set by the coordinator (under Scheduler::mu)
    bool finished = false; // the thread has left its loop
    int running = 0;       // jobs in the batch (under Scheduler::mu)
};

struct Scheduler {
    Ctx *c;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<dp_ticket, std::shared_ptr<Request>> all;
    std::map<uint64_t, std::unique_ptr<Worker>> workers;  // by field id
    bool stop = false, drain = true;
    size_t budget = 0, in_use = 0;
    int max_slots = 48;
    dp_ticket next = 1;
    long submitted = 0, completed = 0, rejected = 0;
    std::vector<double> lat_ms;
    Clock::time_point first_done, last_done;
    int in_round = 0, max_in_round = 0;  // batches inside a round at once
    long yields = 0;                     // inner solves cut short to admit a request

    // a running batch's convergence-check hook: true (the inner solve yields)
    // when a request of its field waits and the batch has free slots
    void install_yield(Worker *w);
    dp_solve_opts opts{};

    void run();            // coordinator
    void work(Worker *w);  // a field's batch
    // (under mu) a request ends with a status
    void finish(Request *rq, dp_status s, const char *why);
};

void SchedDeleter::operator()(Scheduler *s) const { delete s; }

void Scheduler::install_yield(Worker *w)
{
    w->B->set_yield([this, w] {
        std::lock_guard<std::mutex> lk(mu);
        if (!w->B->can_admit(12)) return false;
        for (auto &rq : queue)
            if (!rq->cancelled && rq->req.field == w->fid) {
                yields++;
                return true;
            }
        return false;
    });
}

void Scheduler::finish(Request *rq, dp_status s, const char *why)
{
    rq->status = s;
    if (s != DP_OK) rq->err = why;
    rq->done = true;
    rq->t_done = Clock::now();
    rq->field->users--;
}

void Scheduler::work(Worker *w)
{
    cudaSetDevice(c->device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        Batch &B = *w->B;  // (replaced after a failing round)
        // admit this field's queued requests into free slots (FIFO)
        for (auto it = queue.begin(); it != queue.end();) {
            auto rq = *it;
            if (rq->cancelled) {
                it = queue.erase(it);
                continue;
            }
            if (rq->req.field != w->fid) {
                ++it;
                continue;
            }
            if (!B.can_admit(12)) break;
            queue.erase(it);
            rq->admitted = true;
            lk.unlock();
            dp_status s = B.admit(&rq->job);
            std::string msg = s != DP_OK ? dp_last_error() : "";
            lk.lock();
            // the queue may have changed while unlocked (submits, other
            // fields' workers): its iterators are stale, scan it afresh
            it = queue.begin();
            if (s != DP_OK) {
                finish(rq.get(), s, msg.c_str());
                done_cv.notify_all();
                continue;
            }
            w->running++;
        }
        if (B.active_jobs() == 0) {
            if (w->stop) break;
            cv.wait_for(lk, std::chrono::milliseconds(20));
            continue;
        }
        in_round++;
        max_in_round = std::max(max_in_round, in_round);
        lk.unlock();
        std::vector<Job *> fin;
        dp_status s = B.round();
        if (s == DP_OK) s = B.harvest(fin);
        std::string msg = s != DP_OK ? dp_last_error() : "";
        lk.lock();
        in_round--;
        for (Job *j : fin) {
            Request *rq = static_cast<Request *>(j->user);
            const dp_status st = (dp_status)j->res.status;
            finish(rq, st, st == DP_ERR_NOT_CONVERGED
                               ? "solve did not reach the requested residue or per-slice accuracy"
                               : "solve failed");
            w->running--;
            completed++;
            lat_ms.push_back(std::chrono::duration<double, std::milli>(rq->t_done - rq->t_submit).count());
            if (completed == 1) first_done = rq->t_done;
            last_done = rq->t_done;
        }
        if (s != DP_OK) {
            // a failing batch fails its running jobs and starts afresh
            for (auto &ar : all)
                if (ar.second->admitted && !ar.second->done && ar.second->req.field == w->fid)
                    finish(ar.second.get(), s, msg.c_str());
            w->running = 0;
            lk.unlock();
            w->B.reset(new Batch(c, w->field, max_slots, opts, 200, 0, true));
            dp_status e = w->B->init();
            install_yield(w);
            lk.lock();
            done_cv.notify_all();
            if (e != DP_OK) break;
            continue;
        }
        if (!fin.empty()) done_cv.notify_all();
    }
    w->finished = true;
    cv.notify_all();
}

void Scheduler::run()
{
    cudaSetDevice(c->device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        // a batch for every field with queued requests, as the budget allows
        for (auto &rq : queue) {
            if (rq->cancelled) continue;
            const uint64_t fid = rq->req.field;
            if (workers.count(fid)) continue;
            const size_t need = Batch::bytes_needed(rq->field->g, max_slots, rq->req.prec);
            if (in_use + need > budget) continue;
            auto w = std::make_unique<Worker>();
            w->fid = fid;
            w->field = rq->field;
            w->bytes = need;
            in_use += need;
            Worker *wp = w.get();
            workers.emplace(fid, std::move(w));
            lk.unlock();
            wp->B = std::make_unique<Batch>(c, wp->field, max_slots, opts, 200, 0, true);
            dp_status s = wp->B->init();
            std::string msg = s != DP_OK ? dp_last_error() : "";
            lk.lock();
            if (s != DP_OK) {
                for (auto it = queue.begin(); it != queue.end();) {
                    if ((*it)->req.field == fid) {
                        finish(it->get(), s, msg.c_str());
                        it = queue.erase(it);
                    } else {
                        ++it;
                    }
                }
                lk.unlock();
                wp->B.reset();
                lk.lock();
                in_use -= wp->bytes;
                workers.erase(fid);
                done_cv.notify_all();
                break;  // the queue changed under the loop
            }
            install_yield(wp);
            wp->th = std::thread([this, wp] { work(wp); });
            break;  // the queue iterator may be stale after unlocking
        }
        // retire idle batches when other fields wait for memory
        bool waiting_other = false;
        for (auto &rq : queue)
            if (!rq->cancelled && !workers.count(rq->req.field)) waiting_other = true;
        for (auto &kv : workers) {
            Worker &w = *kv.second;
            bool queued_here = false;
            for (auto &rq : queue)
                if (rq->req.field == kv.first && !rq->cancelled) queued_here = true;
            const bool idle = w.running == 0 && !queued_here;
            if (idle && (waiting_other || stop)) w.stop = true;
        }
        for (auto it = workers.begin(); it != workers.end();) {
            Worker &w = *it->second;
            if (!w.finished) {
                ++it;
                continue;
            }
            lk.unlock();
            if (w.th.joinable()) w.th.join();
            w.B.reset();
            lk.lock();
            in_use -= w.bytes;
            it = workers.erase(it);
        }
        if (stop) {
            if (!drain) {
                for (auto &rq : queue) {
                    if (rq->cancelled) continue;
                    rq->cancelled = true;
                    finish(rq.get(), DP_ERR_REJECTED, "scheduler stopped");
                }
                queue.clear();
                done_cv.notify_all();
            }
            if (queue.empty() && workers.empty()) break;
        }
        cv.wait_for(lk, std::chrono::milliseconds(10));
    }
    done_cv.notify_all();
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
    out->max_concurrent_batches = S.max_in_round;
    out->yields = S.yields;
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
