// Continuous-batching serve loop behind hot_submit / hot_poll.
//
// A background thread owns one stream and one Batch (the same graph-captured
// check block as the synchronous solver).  Between blocks it
//   * admits queued requests while batch slots and the device-memory budget
//     allow (admission is at block boundaries, so every instance's checks fall
//     on its own iterations 10, 20, ... exactly as when it runs alone);
//   * retires instances whose last check ended them (converged, capped,
//     numeric failure or cancelled), returning their memory.
// Instances never interact on the device: every reduction is per instance, so
// a request's result is bit-identical alone and in any mix.
#include <algorithm>
#include <chrono>
#include <cstring>

#include "hot_engine.h"

namespace hot {

using Clock = std::chrono::steady_clock;

struct Req {
    unsigned long long ticket = 0;
    PairHost pair;
    double tol = 1e-6;
    long long max_iter = 0;
    int keep = 0;
    int state = 0;                // 0 queued, 1 running, 2 done
    int status = HOT_PENDING;
    bool cancel = false;
    bool cancel_sent = false;
    hot_result res{};
    Inst* inst = nullptr;
    size_t bytes = 0;
    Clock::time_point t_submit, t_admit, t_done;
};

struct ServeState {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req*> queue;
    std::map<unsigned long long, std::unique_ptr<Req>> reqs;
    std::vector<Req*> active;
    std::thread th;
    bool stop = false;
    bool started = false;
    cudaStream_t st = nullptr;
    std::unique_ptr<Batch> batch;
    size_t budget = 0, in_use = 0;
    unsigned long long next_ticket = 1;
    long long submitted = 0, completed = 0, cancelled = 0, rejected = 0, blocks = 0;
    std::vector<double> lat_ms, queue_ms;
};

static int serve_tile_rows(Ctx* ctx, int m, int n, int fp64) {
    const int t = tuned_tile_rows(ctx, m, n, fp64);
    return t ? t : tile_rows(m, n, fp64, sweep_grid(fp64));
}

// Device bytes of one instance (an upper bound of inst_create's layout).
static size_t inst_bytes_estimate(Ctx* ctx, int m, int n, int fp64) {
    const size_t MN = (size_t)m * n;
    const size_t V = MN * (size_t)(m + n);
    const size_t big = 5 * (V * (fp64 ? 8 : 4) + 256);
    const int tr = serve_tile_rows(ctx, m, n, fp64);
    const size_t CP = (size_t)n * ((m + tr - 1) / tr) * m + (size_t)m * ((n + tr - 1) / tr) * n;
    // pieces 3 x 32 MN, slab-row sums 5 x 16 MN, marginals 16 MN, column partials 28 CP
    size_t small = MN * (96 + 80 + 16) + CP * 28 + 1024 * 64;
    if (!fp64) small += MN * 192;       // double-float arrays of FP32 mode
    return big + small;
}

static void finish_req(Ctx* ctx, ServeState* s, Req* r, int status) {
    r->state = 2;
    r->status = status;
    r->t_done = Clock::now();
    r->res.status = status;
    r->res.queue_ms = std::chrono::duration<double, std::milli>(r->t_admit - r->t_submit).count();
    if (r->inst) {
        r->res.solve_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_admit).count();
        if (r->keep) {
            std::lock_guard<std::mutex> g(ctx->mu);
            const unsigned long long id = ctx->next_id++;
            ctx->solutions[id].inst = r->inst;
            r->res.solution_id = id;
        } else {
            inst_destroy(r->inst, s->st);
        }
        s->in_use -= std::min(s->in_use, r->bytes);
        r->inst = nullptr;
    }
    if (status == HOT_ECANCELLED) {
        ++s->cancelled;                 // latency statistics cover served requests only
        return;
    }
    ++s->completed;
    s->lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
    s->queue_ms.push_back(r->res.queue_ms);
}

static void serve_loop(Ctx* ctx) {
    ServeState* s = ctx->serve.get();
    cudaSetDevice(ctx->device);
    const int fp64 = ctx->cfg.precision == HOT_FP64 ? 1 : 0;
    const int max_batch = ctx->cfg.max_batch > 0 ? ctx->cfg.max_batch : 1024;
    bool changed = false;
    for (;;) {
        std::vector<Req*> admit;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop) break;
            while (!s->queue.empty() && (int)(s->active.size() + admit.size()) < max_batch) {
                Req* r = s->queue.front();
                if (r->cancel) {
                    s->queue.pop_front();
                    r->t_admit = Clock::now();
                    finish_req(ctx, s, r, HOT_ECANCELLED);
                    continue;
                }
                const size_t need = inst_bytes_estimate(ctx, r->pair.m, r->pair.n, fp64);
                if (s->in_use + need > s->budget) {
                    if (s->active.empty() && admit.empty() && s->in_use == 0) {
                        // can never fit
                        s->queue.pop_front();
                        r->t_admit = Clock::now();
                        ++s->rejected;
                        finish_req(ctx, s, r, HOT_ENOMEM);
                        continue;
                    }
                    break;
                }
                s->queue.pop_front();
                r->bytes = need;
                s->in_use += need;
                admit.push_back(r);
            }
            if (admit.empty() && s->active.empty()) {
                s->cv_done.notify_all();
                s->cv_work.wait_for(lk, std::chrono::milliseconds(20));
                continue;
            }
        }
        for (Req* r : admit) {
            Inst* I = nullptr;
            r->t_admit = Clock::now();
            const int rc = inst_create(r->pair, fp64, ctx->cfg, r->tol, r->max_iter, tuned_tile_rows(ctx, r->pair.m, r->pair.n, fp64), s->st, &I);
            std::lock_guard<std::mutex> g(s->mu);
            if (rc != HOT_OK) {
                s->in_use -= std::min(s->in_use, r->bytes);
                r->bytes = 0;
                finish_req(ctx, s, r, rc);
                continue;
            }
            r->inst = I;
            r->state = 1;
            s->active.push_back(r);
            changed = true;
        }
        if (s->active.empty()) continue;
        std::vector<Inst*> insts;
        {
            std::lock_guard<std::mutex> g(s->mu);
            for (Req* r : s->active) insts.push_back(r->inst);
            // forward cancellations of running requests to their control blocks
            for (Req* r : s->active)
                if (r->cancel && !r->cancel_sent) {
                    static const int one = 1;
                    cudaMemcpyAsync(&r->inst->desc.ctl->cancel, &one, sizeof(int), cudaMemcpyHostToDevice, s->st);
                    r->cancel_sent = true;
                }
        }
        if (changed) {
            if (s->batch->set_instances(insts, s->st) != HOT_OK || s->batch->ensure_graph() != HOT_OK) {
                std::lock_guard<std::mutex> g(s->mu);
                for (Req* r : s->active) finish_req(ctx, s, r, HOT_ECUDA);
                s->active.clear();
                s->cv_done.notify_all();
                continue;
            }
            changed = false;
        }
        // two blocks back to back, then look at the statuses
        s->batch->launch_block(s->st);
        s->batch->launch_block(s->st);
        const int n = (int)insts.size();
        cudaMemcpyAsync(s->batch->h_st, s->batch->d_st, sizeof(int) * n, cudaMemcpyDeviceToHost, s->st);
        const cudaError_t e = cudaStreamSynchronize(s->st);
        std::lock_guard<std::mutex> g(s->mu);
        s->blocks += 2;
        std::vector<Req*> still;
        for (int i = 0; i < n; ++i) {
            Req* r = s->active[i];
            if (e != cudaSuccess) {
                finish_req(ctx, s, r, HOT_ECUDA);
                changed = true;
                continue;
            }
            if (s->batch->h_st[i] != ST_RUNNING) {
                cudaMemcpy(&r->inst->ctl_host, r->inst->desc.ctl, sizeof(HotCtl), cudaMemcpyDeviceToHost);
                fill_result(r->inst, &r->res);
                finish_req(ctx, s, r, r->res.status);
                changed = true;
            } else {
                still.push_back(r);
            }
        }
        s->active.swap(still);
        s->cv_done.notify_all();
    }
    // shutdown: release whatever is left
    std::lock_guard<std::mutex> g(s->mu);
    cudaStreamSynchronize(s->st);
    for (Req* r : s->active) {
        r->t_admit = Clock::now();
        finish_req(ctx, s, r, HOT_ECANCELLED);
    }
    s->active.clear();
    while (!s->queue.empty()) {
        Req* r = s->queue.front();
        s->queue.pop_front();
        r->t_admit = Clock::now();
        finish_req(ctx, s, r, HOT_ECANCELLED);
    }
    s->cv_done.notify_all();
}

static int serve_start(Ctx* ctx) {
    if (ctx->serve && ctx->serve->started) return HOT_OK;
    if (!ctx->serve) ctx->serve.reset(new ServeState());
    ServeState* s = ctx->serve.get();
    HOT_CK(cudaSetDevice(ctx->device));
    HOT_CK(cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking));
    s->batch.reset(new Batch());
    s->batch->device = ctx->device;
    s->batch->fp64 = ctx->cfg.precision == HOT_FP64 ? 1 : 0;
    s->batch->K = ctx->cfg.check_every;
    s->batch->a1 = ctx->cfg.restart_sufficient;
    s->batch->a2 = ctx->cfg.restart_necessary;
    s->batch->a3 = ctx->cfg.restart_long;
    size_t fr = 0, tot = 0;
    HOT_CK(cudaMemGetInfo(&fr, &tot));
    s->budget = ctx->cfg.mem_budget ? ctx->cfg.mem_budget : (size_t)(0.8 * (double)fr);
    s->started = true;
    s->th = std::thread(serve_loop, ctx);
    return HOT_OK;
}

void serve_shutdown(Ctx* ctx) {
    if (!ctx->serve) return;
    ServeState* s = ctx->serve.get();
    if (s->started) {
        {
            std::lock_guard<std::mutex> g(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        if (s->th.joinable()) s->th.join();
        s->batch.reset();
        if (s->st) cudaStreamDestroy(s->st);
        s->st = nullptr;
        s->started = false;
    }
    for (auto& kv : s->reqs)
        if (kv.second->inst) inst_destroy(kv.second->inst, ctx->stream);
    s->reqs.clear();
}

int serve_submit(Ctx* ctx, const hot_request* req, unsigned long long* ticket) {
    if (!req || !ticket) {
        set_error("null request or ticket pointer");
        return HOT_EINVAL;
    }
    if (req->tol < 0.0 || req->max_iter <= 0) {
        set_error("tol must be >= 0 and max_iter > 0");
        return HOT_EINVAL;
    }
    std::unique_ptr<Req> r(new Req());
    const int fp64 = ctx->cfg.precision == HOT_FP64 ? 1 : 0;
    int rc = validate_pair(req->mu, req->nu, req->m, req->n, HOT_SPACE_HOST, fp64, r->pair);
    if (rc != HOT_OK) return rc;
    rc = serve_start(ctx);
    if (rc != HOT_OK) return rc;
    ServeState* s = ctx->serve.get();
    r->tol = req->tol;
    r->max_iter = req->max_iter;
    r->keep = req->keep_solution;
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> g(s->mu);
    const int max_queue = ctx->cfg.max_queue > 0 ? ctx->cfg.max_queue : 65536;
    if ((int)s->queue.size() >= max_queue) {
        set_error("serve queue is full");
        return HOT_EBUSY;
    }
    r->ticket = s->next_ticket++;
    *ticket = r->ticket;
    s->queue.push_back(r.get());
    s->reqs[r->ticket] = std::move(r);
    ++s->submitted;
    s->cv_work.notify_all();
    return HOT_OK;
}

int serve_poll(Ctx* ctx, unsigned long long ticket, double timeout_ms, hot_result* out) {
    if (!ctx->serve) {
        set_error("unknown ticket");
        return HOT_ENOTFOUND;
    }
    ServeState* s = ctx->serve.get();
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        set_error("unknown ticket");
        return HOT_ENOTFOUND;
    }
    Req* r = it->second.get();
    if (r->state != 2 && timeout_ms != 0.0) {
        auto pred = [&] { return r->state == 2; };
        if (timeout_ms < 0) s->cv_done.wait(lk, pred);
        else s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), pred);
    }
    if (r->state != 2) return timeout_ms != 0.0 ? HOT_TIMEOUT : HOT_PENDING;
    if (out) *out = r->res;
    return r->status;
}

int serve_cancel(Ctx* ctx, unsigned long long ticket) {
    if (!ctx->serve) return HOT_ENOTFOUND;
    ServeState* s = ctx->serve.get();
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end() || it->second->state == 2) {
        set_error("unknown or finished ticket");
        return HOT_ENOTFOUND;
    }
    Req* r = it->second.get();
    r->cancel = true;
    if (r->state == 0) {
        // still queued: leave the queue now (an admitted request stops at its next check)
        for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
            if (*q == r) {
                s->queue.erase(q);
                r->t_admit = Clock::now();
                finish_req(ctx, s, r, HOT_ECANCELLED);
                s->cv_done.notify_all();
                break;
            }
    }
    s->cv_work.notify_all();
    return HOT_OK;
}

int serve_forget(Ctx* ctx, unsigned long long ticket) {
    if (!ctx->serve) return HOT_ENOTFOUND;
    ServeState* s = ctx->serve.get();
    unsigned long long sol = 0;
    {
        std::lock_guard<std::mutex> g(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end() || it->second->state != 2) {
            set_error("unknown or unfinished ticket");
            return HOT_ENOTFOUND;
        }
        sol = it->second->res.solution_id;
        s->reqs.erase(it);
    }
    if (sol) {
        std::lock_guard<std::mutex> g(ctx->mu);
        auto it = ctx->solutions.find(sol);
        if (it != ctx->solutions.end()) {
            cudaStreamSynchronize(ctx->stream);
            inst_destroy(it->second.inst, ctx->stream);
            ctx->solutions.erase(it);
        }
    }
    return HOT_OK;
}

static double pct(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (v.size() - 1);
    const size_t lo = (size_t)pos;
    const size_t hi = std::min(v.size() - 1, lo + 1);
    return v[lo] + (v[hi] - v[lo]) * (pos - lo);
}

int serve_stats(Ctx* ctx, hot_serve_stats* out) {
    if (!out) return HOT_EINVAL;
    std::memset(out, 0, sizeof(*out));
    if (!ctx->serve) return HOT_OK;
    ServeState* s = ctx->serve.get();
    std::lock_guard<std::mutex> g(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->cancelled = s->cancelled;
    out->rejected = s->rejected;
    out->queued = (int)s->queue.size();
    out->running = (int)s->active.size();
    out->device_bytes_in_use = s->in_use;
    out->p50_ms = pct(s->lat_ms, 0.50);
    out->p99_ms = pct(s->lat_ms, 0.99);
    double m = 0.0;
    for (double q : s->queue_ms) m += q;
    out->mean_queue_ms = s->queue_ms.empty() ? 0.0 : m / s->queue_ms.size();
    out->blocks_run = s->blocks;
    return HOT_OK;
}

Ctx::Ctx() = default;

Ctx::~Ctx() {
    serve_shutdown(this);
    if (stream) cudaStreamSynchronize(stream);
    for (auto& kv : solutions) inst_destroy(kv.second.inst, stream);
    solutions.clear();
    batch.reset();
    if (stream) cudaStreamSynchronize(stream);
    if (own_stream && stream) cudaStreamDestroy(stream);
}

}  // namespace hot
