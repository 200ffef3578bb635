// The extern "C" entry points declared in include/hot.h.
#include <cstring>
#include <exception>

#include "hot_engine.h"

namespace hot {
int serve_submit(Ctx* ctx, const hot_request* req, unsigned long long* ticket);
int serve_poll(Ctx* ctx, unsigned long long ticket, double timeout_ms, hot_result* out);
int serve_cancel(Ctx* ctx, unsigned long long ticket);
int serve_forget(Ctx* ctx, unsigned long long ticket);
int serve_stats(Ctx* ctx, hot_serve_stats* out);
}  // namespace hot

struct hot_ctx {
    hot::Ctx impl;
};

using hot::set_error;

#define HOT_GUARD_BEGIN try {
#define HOT_GUARD_END                                                 \
    }                                                                 \
    catch (const std::bad_alloc&) {                                   \
        set_error("host allocation failed");                          \
        return HOT_ENOMEM;                                            \
    }                                                                 \
    catch (const std::exception& ex) {                                \
        set_error(std::string("internal error: ") + ex.what());       \
        return HOT_ECUDA;                                             \
    }                                                                 \
    catch (...) {                                                     \
        set_error("internal error");                                  \
        return HOT_ECUDA;                                             \
    }

extern "C" {

void hot_config_default(hot_config* cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->device = 0;
    cfg->stream = nullptr;
    cfg->precision = HOT_FP32_BULK;
    cfg->check_every = 10;
    cfg->sigma0 = 0.0;
    cfg->restart_sufficient = 0.2;
    cfg->restart_necessary = 0.8;
    cfg->restart_long = 0.2;
    cfg->mem_budget = 0;
    cfg->max_batch = 1024;
    cfg->max_queue = 65536;
    cfg->autotune_cache = nullptr;
    cfg->method = HOT_METHOD_HALPERN;
    cfg->relaxation = 1.7;
    cfg->stop_rule = HOT_STOP_RELATIVE;
}

const char* hot_status_string(int status) {
    switch (status) {
        case HOT_OK: return "HOT_OK";
        case HOT_PENDING: return "HOT_PENDING";
        case HOT_NOT_CONVERGED: return "HOT_NOT_CONVERGED";
        case HOT_EINVAL: return "HOT_EINVAL";
        case HOT_ENOMEM: return "HOT_ENOMEM";
        case HOT_NUMERIC: return "HOT_NUMERIC";
        case HOT_TIMEOUT: return "HOT_TIMEOUT";
        case HOT_ECUDA: return "HOT_ECUDA";
        case HOT_ENOTFOUND: return "HOT_ENOTFOUND";
        case HOT_ECANCELLED: return "HOT_ECANCELLED";
        case HOT_EBUSY: return "HOT_EBUSY";
        default: return "HOT_UNKNOWN";
    }
}

const char* hot_last_error(hot_ctx* ctx) {
    (void)ctx;
    return hot::get_error();
}

int hot_create(hot_ctx** out, const hot_config* cfg) {
    HOT_GUARD_BEGIN
    if (!out) {
        set_error("out is NULL");
        return HOT_EINVAL;
    }
    *out = nullptr;
    hot_config c;
    if (cfg) c = *cfg;
    else hot_config_default(&c);
    if (c.precision != HOT_FP32_BULK && c.precision != HOT_FP64) {
        set_error("precision must be HOT_FP32_BULK or HOT_FP64");
        return HOT_EINVAL;
    }
    if (c.check_every < 2 || c.check_every > 64 || (c.check_every & 1)) {
        set_error("check_every must be even and in [2, 64]");
        return HOT_EINVAL;
    }
    if (!(c.restart_sufficient > 0 && c.restart_necessary > 0 && c.restart_long > 0)) {
        set_error("restart thresholds must be positive");
        return HOT_EINVAL;
    }
    if (c.method != HOT_METHOD_HALPERN && c.method != HOT_METHOD_GADMM) {
        set_error("method must be HOT_METHOD_HALPERN or HOT_METHOD_GADMM");
        return HOT_EINVAL;
    }
    if (c.method == HOT_METHOD_GADMM && !(c.relaxation > 0.0 && c.relaxation < 2.0)) {
        set_error("relaxation must be in (0, 2)");
        return HOT_EINVAL;
    }
    if (c.stop_rule != HOT_STOP_RELATIVE && c.stop_rule != HOT_STOP_ABSOLUTE) {
        set_error("stop_rule must be HOT_STOP_RELATIVE or HOT_STOP_ABSOLUTE");
        return HOT_EINVAL;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
        set_error("no CUDA device available");
        return HOT_ECUDA;
    }
    if (c.device < 0 || c.device >= ndev) {
        set_error("device ordinal out of range");
        return HOT_EINVAL;
    }
    HOT_CK(cudaSetDevice(c.device));
    // keep freed pool memory cached so repeated solves do not return it to the driver
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, c.device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    HOT_CK(hot::kernels_init(c.device));
    hot_ctx* h = new hot_ctx();
    hot::Ctx& x = h->impl;
    x.cfg = c;
    x.device = c.device;
    if (c.autotune_cache) x.tune_cache = c.autotune_cache;   // the caller's string is not kept
    x.cfg.autotune_cache = nullptr;
    hot::autotune_load(&x);
    if (c.stream) {
        x.stream = (cudaStream_t)c.stream;
        x.own_stream = false;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&x.stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete h;
            set_error(std::string("stream creation failed: ") + cudaGetErrorString(e));
            return HOT_ECUDA;
        }
        x.own_stream = true;
    }
    *out = h;
    return HOT_OK;
    HOT_GUARD_END
}

void hot_destroy(hot_ctx* ctx) {
    if (!ctx) return;
    try {
        cudaSetDevice(ctx->impl.device);
        delete ctx;
    } catch (...) {
    }
}

int hot_solve(hot_ctx* ctx, const double* mu, const double* nu, int m, int n, int space, double tol,
              long long max_iter, hot_result* out) {
    HOT_GUARD_BEGIN
    if (!ctx || !out) {
        set_error("ctx or out is NULL");
        return HOT_EINVAL;
    }
    if (!(tol >= 0.0) || max_iter <= 0) {
        set_error("tol must be >= 0 and max_iter > 0");
        return HOT_EINVAL;
    }
    hot::Ctx& x = ctx->impl;
    std::lock_guard<std::mutex> g(x.mu);
    HOT_CK(cudaSetDevice(x.device));
    std::vector<hot::PairHost> pairs(1);
    int rc = hot::validate_pair(mu, nu, m, n, space, x.cfg.precision == HOT_FP64, pairs[0]);
    if (rc != HOT_OK) return rc;
    return hot::run_solve(&x, pairs, tol, max_iter, true, out);
    HOT_GUARD_END
}

int hot_solve_coords(hot_ctx* ctx, const double* mu, const double* nu, int m, int n, int space, const double* xs,
                     const double* ys, double tol, long long max_iter, hot_result* out) {
    HOT_GUARD_BEGIN
    if (!ctx || !out) {
        set_error("ctx or out is NULL");
        return HOT_EINVAL;
    }
    if (!(tol >= 0.0) || max_iter <= 0) {
        set_error("tol must be >= 0 and max_iter > 0");
        return HOT_EINVAL;
    }
    hot::Ctx& x = ctx->impl;
    std::lock_guard<std::mutex> g(x.mu);
    HOT_CK(cudaSetDevice(x.device));
    std::vector<hot::PairHost> pairs(1);
    const int fp64 = x.cfg.precision == HOT_FP64;
    int rc = hot::validate_pair(mu, nu, m, n, space, fp64, pairs[0]);
    if (rc == HOT_OK) rc = hot::set_coordinates(xs, ys, m, n, fp64, pairs[0]);
    if (rc != HOT_OK) return rc;
    return hot::run_solve(&x, pairs, tol, max_iter, true, out);
    HOT_GUARD_END
}

int hot_solve_profiled(hot_ctx* ctx, const double* mu, const double* nu, int m, int n, int space, double tol,
                       long long max_iter, hot_result* out, hot_kernel_times* kt) {
    HOT_GUARD_BEGIN
    if (!ctx || !out || !kt) {
        set_error("ctx, out or kt is NULL");
        return HOT_EINVAL;
    }
    if (!(tol >= 0.0) || max_iter <= 0) {
        set_error("tol must be >= 0 and max_iter > 0");
        return HOT_EINVAL;
    }
    hot::Ctx& x = ctx->impl;
    std::lock_guard<std::mutex> g(x.mu);
    HOT_CK(cudaSetDevice(x.device));
    std::vector<hot::PairHost> pairs(1);
    int rc = hot::validate_pair(mu, nu, m, n, space, x.cfg.precision == HOT_FP64, pairs[0]);
    if (rc != HOT_OK) return rc;
    return hot::run_solve(&x, pairs, tol, max_iter, true, out, kt);
    HOT_GUARD_END
}

int hot_sweep_timing(hot_ctx* ctx, int enable, double* total_ms, long long* launches, double* bytes) {
    HOT_GUARD_BEGIN
    if (!ctx) {
        set_error("ctx is NULL");
        return HOT_EINVAL;
    }
    if (enable < -1 || enable > 1) {
        set_error("enable must be -1, 0 or 1");
        return HOT_EINVAL;
    }
    hot::Ctx& x = ctx->impl;
    std::lock_guard<std::mutex> g(x.mu);
    if (total_ms) *total_ms = x.st_ms;
    if (launches) *launches = x.st_launches;
    if (bytes) *bytes = x.st_bytes;
    x.st_ms = 0.0;
    x.st_bytes = 0.0;
    x.st_launches = 0;
    if (enable >= 0) x.sweep_timing = enable;
    return HOT_OK;
    HOT_GUARD_END
}

int hot_solve_batch(hot_ctx* ctx, int count, const double* const* mus, const double* const* nus, const int* ms,
                    const int* ns, int space, double tol, long long max_iter, hot_result* out) {
    HOT_GUARD_BEGIN
    if (!ctx || !out || count < 0 || (count > 0 && (!mus || !nus || !ms || !ns))) {
        set_error("bad arguments to hot_solve_batch");
        return HOT_EINVAL;
    }
    if (!(tol >= 0.0) || max_iter <= 0) {
        set_error("tol must be >= 0 and max_iter > 0");
        return HOT_EINVAL;
    }
    if (count == 0) return HOT_OK;
    hot::Ctx& x = ctx->impl;
    std::lock_guard<std::mutex> g(x.mu);
    HOT_CK(cudaSetDevice(x.device));
    std::vector<hot::PairHost> pairs(count);
    for (int q = 0; q < count; ++q) {
        int rc = hot::validate_pair(mus[q], nus[q], ms[q], ns[q], space, x.cfg.precision == HOT_FP64, pairs[q]);
        if (rc != HOT_OK) return rc;
    }
    const bool keep = x.cfg.keep_batch_solutions != 0;
    return hot::run_solve(&x, pairs, tol, max_iter, keep, out);
    HOT_GUARD_END
}

int hot_get_flows(hot_ctx* ctx, unsigned long long solution_id, double* xout, int space) {
    HOT_GUARD_BEGIN
    if (!ctx || !xout) {
        set_error("ctx or x is NULL");
        return HOT_EINVAL;
    }
    hot::Ctx& x = ctx->impl;
    std::lock_guard<std::mutex> g(x.mu);
    auto it = x.solutions.find(solution_id);
    if (it == x.solutions.end()) {
        set_error("unknown solution id");
        return HOT_ENOTFOUND;
    }
    HOT_CK(cudaSetDevice(x.device));
    return hot::export_flows(it->second.inst, xout, space, x.stream);
    HOT_GUARD_END
}

int hot_recover_plan(hot_ctx* ctx, unsigned long long solution_id, int32_t* src, int32_t* dst, double* mass,
                     int space, size_t cap, size_t* nnz, double* marg_l1) {
    HOT_GUARD_BEGIN
    if (!ctx || !nnz) {
        set_error("ctx or nnz is NULL");
        return HOT_EINVAL;
    }
    if (cap > 0 && (!src || !dst || !mass)) {
        set_error("output arrays are NULL");
        return HOT_EINVAL;
    }
    if (space != HOT_SPACE_HOST && space != HOT_SPACE_DEVICE) {
        set_error("bad space");
        return HOT_EINVAL;
    }
    hot::Ctx& x = ctx->impl;
    std::lock_guard<std::mutex> g(x.mu);
    auto it = x.solutions.find(solution_id);
    if (it == x.solutions.end()) {
        set_error("unknown solution id");
        return HOT_ENOTFOUND;
    }
    HOT_CK(cudaSetDevice(x.device));
    return hot::recover_plan(&x, it->second.inst, src, dst, mass, space, cap, nnz, marg_l1, x.stream);
    HOT_GUARD_END
}

int hot_release(hot_ctx* ctx, unsigned long long solution_id) {
    HOT_GUARD_BEGIN
    if (!ctx) return HOT_EINVAL;
    hot::Ctx& x = ctx->impl;
    std::lock_guard<std::mutex> g(x.mu);
    auto it = x.solutions.find(solution_id);
    if (it == x.solutions.end()) {
        set_error("unknown solution id");
        return HOT_ENOTFOUND;
    }
    HOT_CK(cudaSetDevice(x.device));
    HOT_CK(cudaStreamSynchronize(x.stream));
    hot::inst_destroy(it->second.inst, x.stream);
    x.solutions.erase(it);
    return HOT_OK;
    HOT_GUARD_END
}

int hot_submit(hot_ctx* ctx, const hot_request* req, unsigned long long* ticket) {
    HOT_GUARD_BEGIN
    if (!ctx) return HOT_EINVAL;
    return hot::serve_submit(&ctx->impl, req, ticket);
    HOT_GUARD_END
}

int hot_poll(hot_ctx* ctx, unsigned long long ticket, hot_result* out) {
    HOT_GUARD_BEGIN
    if (!ctx) return HOT_EINVAL;
    return hot::serve_poll(&ctx->impl, ticket, 0.0, out);
    HOT_GUARD_END
}

int hot_wait(hot_ctx* ctx, unsigned long long ticket, double timeout_ms, hot_result* out) {
    HOT_GUARD_BEGIN
    if (!ctx) return HOT_EINVAL;
    if (timeout_ms == 0.0) return hot::serve_poll(&ctx->impl, ticket, 0.0, out);
    return hot::serve_poll(&ctx->impl, ticket, timeout_ms, out);
    HOT_GUARD_END
}

int hot_cancel(hot_ctx* ctx, unsigned long long ticket) {
    HOT_GUARD_BEGIN
    if (!ctx) return HOT_EINVAL;
    return hot::serve_cancel(&ctx->impl, ticket);
    HOT_GUARD_END
}

int hot_forget(hot_ctx* ctx, unsigned long long ticket) {
    HOT_GUARD_BEGIN
    if (!ctx) return HOT_EINVAL;
    return hot::serve_forget(&ctx->impl, ticket);
    HOT_GUARD_END
}

int hot_serve_stats_get(hot_ctx* ctx, hot_serve_stats* out) {
    HOT_GUARD_BEGIN
    if (!ctx) return HOT_EINVAL;
    return hot::serve_stats(&ctx->impl, out);
    HOT_GUARD_END
}

int hot_barycentric_map(const int32_t* src, const int32_t* dst, const double* mass, size_t nnz, const double* y,
                        int ndst, int D, double* out, double* weight, int nsrc, void* stream) {
    HOT_GUARD_BEGIN
    return hot::barycentric_map(src, dst, mass, nnz, y, ndst, D, out, weight, nsrc, (cudaStream_t)stream);
    HOT_GUARD_END
}

int hot_autotune(hot_ctx* ctx, int S, int* tile_rows, double* us_per_iter) {
    HOT_GUARD_BEGIN
    if (!ctx) {
        set_error("ctx is NULL");
        return HOT_EINVAL;
    }
    hot::Ctx& x = ctx->impl;
    std::lock_guard<std::mutex> g(x.mu);
    HOT_CK(cudaSetDevice(x.device));
    return hot::autotune(&x, S, tile_rows, us_per_iter);
    HOT_GUARD_END
}

int hot_autotune_cache_lookup(const char* path, const char* device, int precision, int S, int* tile_rows,
                              double* us_per_iter) {
    HOT_GUARD_BEGIN
    return hot::autotune_cache_lookup(path, device, precision, S, tile_rows, us_per_iter);
    HOT_GUARD_END
}

}  // extern "C"
