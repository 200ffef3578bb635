/*
 * hot.h -- C ABI of libhot, a GB300 (sm_103a) implementation of the HOT method
 * (Halpern-accelerated splitting on the reduced optimal-transport model) of
 * Zhang, Gu, Yuan, Sun, "HOT: An Efficient Halpern Accelerating Algorithm for
 * Optimal Transport Problems", arXiv 2408.00598.
 *
 * Problem (Sec. II-A, eq. (1)-(2)): two histograms mu (source) and nu (target)
 * on an m x n grid, each non-negative with total mass 1, cost
 * c_{ij;kl} = (i-k)^2 + (j-l)^2; the library returns the optimal value of
 * eq. (1) computed through the equivalent reduced model eq. (3), and on request
 * the transport plan of Algorithm 1.  Plan entries run from source bin
 * (i, j), index i*n + j of mu, to target bin (k, l), index k*n + l of nu.
 *
 * Conventions for every entry point:
 *   - histograms are row-major m x n arrays of double: mu[i*n + j] is the mass
 *     of bin (i, j) (row i, column j);
 *   - m and n are in [2, 1024] (FP64 mode: [2, 512]); m may differ from n
 *     (the cost along each axis is that axis' own squared distance, Sec.
 *     II-A); other shapes return HOT_EINVAL;
 *   - a histogram is valid when every entry is finite and >= 0 and its sum is
 *     1 within 1e-9; unequal masses are rejected, never renormalised;
 *   - pointers marked "host or device" are read according to `space`
 *     (HOT_SPACE_HOST / HOT_SPACE_DEVICE); device pointers must be
 *     addressable from the context's device;
 *   - the caller keeps ownership of every buffer it passes; the library copies
 *     inputs before the call returns (solve, submit) and writes outputs only
 *     into caller buffers; the library's own device memory is released by
 *     hot_release / hot_destroy;
 *   - every function returns an int status (below); no exception, abort or
 *     exit crosses the ABI; hot_last_error(ctx) gives a one-line reason for
 *     the last failure on the calling thread.
 */
#ifndef HOT_H_
#define HOT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HOT_ABI_VERSION 1

/* Symbols of the ABI are exported even when the library is built with hidden
 * default visibility. */
#if defined(__GNUC__)
#define HOT_API __attribute__((visibility("default")))
#else
#define HOT_API
#endif

/* ---- status codes ------------------------------------------------------- */
#define HOT_OK              0   /* converged: relative KKT <= tol             */
#define HOT_PENDING         1   /* hot_poll: request not finished yet         */
#define HOT_NOT_CONVERGED   2   /* iteration cap reached; result still filled */
#define HOT_EINVAL        (-1)  /* invalid argument or histogram              */
#define HOT_ENOMEM        (-2)  /* device memory (or budget) exhausted        */
#define HOT_NUMERIC       (-3)  /* NaN/Inf met in the KKT reductions          */
#define HOT_TIMEOUT       (-4)  /* a bounded wait ran out                      */
#define HOT_ECUDA         (-5)  /* CUDA runtime error                          */
#define HOT_ENOTFOUND     (-6)  /* unknown ticket or solution id               */
#define HOT_ECANCELLED    (-7)  /* request cancelled before it finished        */
#define HOT_EBUSY         (-8)  /* queue full                                  */

/* ---- enums -------------------------------------------------------------- */
#define HOT_FP32_BULK  0   /* flow state in FP32 (anchor + delta), FP64 solve and reductions */
#define HOT_FP64       1   /* everything in FP64                                             */

#define HOT_SPACE_HOST    0
#define HOT_SPACE_DEVICE  1

/* Iteration (Step 4 of Algorithm 2).  HOT_METHOD_GADMM is the generalized
   ADMM the paper compares against (Sec. IV-A): Step 4 replaced by
   w^{k+1} = (1 - rho) w^k + rho w-bar^k; the restart rule and sigma update
   apply unchanged. */
#define HOT_METHOD_HALPERN 0
#define HOT_METHOD_GADMM   1
/* Stopping rule: the relative KKT residual eq. (kkt_res), or the absolute one
   of Table VI (the same three terms without their normalisers).  Both are
   measured on the scaled problem and both are reported. */
#define HOT_STOP_RELATIVE  0
#define HOT_STOP_ABSOLUTE  1

typedef struct hot_ctx hot_ctx;

/* ---- configuration (hot_config_default fills the defaults) -------------- */
typedef struct hot_config {
    int    device;              /* CUDA device ordinal                                      */
    void  *stream;              /* cudaStream_t for hot_solve*; NULL: the context makes one  */
    int    precision;           /* HOT_FP32_BULK (default) or HOT_FP64                      */
    int    check_every;         /* K: iterations between KKT/restart checks; even, 2..64 (10) */
    double sigma0;              /* initial sigma; <= 0: ||b|| / ||c|| of the scaled problem */
    double restart_sufficient;  /* restart when r <= this * r0                  (0.2)       */
    double restart_necessary;   /* ... or r <= this * r0 and r grew             (0.8)       */
    double restart_long;        /* ... or the cycle is >= this * total iterations (0.2)    */
    size_t mem_budget;          /* bytes of device memory the serve loop may hold; 0: 80 % of free */
    int    max_batch;           /* instances resident at once in the serve loop (0: 1024)   */
    int    max_queue;           /* queued requests before hot_submit returns HOT_EBUSY (0: 65536) */
    const char *autotune_cache; /* file of tuned tile shapes (hot_autotune); NULL: no file   */
    int    keep_batch_solutions;/* 1: hot_solve_batch keeps every final iterate (solution_id) */
    int    method;              /* HOT_METHOD_HALPERN (Algorithm 2, default) or HOT_METHOD_GADMM */
    double relaxation;          /* rho of HOT_METHOD_GADMM, in (0, 2)                   (1.7) */
    int    stop_rule;           /* HOT_STOP_RELATIVE (eq. kkt_res, default) or HOT_STOP_ABSOLUTE */
    int    reserved[3];
} hot_config;

/* ---- result of one solve ------------------------------------------------ */
typedef struct hot_result {
    double ot_value;      /* <c, x-bar>: the optimal-transport value, unscaled (eq. 1)       */
    double dual_value;    /* <b, y-bar>, unscaled (dual objective of eq. 9)                  */
    double rel_kkt;       /* relative KKT residual eq. (kkt_res) on the scaled problem       */
    double rel_dual;      /* ||A^T y + z - c|| / (1 + ||c||)                                  */
    double rel_comp;      /* ||min(x, z)|| / (1 + ||x|| + ||z||)                               */
    double rel_primal;    /* ||A x - b|| / (1 + ||b||)                                         */
    double sigma;         /* sigma at termination                                              */
    double cost_scale;    /* power-of-two scale the cost was divided by                        */
    double solve_ms;      /* hot_solve: device time of the solve; hot_solve_batch: time from
                             the batch's start until this pair's last check was seen complete;
                             serve loop: time from admission to completion                     */
    double queue_ms;      /* serve loop: wait between hot_submit and admission                 */
    long long iters;      /* iterations of Algorithm 2 performed                               */
    int    restarts;
    int    status;        /* HOT_OK, HOT_NOT_CONVERGED or HOT_NUMERIC                          */
    unsigned long long solution_id;   /* handle for hot_get_flows / hot_recover_plan / hot_release; 0: none kept */
    float  max_abs_dual;  /* largest |A^T y| entry seen (scaled), a numerics diagnostic       */
    int    m, n;
    long long kernel_launches;  /* device kernels this call launched (early-exiting ones included) */
    long long blocks;           /* check blocks (K iterations each) launched                      */
    double abs_kkt;             /* absolute KKT residual (Table VI) on the scaled problem          */
} hot_result;

/* Fill `cfg` with the defaults listed above.  Never fails. */
HOT_API void hot_config_default(hot_config *cfg);

/* Create a context on cfg->device.  Allocates nothing large; fails with
 * HOT_ECUDA if the device cannot be used, HOT_EINVAL for a bad config. */
HOT_API int hot_create(hot_ctx **out, const hot_config *cfg);

/* Free every device and host resource of the context, cancelling queued
 * requests and waiting (bounded) for work in flight.  NULL is a no-op. */
HOT_API void hot_destroy(hot_ctx *ctx);

/* Human-readable name of a status code (static storage). */
HOT_API const char *hot_status_string(int status);

/* Last error message recorded on the calling thread for `ctx` (or globally
 * when ctx is NULL); "" if none.  Valid until the next call on this thread. */
HOT_API const char *hot_last_error(hot_ctx *ctx);

/* Solve one pair synchronously (Algorithm 2 with the Prop. 3 linear solve, the
 * stopping rule eq. (kkt_res) at tolerance `tol`; the iteration cap is tested
 * at check iterations, so up to check_every-1 more iterations than max_iter
 * may run).  mu, nu: host or device (space), m*n doubles each.  On success
 * (HOT_OK or HOT_NOT_CONVERGED) *out is filled and out->solution_id keeps the
 * final iterate on the device until hot_release. */
HOT_API int hot_solve(hot_ctx *ctx, const double *mu, const double *nu, int m, int n, int space,
              double tol, long long max_iter, hot_result *out);

/* hot_solve on bins with given coordinates (Sec. IV-B, App. E: colour and
 * point-cloud bins need not sit on a unit grid): the cost of moving mass
 * from bin (i, j) to bin (k, l) is (xs[i] - xs[k])^2 + (ys[j] - ys[l])^2.
 *   xs: host, m doubles (coordinates of the row index i, k)
 *   ys: host, n doubles (coordinates of the column index j, l)
 *   xs = ys = NULL: the unit grid 0..m-1, 0..n-1 (as hot_solve).
 * Coordinates must be finite.  FP32 bulk mode forms the reduced cost exactly
 * on the cost grid for integer coordinates in [-2048, 2048]; it solves
 * eq. (1) with every coordinate rounded to FP32 (exact for integers up to
 * 2^24, the results are those of the rounded positions), and for
 * non-integer or larger coordinates forms the reduced cost and the
 * objective's parts in double-float pairs, in a slower sweep.  The cost is scaled by the power of two 2^ceil(log2 max c); results
 * are unscaled as for hot_solve. */
HOT_API int hot_solve_coords(hot_ctx *ctx, const double *mu, const double *nu, int m, int n, int space,
                             const double *xs, const double *ys, double tol, long long max_iter, hot_result *out);

/* Solve `count` independent pairs in one batched, graph-captured device loop;
 * each pair stops on its own when it converges.  mus[q], nus[q]: host or
 * device (space) arrays of ms[q]*ns[q] doubles.  out: `count` results.
 * Returns HOT_OK if every call-level step succeeded (per-pair outcomes are in
 * out[q].status), or the first error. */
HOT_API int hot_solve_batch(hot_ctx *ctx, int count, const double *const *mus, const double *const *nus,
                    const int *ms, const int *ns, int space, double tol, long long max_iter,
                    hot_result *out);

/* Copy the final flows x-bar = [f1; f2] of a kept solution, in the vec order
 * of eq. (4)-(6) (f1_{i,k,j} at i + m*k + m*m*j, then f2_{k,j,l} at
 * m*m*n + k + m*j + m*n*l), as m*m*n + m*n*n doubles into x (host or device). */
HOT_API int hot_get_flows(hot_ctx *ctx, unsigned long long solution_id, double *x, int space);

/* Transport plan by Algorithm 1 (run on the device, one intermediate node
 * (k, j) per warp) from the clipped flows max(x-bar, 0) of a kept solution.
 * Entries pi_{ij;kl} > 0 are written as COO triplets, ordered by node (k, j),
 * then i, then l:  src[q] = i*n + j,  dst[q] = k*n + l,  mass[q] = pi.
 * The three arrays live in `space` and hold `cap` entries each.  Call with
 * cap = 0 (arrays may be NULL) to get the exact count in *nnz; if cap < count,
 * nothing is written and HOT_EINVAL is returned with *nnz set.  marg_l1
 * (optional, 2 doubles, host): L1 distance of the plan's source and target
 * marginals to mu and nu. */
HOT_API int hot_recover_plan(hot_ctx *ctx, unsigned long long solution_id, int32_t *src, int32_t *dst,
                     double *mass, int space, size_t cap, size_t *nnz, double *marg_l1);

/* Per-kernel-family device times of one profiled solve (hot_solve_profiled). */
typedef struct hot_kernel_times {
    double    sweep_ms;              /* Steps 2-4 fused sweep, non-check iterations: total ms     */
    long long sweep_launches;
    double    sweep_check_ms;        /* the same sweep on check iterations (adds KKT sums)        */
    long long sweep_check_launches;
    double    solve_ms;              /* Prop. 3 kernels (slab sums -> y-bar -> alpha/beta)        */
    long long solve_launches;
    double    block_end_ms;          /* KKT check, restart rule, restart, finalisation            */
    long long block_end_launches;
    double    sweep_bytes;           /* algorithmic bytes of one non-check sweep launch:
                                        FP32 bulk 12 B per flow variable (read anchor, read
                                        delta, write delta), FP64 24 B                            */
} hot_kernel_times;

/* Diagnostics: hot_solve with the kernels launched one by one (no CUDA graph)
 * and a CUDA event pair around each kernel family on the context's stream;
 * the solve itself (iterates, result) is identical to hot_solve.  *kt gets
 * the summed device times. */
HOT_API int hot_solve_profiled(hot_ctx *ctx, const double *mu, const double *nu, int m, int n, int space,
                       double tol, long long max_iter, hot_result *out, hot_kernel_times *kt);

/* Live timing of the dominant kernel, the fused Steps 2-4 sweep of a
 * non-check iteration (the paper has no counterpart; it measures the kernel
 * inside the production path, not in a separate profiled run).  enable = 1:
 * later single-instance hot_solve calls on this context launch block graphs
 * that carry a CUDA event pair around one non-check sweep per block of
 * check_every iterations (check_every >= 2), and add each measured duration
 * to the context's counters; enable = 0: plain graphs again; enable = -1:
 * the mode is left as it is.  Every call returns the counters accumulated
 * since the previous call, then resets them: *total_ms the summed durations,
 * *launches the number of timed sweeps, *bytes their algorithmic bytes
 * (12 B per flow variable in FP32 bulk mode, 24 B in FP64 mode).  Output
 * pointers (host) may be NULL.  Batches, the serve loop and
 * hot_solve_profiled are never timed this way. */
HOT_API int hot_sweep_timing(hot_ctx *ctx, int enable, double *total_ms, long long *launches, double *bytes);

/* Algorithm 1 without any device allocation (the paper has no counterpart;
 * this exists for callers that cannot let a library allocate device memory at
 * call time: code with a fixed, pre-accounted device-memory footprint, or a
 * latency-critical loop that must not pay for or synchronise on an
 * allocation).  Its scratch is a static device array inside the library,
 * sized for square grids up to 256 x 256 (about 1.8 MB, held on every GPU
 * that loads the library until the process exits); larger or non-square
 * grids (m != n) return HOT_EINVAL.  The first call on a device resolves that array's device
 * address (cudaGetSymbolAddress) and should therefore come before any stream
 * capture.
 *   x:       device, the flows in the vec order of hot_get_flows (m*m*n + m*n*n doubles)
 *   mu, nu:  device, row-major m*n histograms, read only when marg_l1 != NULL
 *   src, dst, mass, cap, nnz: as in hot_recover_plan, outputs in device memory;
 *            cap = 0 with src == NULL only counts
 *   marg_l1: host, 2 doubles (optional)
 *   stream:  cudaStream_t to run on (NULL: the legacy default stream); the call
 *            returns after its work on that stream has finished.
 * Every call shares the one scratch array and overwrites it; calls whose work
 * overlaps on the GPU race and produce wrong results.
 * The prefix sums of Algorithm 1 are formed in FP64 from x.  For a solution of
 * an FP64-mode context the result equals hot_recover_plan's; for an FP32-bulk
 * solution (x its hot_get_flows export) hot_recover_plan works on the FP32
 * flows with double-float prefix sums, so the two plans agree to the rounding
 * of those sums (about 1e-12 of the total mass), not entry for entry. */
HOT_API int hot_recover_plan_static(const double *x, int m, int n, const double *mu, const double *nu,
                            int32_t *src, int32_t *dst, double *mass, size_t cap, size_t *nnz,
                            double *marg_l1, void *stream);

/* Barycentric projection of a transport plan, the colour-transfer use of a
 * plan (Sec. IV-B, App. G): for every source bin s,
 *     out[s] = sum_t pi(s, t) y[t] / sum_t pi(s, t),   weight[s] = sum_t pi(s, t),
 * over the entries (src[e], dst[e], mass[e]) of a plan such as the output of
 * hot_recover_plan (source bins are row-major m x n indices of mu, target
 * bins those of nu).  A source with no mass gets out = 0 and weight = 0.
 *   src, dst, mass: device, nnz entries (int32, int32, double)
 *   y:       device, ndst x D doubles, row-major (a D-vector per target bin, 1 <= D <= 8)
 *   out:     device, nsrc x D doubles, row-major (written)
 *   weight:  device, nsrc doubles (written)
 *   stream:  cudaStream_t to run on (NULL: the legacy default stream); the call
 *            returns after its work on that stream has finished.
 * Entries whose bin index is out of range are skipped and make the call
 * return HOT_EINVAL (the other entries are still applied).  Sums are FP64
 * atomic adds in unspecified order: reproducible to rounding, not bit for bit.
 * Allocates 4 bytes of device memory for the error count. */
HOT_API int hot_barycentric_map(const int32_t *src, const int32_t *dst, const double *mass, size_t nnz,
                                const double *y, int ndst, int D, double *out, double *weight, int nsrc,
                                void *stream);

/* Tile-shape autotuner.  The sweep tiles every S x S slab into bands of TR
 * rows; this times each candidate TR on a synthetic S x S instance on the
 * context's device (a fixed number of iterations, no early stop) and keeps
 * the fastest for every later instance of that size on this context,
 * including the serve loop.  With cfg.autotune_cache set, hot_create loads
 * the entries for this device from that file and hot_autotune appends its
 * result (text, one entry per line: device name, fp32|fp64, S, TR,
 * microseconds per iteration; the last entry for a key wins).
 *   tile_rows, us_per_iter: host, optional (NULL: not written)
 * Allocates and frees the device memory of one instance per candidate;
 * serialised with hot_solve on the same context.  HOT_EINVAL for grid sides
 * the solver does not take, or when the cache file cannot be written. */
HOT_API int hot_autotune(hot_ctx *ctx, int S, int *tile_rows, double *us_per_iter);

/* The entry of an autotune cache file for (device name as written there,
 * precision HOT_FP32_BULK or HOT_FP64, S): host only, needs no GPU.
 * HOT_ENOTFOUND when the file or the entry is missing. */
HOT_API int hot_autotune_cache_lookup(const char *path, const char *device, int precision, int S, int *tile_rows,
                                      double *us_per_iter);

/* Free the device memory of a kept solution.  Unknown id: HOT_ENOTFOUND. */
HOT_API int hot_release(hot_ctx *ctx, unsigned long long solution_id);

/* ---- serving: continuous batching ----------------------------------------
 * Requests of any supported size are admitted by a background loop as device
 * memory (cfg.mem_budget) and batch slots (cfg.max_batch) free up; admitted
 * instances join the running batch at the next check boundary and leave it
 * when they converge, so work of different requests overlaps on the device.
 * A request's iterates stay on the device from admission to completion.  The
 * result of a request does not depend on what else is in the batch.
 * hot_submit and hot_poll are thread-safe. */
typedef struct hot_request {
    const double *mu;       /* host, m*n doubles, copied by hot_submit */
    const double *nu;       /* host, m*n doubles, copied by hot_submit */
    int m, n;
    double tol;
    long long max_iter;
    int keep_solution;      /* 1: keep the final iterate (needs hot_release) */
    int reserved[3];
} hot_request;

typedef struct hot_serve_stats {
    long long submitted, completed, cancelled, rejected;
    int queued, running;
    size_t device_bytes_in_use;
    double p50_ms, p99_ms;          /* completion latency (submit -> done) over finished requests */
    double mean_queue_ms;
    long long blocks_run;           /* check blocks executed by the loop */
} hot_serve_stats;

/* Queue one request; *ticket identifies it.  HOT_EBUSY when the queue is
 * full, HOT_EINVAL for a bad request (nothing is queued). */
HOT_API int hot_submit(hot_ctx *ctx, const hot_request *req, unsigned long long *ticket);

/* HOT_PENDING while queued or running; otherwise the request's final status
 * with *out filled (HOT_OK / HOT_NOT_CONVERGED / HOT_NUMERIC /
 * HOT_ECANCELLED).  A finished ticket can be polled again until
 * hot_forget(ctx, ticket).  Unknown ticket: HOT_ENOTFOUND. */
HOT_API int hot_poll(hot_ctx *ctx, unsigned long long ticket, hot_result *out);

/* Like hot_poll but blocks up to timeout_ms (< 0: no limit) for completion;
 * HOT_TIMEOUT if it is still pending then. */
HOT_API int hot_wait(hot_ctx *ctx, unsigned long long ticket, double timeout_ms, hot_result *out);

/* Cancel a queued request (HOT_OK) or mark a running one to stop at its next
 * check (HOT_OK); HOT_ENOTFOUND if unknown or already finished. */
HOT_API int hot_cancel(hot_ctx *ctx, unsigned long long ticket);

/* Drop the record of a finished ticket (frees its kept solution too). */
HOT_API int hot_forget(hot_ctx *ctx, unsigned long long ticket);

/* Counters of the serve loop since hot_create. */
HOT_API int hot_serve_stats_get(hot_ctx *ctx, hot_serve_stats *out);

#ifdef __cplusplus
}
#endif
#endif /* HOT_H_ */
