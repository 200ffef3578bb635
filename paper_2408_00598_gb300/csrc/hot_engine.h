// Host engine of libhot: instance memory, batch work tables, the graph-captured
// check block, and the context object behind the C ABI.
#pragma once

#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/hot.h"
#include "hot_internal.h"

namespace hot {

void set_error(const std::string& msg);
const char* get_error();

#define HOT_CK(call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            ::hot::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));             \
            return e_ == cudaErrorMemoryAllocation ? HOT_ENOMEM : HOT_ECUDA;                 \
        }                                                                                     \
    } while (0)

// One instance's device memory and descriptor.
struct Inst {
    int m = 0, n = 0;        // grid: the histograms are m x n
    int fp64 = 0;
    int TR = 0, nb1 = 0, nb2 = 0, n_k1 = 0;
    size_t big_bytes = 0, small_bytes = 0;
    char* big = nullptr;     // v0, d0, d1, xr, zr
    char* small = nullptr;   // sums, vectors, mu, ctl
    HotInst desc{};
    double cost_scale = 1.0;
    HotCtl ctl_host{};       // last copy of the control block
    double t_admit_ms = 0.0; // serve loop bookkeeping
};

// Host-side constants of a histogram pair (validated).
struct PairHost {
    int m = 0, n = 0;
    std::vector<double> mu1, mu2;          // m x n, row-major
    std::vector<double> xs, ys;            // bin coordinates: xs[m] of rows i/k, ys[n] of columns j/l; empty: 0, 1, ...
};

// Checks bin coordinates and stores them in `out` (NULL: uniform 0, 1, ...).
int set_coordinates(const double* xs, const double* ys, int m, int n, int fp64, PairHost& out);

int validate_pair(const double* mu, const double* nu, int m, int n, int space, int fp64, PairHost& out);
// rows per sweep tile; grid: resident CTAs of the sweep (0: no balancing)
int tile_rows(int m, int n, int fp64, int grid);

// Allocate and initialise an instance on stream `st` (inputs already validated).
// Barycentric projection of a plan (hot_consumers.cu).
int barycentric_map(const int* src, const int* dst, const double* mass, size_t nnz, const double* y, int ndst,
                    int D, double* out, double* weight, int nsrc, cudaStream_t st);

int inst_create(const PairHost& p, int fp64, const hot_config& cfg, double tol, long long max_iter, int tr_override,
                cudaStream_t st, Inst** out);
void inst_destroy(Inst* I, cudaStream_t st);

// Device work tables plus the instantiated block graph that reads them.
// Prefix tables (cap + 1 ints each): tiles, slabs, k_vec items, k_kkt1 chunks, k_alpha32 chunks.
constexpr int kPreTables = 5;
struct Batch {
    int device = 0;
    int cap = 0;
    int fp64 = 0;
    int K = 10;
    double a1 = 0.2, a2 = 0.8, a3 = 0.2;
    WorkDev* d_work = nullptr;
    HotInst* d_inst = nullptr;
    int* d_pre = nullptr;
    int* d_running = nullptr;
    int* d_st = nullptr;            // [cap] per-instance status after each check
    int* h_st = nullptr;            // pinned mirror
    int* h_stb = nullptr;           // pinned, [2][cap]: statuses after the last two blocks (finish times)
    WorkDev* h_work = nullptr;      // pinned
    HotInst* h_inst = nullptr;      // pinned
    int* h_pre = nullptr;           // pinned
    int* h_running = nullptr;       // pinned, [4]
    cudaGraphExec_t graph = nullptr;
    // sweep-timing mode: two instances of the block graph, launched
    // alternately, each with a CUDA event pair around the sweep of iteration
    // timed_iter; the host reads one block's pair while the next block runs
    // on the other instance
    cudaGraphExec_t tgraph[2] = {nullptr, nullptr};
    cudaEvent_t tev[2][2] = {};
    int timing = 0;
    cudaStream_t cap_stream = nullptr;
    LaunchDims ld{};
    int ninst = 0;
    int single = -1;                // the instance count the graphs were captured for is 1 (1), more (0), none (-1)
    int pad = 0;                    // some instance needs the general sweep: a side that is not a
                                    // multiple of 4, or (FP32) real-valued bin coordinates
    int pad_captured = -1;          // pad of the captured graphs
    void drop_graphs();
    ~Batch();
    int reserve(int n);
    int set_instances(const std::vector<Inst*>& v, cudaStream_t st);   // async H2D
    int ensure_graph(int timing = 0);
    int launch_block(cudaStream_t st, long long block = 0) const;
    int timed_iter() const { return (K - 1) / 2; }   // a non-check iteration when K >= 2
    int capture(cudaGraphExec_t* out, cudaEvent_t* ev);
};

struct Solution {
    Inst* inst = nullptr;
};

struct ServeState;

struct Ctx {
    hot_config cfg{};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::mutex mu;                         // serialises hot_solve* / recovery / solutions
    std::unique_ptr<Batch> batch;          // for hot_solve / hot_solve_batch
    std::map<unsigned long long, Solution> solutions;
    std::atomic<unsigned long long> next_id{1};
    std::unique_ptr<ServeState> serve;
    int tile_override = 0;                 // force TR (0 = tuned or default); the autotuner sets it
    std::mutex tune_mu;                    // guards tuned (the serve thread reads it)
    std::map<int, std::pair<int, double>> tuned[2];   // [fp64][S] -> (TR, us per iteration)
    std::string tune_cache;                // hot_config.autotune_cache, copied
    // live timing of the non-check sweep inside the block graph (hot_sweep_timing)
    int sweep_timing = 0;
    double st_ms = 0.0, st_bytes = 0.0;
    long long st_launches = 0;
    Ctx();
    ~Ctx();
};

int run_solve(Ctx* ctx, const std::vector<PairHost>& pairs, double tol, long long max_iter, bool keep,
              hot_result* out, hot_kernel_times* kt = nullptr);
void fill_result(const Inst* I, hot_result* r);
int recover_plan(Ctx* ctx, Inst* I, int32_t* src, int32_t* dst, double* mass, int space, size_t cap, size_t* nnz,
                 double* marg_l1, cudaStream_t st);
int export_flows(Inst* I, double* x, int space, cudaStream_t st);

// tile-shape autotuner (hot_autotune.cpp)
std::vector<int> tile_candidates(int S, int fp64);
int tuned_tile_rows(Ctx* ctx, int m, int n, int fp64);   // 0: not tuned (or m != n)
void autotune_load(Ctx* ctx);
int autotune(Ctx* ctx, int S, int* tr_out, double* us_out);
int autotune_cache_lookup(const char* path, const char* device, int precision, int S, int* tr, double* us);

// serve loop (hot_serve.cpp)
void serve_shutdown(Ctx* ctx);

}  // namespace hot
