// Tile-shape autotuner.  The sweep tiles each slab into bands of TR rows
// (TR * S <= 16384 in FP32 mode, <= 4096 in FP64 mode).  Taller tiles pay
// the per-tile set-up and reductions fewer times; shorter ones spread a small
// slab set over more CTAs.  Which wins depends on S and the device, so the
// context can measure it: every candidate TR runs the same synthetic
// instance for a fixed number of iterations (tol = 0, so no early stop) and
// the fastest per-iteration time is kept for that (precision, S).  The table
// lives in the context and, when hot_config.autotune_cache names a file, in
// that file (one line per entry: device, precision, S, TR, microseconds per
// iteration), so later processes start tuned.  The table covers square S x S
// grids; an m x n grid with m != n takes the rule of tile_rows.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "hot_engine.h"

namespace hot {

namespace {

std::string device_key(int device) {
    cudaDeviceProp p{};
    std::string name = "unknown";
    if (cudaGetDeviceProperties(&p, device) == cudaSuccess) name = p.name;
    for (char& c : name)
        if (c == ' ' || c == '\t') c = '_';
    return name;
}

const char* prec_name(int fp64) { return fp64 ? "fp64" : "fp32"; }

// Entries of a cache file for one device and precision: S -> (TR, us).
bool cache_read(const std::string& path, const std::string& dev, int fp64, std::map<int, std::pair<int, double>>& t) {
    std::ifstream f(path);
    if (!f) return false;
    std::string line;
    while (std::getline(f, line)) {
        if (line.empty() || line[0] == '#') continue;
        std::istringstream is(line);
        std::string d, pr;
        int S = 0, tr = 0;
        double us = 0.0;
        if (!(is >> d >> pr >> S >> tr >> us)) continue;
        if (d != dev || pr != prec_name(fp64) || S <= 0 || tr <= 0) continue;
        t[S] = {tr, us};                       // a later line for the same S wins
    }
    return true;
}

bool cache_append(const std::string& path, const std::string& dev, int fp64, int S, int tr, double us) {
    FILE* f = std::fopen(path.c_str(), "a");
    if (!f) return false;
    std::fprintf(f, "%s %s %d %d %.3f\n", dev.c_str(), prec_name(fp64), S, tr, us);
    std::fclose(f);
    return true;
}

// Seeded white-noise histograms (host LCG; the values only need to be a
// typical dense input, the tuner does not look at the result).
void tune_pair(int S, PairHost& p) {
    p.m = p.n = S;
    p.mu1.assign((size_t)S * S, 0.0);
    p.mu2.assign((size_t)S * S, 0.0);
    unsigned long long z = 0x9E3779B97F4A7C15ull ^ (unsigned long long)S;
    auto next = [&]() {
        z = z * 6364136223846793005ull + 1442695040888963407ull;
        return 0.1 + 0.9 * (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    double s1 = 0.0, s2 = 0.0;
    for (auto& v : p.mu1) s1 += (v = next());
    for (auto& v : p.mu2) s2 += (v = next());
    for (auto& v : p.mu1) v /= s1;
    for (auto& v : p.mu2) v /= s2;
}

}  // namespace

std::vector<int> tile_candidates(int S, int fp64) {
    const int cap = fp64 ? 4096 : kMaxTileElems;
    const int Sp = (S + 3) & ~3;             // the row pitch of an S x S slab
    std::vector<int> out;
    for (int tr = std::min(S, cap / Sp); tr >= 1 && out.size() < 4; tr /= 2) {
        if ((long long)tr * Sp < 1024 && !out.empty()) break;
        if (fp64 && S >= 96 && tr > 32) continue;
        out.push_back(tr);
    }
    if (out.empty()) out.push_back(1);
    return out;
}

int tuned_tile_rows(Ctx* ctx, int m, int n, int fp64) {
    if (m != n) return 0;
    std::lock_guard<std::mutex> g(ctx->tune_mu);
    auto& t = ctx->tuned[fp64 ? 1 : 0];
    auto it = t.find(m);
    return it == t.end() ? 0 : it->second.first;
}

void autotune_load(Ctx* ctx) {
    if (ctx->tune_cache.empty()) return;
    const std::string dev = device_key(ctx->device);
    std::lock_guard<std::mutex> g(ctx->tune_mu);
    for (int fp64 = 0; fp64 < 2; ++fp64) cache_read(ctx->tune_cache, dev, fp64, ctx->tuned[fp64]);
}

int autotune(Ctx* ctx, int S, int* tr_out, double* us_out) {
    const int fp64 = ctx->cfg.precision == HOT_FP64 ? 1 : 0;
    if (S < 2 || S > kMaxS || (fp64 && S > 512)) {
        set_error("autotune: unsupported grid side");
        return HOT_EINVAL;
    }
    PairHost p;
    tune_pair(S, p);
    const std::vector<int> cand = tile_candidates(S, fp64);
    const long long iters = (long long)ctx->cfg.check_every * (S >= 512 ? 2 : 4);
    int best = 0;
    double best_us = 1e300;
    const int saved = ctx->tile_override;
    for (int tr : cand) {
        ctx->tile_override = tr;
        std::vector<PairHost> one(1, p);
        hot_result r{};
        int rc = run_solve(ctx, one, 0.0, ctx->cfg.check_every, false, &r);   // warm-up: graph, pools
        if (rc == HOT_OK || rc == HOT_NOT_CONVERGED) rc = run_solve(ctx, one, 0.0, iters, false, &r);
        if (rc != HOT_OK && rc != HOT_NOT_CONVERGED) {
            ctx->tile_override = saved;
            return rc;
        }
        const double us = 1000.0 * r.solve_ms / (double)std::max(1LL, r.iters);
        if (us < best_us) {
            best_us = us;
            best = tr;
        }
    }
    ctx->tile_override = saved;
    {
        std::lock_guard<std::mutex> g(ctx->tune_mu);
        ctx->tuned[fp64][S] = {best, best_us};
    }
    if (!ctx->tune_cache.empty() && !cache_append(ctx->tune_cache, device_key(ctx->device), fp64, S, best, best_us)) {
        set_error("autotune: cannot write the cache file " + ctx->tune_cache);
        return HOT_EINVAL;
    }
    if (tr_out) *tr_out = best;
    if (us_out) *us_out = best_us;
    return HOT_OK;
}

int autotune_cache_lookup(const char* path, const char* device, int precision, int S, int* tr, double* us) {
    if (!path || !device || !tr) {
        set_error("autotune cache lookup: null argument");
        return HOT_EINVAL;
    }
    std::map<int, std::pair<int, double>> t;
    if (!cache_read(path, device, precision == HOT_FP64 ? 1 : 0, t)) {
        set_error(std::string("autotune cache lookup: cannot read ") + path);
        return HOT_ENOTFOUND;
    }
    auto it = t.find(S);
    if (it == t.end()) {
        set_error("autotune cache lookup: no entry");
        return HOT_ENOTFOUND;
    }
    *tr = it->second.first;
    if (us) *us = it->second.second;
    return HOT_OK;
}

}  // namespace hot
