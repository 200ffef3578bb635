// Host engine: instance set-up (Sec. II-A data of arXiv 2408.00598: b, the
// power-of-two cost scale, norms), the batch work tables, the CUDA graph of
// one check block (K iterations of Algorithm 2 plus the stopping/restart
// step), and the synchronous solve entry points of the C ABI.
#include "hot_engine.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>

namespace hot {

// ------------------------------------------------------------------ errors --

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
const char* get_error() { return g_err.c_str(); }

// ------------------------------------------------------------- validation --

int tile_rows(int m, int n, int fp64, int grid) {
    // one TR for both halves: the row-partial buffer holds TR rows of the
    // longer slab pitch Lp (the side L = max(m, n) rounded up to a multiple
    // of 4); a tile has at most L rows
    const int Ls = std::max(m, n);
    const int L = (Ls + 3) & ~3;
    if (fp64) {
        // row-partial buffer: TR * Lp <= 4096
        int tr = std::min(Ls, 4096 / L);
        if (L >= 96) tr = std::min(tr, 32);
        return std::max(tr, 1);
    }
    // TR * L <= 16384 (row-partial buffer).  Tiles as tall as that allows
    // (the per-tile set-up and reductions cost more than a ragged last round
    // of the persistent grid), halved while a slab-set this small leaves some
    // of the grid's CTAs without a tile and a tile keeps at least 4 passes
    // (measured with the autotuner on GB300: TR = 64 at 64^2, 128^2 and 256^2,
    // 32 at 512^2)
    int tr = std::min(std::min(Ls, kMaxTileElems / L), kMaxTR);
    auto tiles = [&](int t) { return (long long)n * ((m + t - 1) / t) + (long long)m * ((n + t - 1) / t); };
    if (grid > 0)
        while (tiles(tr) < (long long)grid && (long long)(tr / 2) * L >= 4096) tr /= 2;
    return tr;
}

int set_coordinates(const double* xs, const double* ys, int m, int n, int fp64, PairHost& out) {
    out.xs.clear();
    out.ys.clear();
    if (!xs && !ys) return HOT_OK;
    if (!xs || !ys) {
        set_error("give both coordinate arrays or neither");
        return HOT_EINVAL;
    }
    out.xs.assign(xs, xs + m);
    out.ys.assign(ys, ys + n);
    for (int w = 0; w < 2; ++w) {
        const std::vector<double>& v = w ? out.ys : out.xs;
        for (double x : v)
            if (!std::isfinite(x)) {
                set_error("coordinates must be finite");
                return HOT_EINVAL;
            }
    }
    return HOT_OK;
}

int validate_pair(const double* mu, const double* nu, int m, int n, int space, int fp64, PairHost& out) {
    if (!mu || !nu) {
        set_error("null histogram pointer");
        return HOT_EINVAL;
    }
    const int smax = fp64 ? 512 : kMaxS;
    for (int side : {m, n})
        if (side < 2 || side > smax) {
            set_error("grid sides must be in [2, " + std::to_string(smax) + "], got " + std::to_string(m) + " x " +
                      std::to_string(n));
            return HOT_EINVAL;
        }
    out.m = m;
    out.n = n;
    const size_t M = (size_t)m * n;
    out.mu1.resize(M);
    out.mu2.resize(M);
    if (space == HOT_SPACE_DEVICE) {
        cudaError_t e1 = cudaMemcpy(out.mu1.data(), mu, M * sizeof(double), cudaMemcpyDeviceToHost);
        cudaError_t e2 = cudaMemcpy(out.mu2.data(), nu, M * sizeof(double), cudaMemcpyDeviceToHost);
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
            set_error("cannot read device histograms");
            return HOT_EINVAL;
        }
    } else if (space == HOT_SPACE_HOST) {
        std::memcpy(out.mu1.data(), mu, M * sizeof(double));
        std::memcpy(out.mu2.data(), nu, M * sizeof(double));
    } else {
        set_error("space must be HOT_SPACE_HOST or HOT_SPACE_DEVICE");
        return HOT_EINVAL;
    }
    for (int w = 0; w < 2; ++w) {
        const std::vector<double>& v = w ? out.mu2 : out.mu1;
        double s = 0.0;
        for (double x : v) {
            if (!std::isfinite(x) || x < 0.0) {
                set_error(std::string(w ? "nu" : "mu") + " has a negative or non-finite entry");
                return HOT_EINVAL;
            }
            s += x;
        }
        if (std::fabs(s - 1.0) > 1e-9) {
            char buf[128];
            std::snprintf(buf, sizeof buf, "%s must sum to 1 (got %.17g)", w ? "nu" : "mu", s);
            set_error(buf);
            return HOT_EINVAL;
        }
    }
    return HOT_OK;
}

// --------------------------------------------------------------- instances --

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int inst_create(const PairHost& p, int fp64, const hot_config& cfg, double tol, long long max_iter, int tr_override,
                cudaStream_t st, Inst** out) {
    *out = nullptr;
    std::unique_ptr<Inst> I(new Inst());
    const int m = p.m, n = p.n, L = std::max(m, n);
    const int Lp = (L + 3) & ~3;              // longest row pitch
    I->m = m;
    I->n = n;
    I->fp64 = fp64;
    I->TR = tr_override > 0 ? tr_override : tile_rows(m, n, fp64, sweep_grid(fp64));
    const int NV = fp64 ? 2 : 4;
    if (I->TR > (fp64 ? L : kMaxTR) || (size_t)I->TR * Lp > (size_t)(fp64 ? 4096 : kMaxTileElems) ||
        kThreads / (Lp / NV) < 1) {
        set_error("invalid tile rows for this grid");
        return HOT_EINVAL;
    }
    I->nb1 = (m + I->TR - 1) / I->TR;
    I->nb2 = (n + I->TR - 1) / I->TR;
    const size_t MN = (size_t)m * n;
    I->n_k1 = (int)((3 * MN - 1 + kThreads - 1) / kThreads);
    // flow variables: n f1 slabs of m x m, m f2 slabs of n x n, rows stored
    // at a pitch of the side rounded up to a multiple of 4
    const int mp = (m + 3) & ~3, np = (n + 3) & ~3;
    const size_t V = MN * (size_t)(mp + np);
    const size_t es = fp64 ? 8 : 4;
    I->big_bytes = 5 * align256(V * es);

    // small-buffer layout; per-slab arrays hold 2mn entries (one per slab row:
    // n slabs of m rows, m slabs of n rows), column partials one per band
    const int ntiles = n * I->nb1 + m * I->nb2;
    const size_t CP = (size_t)n * I->nb1 * m + (size_t)m * I->nb2 * n;   // column-partial entries
    const int NS = m + n;                                                  // slabs
    const int n_achunk = (int)((4 * MN + kAlphaChunk - 1) / kAlphaChunk);   // k_alpha32 chunks
    const size_t NPART = (size_t)std::max(NS, n_achunk);                   // <b, y> partials
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return o;
    };
    const size_t o_ab32 = fp64 ? 0 : take(4 * MN * sizeof(float4));
    const size_t o_ab0_32 = fp64 ? 0 : take(4 * MN * sizeof(float2));   // y0 = 0 at the start
    const size_t o_ab64 = take(4 * MN * 8);
    const size_t o_dab = take(4 * MN * 8);
    const size_t o_ab0 = take(4 * MN * 8);      // A^T y0 pieces: y0 = 0 at the start
    const size_t o_rs = take(2 * MN * 8);
    const size_t o_cs = take(CP * 8);
    const size_t o_cs32 = take(CP * 4);
    const size_t o_R1a = take(2 * MN * 8);
    const size_t o_kapa = take(2 * MN * 8);
    const size_t o_rs0 = take(2 * MN * 8);
    const size_t o_cs0 = take(CP * 8);
    const size_t o_xrs = take(2 * MN * 8);
    const size_t o_xcs = take(CP * 8);
    const size_t o_tk = take((size_t)ntiles * kNK * 8);
    const size_t o_rp = take((size_t)ntiles * 2 * 8);
    const size_t o_vec = take(4 * (size_t)L * 8);
    const size_t o_mvec = take(4 * (size_t)L * 8);
    const size_t F2 = fp64 ? 0 : sizeof(float2);   // double-float arrays of FP32 mode
    const size_t o_rs2 = take(2 * MN * F2);
    const size_t o_rs02 = take(2 * MN * F2);
    const size_t o_K2 = take(2 * MN * F2);
    const size_t o_vec2 = take(vec2_entries(m, n) * F2);
    const size_t o_dab2 = take(4 * MN * F2);
    const size_t o_stg2 = take(4 * (size_t)L * F2);
    const size_t o_vcnt = take(sizeof(unsigned int));
    const size_t o_zero_end = off;                 // everything above starts at 0
    const size_t o_mu1f = take(MN * F2);
    const size_t o_mu2f = take(MN * F2);
    const size_t o_cm2 = take(n * F2);
    const size_t o_rm2 = take(m * F2);
    const size_t o_p32 = take(sizeof(P32));
    const size_t o_X32 = take((size_t)NS * sizeof(float));
    const size_t o_X64 = take((size_t)NS * sizeof(double));
    const size_t o_cs2 = take((size_t)NS * sizeof(float2));
    const size_t o_cyc = take(sizeof(CycleK));
    const size_t o_mu1 = take(MN * 8);
    const size_t o_mu2 = take(MN * 8);
    const size_t o_cm = take(n * 8);
    const size_t o_rm = take(m * 8);
    const size_t o_k1 = take((size_t)I->n_k1 * 8);
    const size_t o_dp = take(NPART * 8);
    const size_t o_cu = take((size_t)ntiles * 8);
    const size_t o_cD = take(NPART * 8);
    const size_t o_ctl = take(sizeof(HotCtl));
    I->small_bytes = off;

    cudaError_t e = cudaMallocAsync((void**)&I->big, I->big_bytes, st);
    if (e != cudaSuccess) {
        set_error(std::string("device allocation of the flow state failed: ") + cudaGetErrorString(e));
        return HOT_ENOMEM;
    }
    e = cudaMallocAsync((void**)&I->small, I->small_bytes, st);
    if (e != cudaSuccess) {
        cudaFreeAsync(I->big, st);
        set_error(std::string("device allocation failed: ") + cudaGetErrorString(e));
        return HOT_ENOMEM;
    }
    HotInst& d = I->desc;
    d.m = m;
    d.n = n;
    d.mp = mp;
    d.np = np;
    d.TR = I->TR;
    d.nb1 = I->nb1;
    d.nb2 = I->nb2;
    d.n_k1 = I->n_k1;
    d.n_achunk = n_achunk;
    d.fp64 = fp64;
    d.gadmm = cfg.method == HOT_METHOD_GADMM ? 1 : 0;
    d.stop_abs = cfg.stop_rule == HOT_STOP_ABSOLUTE ? 1 : 0;
    d.relax = cfg.relaxation;
    // FP32 mode: integer coordinates of modest size keep the reduced cost
    // exact on the grid 2^-E; others (and FP64 mode never needs it) take the
    // pair arithmetic of the general sweep
    d.coord_real = 0;
    if (!fp64)
        for (const std::vector<double>* v : {&p.xs, &p.ys})
            for (double x : *v)
                if (x != std::rint(x) || std::fabs(x) > 2048.0) d.coord_real = 1;
    // bin coordinates: X[0, m) are the row coordinates (i, k) that the f1
    // slabs' cost uses, X[m, m + n) the column coordinates (j, l) of the f2
    // slabs; default 0, 1, ...
    std::vector<double> X((size_t)NS);
    for (int r = 0; r < m; ++r) X[r] = p.xs.empty() ? (double)r : p.xs[r];
    for (int r = 0; r < n; ++r) X[m + r] = p.ys.empty() ? (double)r : p.ys[r];
    // FP32 mode solves eq. (1) with the positions rounded to FP32 (exact for
    // integers up to 2^24): the cost scale, ||c||, C(x) and every cost the
    // kernels form all come from the same rounded positions
    if (!fp64)
        for (double& x : X) x = (double)(float)x;
    const int hb[3] = {0, m, m + n};
    // power-of-two cost scale: smallest 2^E >= max c (E = 0 for a zero cost)
    double cmax = 0.0;
    for (int hlf = 0; hlf < 2; ++hlf) {
        const auto mm = std::minmax_element(X.begin() + hb[hlf], X.begin() + hb[hlf + 1]);
        cmax = std::max(cmax, (*mm.second - *mm.first) * (*mm.second - *mm.first));
    }
    int E = 0;
    if (cmax > 0.0) {
        E = (int)std::ceil(std::log2(cmax));
        while (std::ldexp(1.0, E) < cmax) ++E;
        while (std::ldexp(1.0, E - 1) >= cmax) --E;
    }
    d.E = E;
    d.h = std::ldexp(1.0, -E);
    I->cost_scale = std::ldexp(1.0, E);
    // ||c||: the n f1 slabs share one cost matrix, the m f2 slabs another;
    // C(x) = sum_y (X_x - X_y)^2 within each half
    double c4[2] = {0.0, 0.0};
    std::vector<double> csum((size_t)NS, 0.0);
    for (int hlf = 0; hlf < 2; ++hlf)
        for (int a = hb[hlf]; a < hb[hlf + 1]; ++a)
            for (int t = hb[hlf]; t < hb[hlf + 1]; ++t) {
                const double dx = X[a] - X[t];
                const double dd = dx * dx;
                c4[hlf] += dd * dd;
                csum[a] += dd;
            }
    d.norm_c = d.h * std::sqrt((double)n * c4[0] + (double)m * c4[1]);
    double b2 = 0.0;
    for (double x : p.mu1) b2 += x * x;
    for (double x : p.mu2) b2 += x * x;
    b2 -= p.mu2[MN - 1] * p.mu2[MN - 1];
    d.norm_b = std::sqrt(b2);
    double s1 = 0.0, s2 = 0.0;
    for (double x : p.mu1) s1 += x;
    for (double x : p.mu2) s2 += x;
    d.sum_mu1 = s1;
    d.sum_mu2 = s2;
    char* big = I->big;
    const size_t VB = align256(V * es);
    d.u = big;
    d.d0 = big + VB;
    d.d1 = big + 2 * VB;
    d.xr = big + 3 * VB;
    d.zr = big + 4 * VB;
    char* sm = I->small;
    d.ab32 = fp64 ? nullptr : (float4*)(sm + o_ab32);
    d.ab0_32 = fp64 ? nullptr : (float2*)(sm + o_ab0_32);
    d.cs32 = (float*)(sm + o_cs32);
    d.R1a = (double*)(sm + o_R1a);
    d.kapa = (double*)(sm + o_kapa);
    d.ab64 = (double*)(sm + o_ab64);
    d.dab64 = (double*)(sm + o_dab);
    d.ab0 = (double*)(sm + o_ab0);
    d.rs = (double*)(sm + o_rs);
    d.cs_part = (double*)(sm + o_cs);
    d.rs0 = (double*)(sm + o_rs0);
    d.cs0_part = (double*)(sm + o_cs0);
    d.xrs = (double*)(sm + o_xrs);
    d.xcs_part = (double*)(sm + o_xcs);
    d.tile_kkt = (double*)(sm + o_tk);
    d.rst_part = (double*)(sm + o_rp);
    d.vecs = (double*)(sm + o_vec);
    d.mvec = (double*)(sm + o_mvec);
    d.mu1 = (double*)(sm + o_mu1);
    d.mu2 = (double*)(sm + o_mu2);
    d.colmu1 = (double*)(sm + o_cm);
    d.rowmu2 = (double*)(sm + o_rm);
    d.k1_part = (double*)(sm + o_k1);
    d.dobj_part = (double*)(sm + o_dp);
    d.cu_part = (double*)(sm + o_cu);
    d.cD_part = (double*)(sm + o_cD);
    d.rs2 = fp64 ? nullptr : (float2*)(sm + o_rs2);
    d.rs02 = fp64 ? nullptr : (float2*)(sm + o_rs02);
    d.K2 = fp64 ? nullptr : (float2*)(sm + o_K2);
    d.vec2 = fp64 ? nullptr : (float2*)(sm + o_vec2);
    d.dab2 = fp64 ? nullptr : (float2*)(sm + o_dab2);
    d.stg2 = fp64 ? nullptr : (float2*)(sm + o_stg2);
    d.vcount = (unsigned int*)(sm + o_vcnt);
    d.mu1f = fp64 ? nullptr : (float2*)(sm + o_mu1f);
    d.mu2f = fp64 ? nullptr : (float2*)(sm + o_mu2f);
    d.cm2 = fp64 ? nullptr : (float2*)(sm + o_cm2);
    d.rm2 = fp64 ? nullptr : (float2*)(sm + o_rm2);
    d.p32 = (P32*)(sm + o_p32);
    d.X32 = (float*)(sm + o_X32);
    d.X64 = (double*)(sm + o_X64);
    d.csum2 = (float2*)(sm + o_cs2);
    d.cyc = (CycleK*)(sm + o_cyc);
    d.ctl = (HotCtl*)(sm + o_ctl);

    // host-side constants uploaded once
    std::vector<double> cm(n, 0.0), rm(m, 0.0);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) {
            cm[j] += p.mu1[(size_t)i * n + j];
            rm[i] += p.mu2[(size_t)i * n + j];
        }
    HotCtl c{};
    c.sigma = cfg.sigma0 > 0.0 ? cfg.sigma0 : d.norm_b / d.norm_c;
    c.tol = tol;
    c.r0 = -1.0;
    c.rprev = -1.0;
    c.max_iter = max_iter;
    c.status = ST_RUNNING;
    I->ctl_host = c;

    cudaError_t ee = cudaMemsetAsync(sm, 0, o_zero_end, st);
    if (ee == cudaSuccess) ee = cudaMemcpyAsync(d.mu1, p.mu1.data(), MN * 8, cudaMemcpyHostToDevice, st);
    if (ee == cudaSuccess) ee = cudaMemcpyAsync(d.mu2, p.mu2.data(), MN * 8, cudaMemcpyHostToDevice, st);
    if (ee == cudaSuccess) ee = cudaMemcpyAsync(d.colmu1, cm.data(), n * 8, cudaMemcpyHostToDevice, st);
    if (ee == cudaSuccess) ee = cudaMemcpyAsync(d.rowmu2, rm.data(), m * 8, cudaMemcpyHostToDevice, st);
    if (ee == cudaSuccess) ee = cudaMemcpyAsync(d.ctl, &I->ctl_host, sizeof(HotCtl), cudaMemcpyHostToDevice, st);
    {
        // coordinates (FP32 mode: already rounded, so the FP32 copies are
        // exact) and the row cost sums C(x) as double-float pairs
        std::vector<float> x32(X.begin(), X.end());
        std::vector<float2> cs2(csum.size());
        for (size_t q = 0; q < csum.size(); ++q) {
            const float hh = (float)csum[q];
            cs2[q] = make_float2(hh, (float)(csum[q] - (double)hh));
        }
        if (ee == cudaSuccess) ee = cudaMemcpyAsync((void*)d.X32, x32.data(), x32.size() * sizeof(float), cudaMemcpyHostToDevice, st);
        if (ee == cudaSuccess) ee = cudaMemcpyAsync((void*)d.X64, X.data(), X.size() * sizeof(double), cudaMemcpyHostToDevice, st);
        if (ee == cudaSuccess) ee = cudaMemcpyAsync((void*)d.csum2, cs2.data(), cs2.size() * sizeof(float2), cudaMemcpyHostToDevice, st);
    }
    if (!fp64) {
        // (hi, lo) pairs of the marginals: hi = fl32(x), lo = fl32(x - hi)
        auto pairs = [](const double* x, size_t n) {
            std::vector<float2> v(n);
            for (size_t q = 0; q < n; ++q) {
                const float h = (float)x[q];
                v[q] = make_float2(h, (float)(x[q] - (double)h));
            }
            return v;
        };
        const std::vector<float2> f1 = pairs(p.mu1.data(), MN), f2 = pairs(p.mu2.data(), MN);
        const std::vector<float2> fc = pairs(cm.data(), n), fr = pairs(rm.data(), m);
        if (ee == cudaSuccess) ee = cudaMemcpyAsync(d.mu1f, f1.data(), MN * F2, cudaMemcpyHostToDevice, st);
        if (ee == cudaSuccess) ee = cudaMemcpyAsync(d.mu2f, f2.data(), MN * F2, cudaMemcpyHostToDevice, st);
        if (ee == cudaSuccess) ee = cudaMemcpyAsync(d.cm2, fc.data(), n * F2, cudaMemcpyHostToDevice, st);
        if (ee == cudaSuccess) ee = cudaMemcpyAsync(d.rm2, fr.data(), m * F2, cudaMemcpyHostToDevice, st);
        // pageable sources: the copies are staged before cudaMemcpyAsync returns
    }
    if (ee == cudaSuccess) {
        launch_init(d, c.sigma, st);   // u = -sigma0 c (w0 = 0), delta and restart references 0
        ee = cudaGetLastError();
    }
    // the staging vectors above are pageable: cudaMemcpyAsync from pageable
    // memory returns after the copy is staged, so they may go out of scope.
    if (ee != cudaSuccess) {
        cudaFreeAsync(I->small, st);
        cudaFreeAsync(I->big, st);
        set_error(std::string("instance initialisation failed: ") + cudaGetErrorString(ee));
        return HOT_ECUDA;
    }
    *out = I.release();
    return HOT_OK;
}

void inst_destroy(Inst* I, cudaStream_t st) {
    if (!I) return;
    if (I->big) cudaFreeAsync(I->big, st);
    if (I->small) cudaFreeAsync(I->small, st);
    delete I;
}

// ------------------------------------------------------------------- batch --

Batch::~Batch() {
    if (graph) cudaGraphExecDestroy(graph);
    for (int p = 0; p < 2; ++p) {
        if (tgraph[p]) cudaGraphExecDestroy(tgraph[p]);
        for (int q = 0; q < 2; ++q)
            if (tev[p][q]) cudaEventDestroy(tev[p][q]);
    }
    if (cap_stream) cudaStreamDestroy(cap_stream);
    cudaFree(d_work);
    cudaFree(d_inst);
    cudaFree(d_pre);
    cudaFree(d_running);
    cudaFree(d_st);
    cudaFreeHost(h_work);
    cudaFreeHost(h_inst);
    cudaFreeHost(h_pre);
    cudaFreeHost(h_running);
    cudaFreeHost(h_st);
    cudaFreeHost(h_stb);
}

void Batch::drop_graphs() {
    if (graph) {
        cudaGraphExecDestroy(graph);
        graph = nullptr;
    }
    for (int p = 0; p < 2; ++p)
        if (tgraph[p]) {
            cudaGraphExecDestroy(tgraph[p]);
            tgraph[p] = nullptr;
        }
    single = -1;
    pad_captured = -1;
}

int Batch::reserve(int n) {
    if (n <= cap && d_work) return HOT_OK;
    int ncap = std::max(n, std::max(16, cap * 2));
    drop_graphs();   // the graphs captured the old table pointers
    cudaFree(d_work);
    cudaFree(d_inst);
    cudaFree(d_pre);
    cudaFree(d_running);
    cudaFree(d_st);
    cudaFreeHost(h_work);
    cudaFreeHost(h_inst);
    cudaFreeHost(h_pre);
    cudaFreeHost(h_running);
    cudaFreeHost(h_st);
    cudaFreeHost(h_stb);
    h_stb = nullptr;
    d_work = nullptr;
    HOT_CK(cudaMalloc(&d_work, sizeof(WorkDev)));
    HOT_CK(cudaMalloc(&d_inst, sizeof(HotInst) * ncap));
    HOT_CK(cudaMalloc(&d_pre, sizeof(int) * kPreTables * (ncap + 1)));
    HOT_CK(cudaMalloc(&d_running, sizeof(int)));
    HOT_CK(cudaMalloc(&d_st, sizeof(int) * ncap));
    HOT_CK(cudaMallocHost(&h_st, sizeof(int) * ncap));
    HOT_CK(cudaMallocHost(&h_stb, sizeof(int) * 2 * ncap));
    HOT_CK(cudaMallocHost(&h_work, sizeof(WorkDev)));
    HOT_CK(cudaMallocHost(&h_inst, sizeof(HotInst) * ncap));
    HOT_CK(cudaMallocHost(&h_pre, sizeof(int) * kPreTables * (ncap + 1)));
    HOT_CK(cudaMallocHost(&h_running, sizeof(int) * 4));
    cap = ncap;
    return HOT_OK;
}

int Batch::set_instances(const std::vector<Inst*>& v, cudaStream_t st) {
    int rc = reserve((int)v.size());
    if (rc != HOT_OK) return rc;
    // a single instance and a batch of several run different Prop. 3 kernels
    // (launch_solve_kernels), and padded slab rows a sweep variant of their
    // own: a change of either needs new graphs
    pad = 0;
    for (const Inst* I : v) pad |= (I->m % 4 != 0) || (I->n % 4 != 0) || I->desc.coord_real;
    if ((single >= 0 && single != (v.size() == 1 ? 1 : 0)) || (pad_captured >= 0 && pad_captured != pad))
        drop_graphs();
    // the pinned staging is rewritten here: wait for earlier copies out of it
    HOT_CK(cudaStreamSynchronize(st));
    const int n = (int)v.size();
    int* pt = h_pre;
    int* ps = h_pre + (cap + 1);
    int* pv = h_pre + 2 * (cap + 1);
    int* pk = h_pre + 3 * (cap + 1);
    int* pa = h_pre + 4 * (cap + 1);
    pt[0] = ps[0] = pv[0] = pk[0] = pa[0] = 0;
    int running = 0;
    size_t swept = 0;                 // bytes one sweep streams: u, d read, d written
    for (int i = 0; i < n; ++i) {
        h_inst[i] = v[i]->desc;
        swept += 3 * (v[i]->big_bytes / 5);
        const int m = v[i]->m, nn = v[i]->n;
        pt[i + 1] = pt[i] + nn * v[i]->nb1 + m * v[i]->nb2;
        ps[i + 1] = ps[i] + m + nn;
        pv[i + 1] = pv[i] + (v[i]->fp64 ? 2 * (m + nn) : vec32_items(m, nn));
        pk[i + 1] = pk[i] + v[i]->n_k1;
        pa[i + 1] = pa[i] + v[i]->desc.n_achunk;
        if (v[i]->ctl_host.status == ST_RUNNING) ++running;
    }
    // a state larger than L2: alternate the sweep's tile order, so that each
    // sweep starts on the tiles the previous one touched last (still in L2);
    // a state that fits gains nothing from it
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device) != cudaSuccess) l2 = 0;
    h_work->ninst = n;
    h_work->alternate = (l2 > 0 && swept > (size_t)l2) ? 1 : 0;
    h_work->inst = d_inst;
    h_work->pre_tile = d_pre;
    h_work->pre_slab = d_pre + (cap + 1);
    h_work->pre_vec = d_pre + 2 * (cap + 1);
    h_work->pre_k1 = d_pre + 3 * (cap + 1);
    h_work->pre_achunk = d_pre + 4 * (cap + 1);
    h_work->n_running = d_running;
    h_work->st_out = d_st;
    for (int i = 0; i < n; ++i) h_st[i] = v[i]->ctl_host.status;
    h_running[0] = running;
    if (n > 0) HOT_CK(cudaMemcpyAsync(d_inst, h_inst, sizeof(HotInst) * n, cudaMemcpyHostToDevice, st));
    HOT_CK(cudaMemcpyAsync(d_pre, h_pre, sizeof(int) * kPreTables * (cap + 1), cudaMemcpyHostToDevice, st));
    HOT_CK(cudaMemcpyAsync(d_work, h_work, sizeof(WorkDev), cudaMemcpyHostToDevice, st));
    HOT_CK(cudaMemcpyAsync(d_running, h_running, sizeof(int), cudaMemcpyHostToDevice, st));
    if (n > 0) HOT_CK(cudaMemcpyAsync(d_st, h_st, sizeof(int) * n, cudaMemcpyHostToDevice, st));
    ninst = n;
    return HOT_OK;
}

// One check block (K iterations plus the block end) captured into *out; with
// ev, an event pair recorded around the sweep of iteration timed_iter().
int Batch::capture(cudaGraphExec_t* out, cudaEvent_t* ev) {
    HOT_CK(cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal));
    for (int j = 0; j < K; ++j) {
        launch_solve_kernels(d_work, ld, fp64, j, j == K - 1, ninst == 1, cap_stream);
        const bool t = ev && j == timed_iter() && j < K - 1;
        if (t) cudaEventRecordWithFlags(ev[0], cap_stream, cudaEventRecordExternal);
        launch_sweep(d_work, ld, fp64, j, j == K - 1, pad != 0, cap_stream);
        if (t) cudaEventRecordWithFlags(ev[1], cap_stream, cudaEventRecordExternal);
    }
    launch_block_end(d_work, ld, fp64, K, a1, a2, a3, cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap_stream, &g);
    if (e != cudaSuccess) {
        set_error(std::string("graph capture failed: ") + cudaGetErrorString(e));
        return HOT_ECUDA;
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *out = nullptr;
        set_error(std::string("graph instantiation failed: ") + cudaGetErrorString(e));
        return HOT_ECUDA;
    }
    return HOT_OK;
}

int Batch::ensure_graph(int want_timing) {
    timing = want_timing && K >= 2 ? 1 : 0;
    if (timing ? (tgraph[0] && tgraph[1]) : graph != nullptr) return HOT_OK;
    if (!cap_stream) HOT_CK(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
    ld = make_launch_dims(device, fp64);
    single = ninst == 1 ? 1 : 0;
    pad_captured = pad;
    if (!timing) return capture(&graph, nullptr);
    for (int p = 0; p < 2; ++p) {
        for (int q = 0; q < 2; ++q)
            if (!tev[p][q]) HOT_CK(cudaEventCreate(&tev[p][q]));
        if (!tgraph[p]) {
            const int rc = capture(&tgraph[p], tev[p]);
            if (rc != HOT_OK) return rc;
        }
    }
    return HOT_OK;
}

int Batch::launch_block(cudaStream_t st, long long block) const {
    HOT_CK(cudaGraphLaunch(timing ? tgraph[block & 1] : graph, st));
    return HOT_OK;
}

// ------------------------------------------------------------------- solve --

void fill_result(const Inst* I, hot_result* r) {
    std::memset(r, 0, sizeof(*r));
    const HotCtl& c = I->ctl_host;
    r->ot_value = c.pobj;
    r->dual_value = c.dobj;
    r->rel_kkt = c.rel_kkt;
    r->rel_dual = c.rel_dual;
    r->rel_comp = c.rel_comp;
    r->rel_primal = c.rel_primal;
    r->abs_kkt = c.abs_kkt;
    r->sigma = c.sigma;
    r->cost_scale = I->cost_scale;
    r->iters = c.total;
    r->restarts = c.restarts;
    switch (c.status) {
        case ST_CONVERGED: r->status = HOT_OK; break;
        case ST_CAPPED: r->status = HOT_NOT_CONVERGED; break;
        case ST_NUMERIC: r->status = HOT_NUMERIC; break;
        case ST_CANCELLED: r->status = HOT_ECANCELLED; break;
        default: r->status = HOT_PENDING; break;
    }
    unsigned int yb = c.ymax_bits;
    float ym;
    std::memcpy(&ym, &yb, 4);
    r->max_abs_dual = ym;
    r->m = I->m;
    r->n = I->n;
}

int run_solve(Ctx* ctx, const std::vector<PairHost>& pairs, double tol, long long max_iter, bool keep,
              hot_result* out, hot_kernel_times* kt) {
    cudaStream_t st = ctx->stream;
    const int fp64 = ctx->cfg.precision == HOT_FP64 ? 1 : 0;
    if (!ctx->batch || ctx->batch->fp64 != fp64) {
        ctx->batch.reset(new Batch());
        Batch& b = *ctx->batch;
        b.device = ctx->device;
        b.fp64 = fp64;
        b.K = ctx->cfg.check_every;
        b.a1 = ctx->cfg.restart_sufficient;
        b.a2 = ctx->cfg.restart_necessary;
        b.a3 = ctx->cfg.restart_long;
    }
    Batch& B = *ctx->batch;
    std::vector<Inst*> insts;
    insts.reserve(pairs.size());
    auto cleanup = [&]() {
        for (Inst* I : insts) inst_destroy(I, st);
    };
    for (const PairHost& p : pairs) {
        Inst* I = nullptr;
        const int tr = ctx->tile_override ? ctx->tile_override : tuned_tile_rows(ctx, p.m, p.n, fp64);
        int rc = inst_create(p, fp64, ctx->cfg, tol, max_iter, tr, st, &I);
        if (rc != HOT_OK) {
            cleanup();
            return rc;
        }
        insts.push_back(I);
    }
    int rc = B.set_instances(insts, st);
    // live sweep timing: single-instance graph solves only (the bytes of a
    // timed launch are then those of the one instance)
    const int timing = ctx->sweep_timing && insts.size() == 1 && !kt ? 1 : 0;
    if (rc == HOT_OK) rc = B.ensure_graph(timing);   // also fixes the launch dimensions
    if (rc != HOT_OK) {
        cleanup();
        return rc;
    }
    cudaEvent_t t0, t1, ev[2];
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming);
    const long long K = B.K;
    const long long max_blocks = (max_iter + K - 1) / K + 2;
    long long nb = 0;
    int err = HOT_OK;
    // profiled mode: direct launches with an event pair around each kernel family
    std::vector<cudaEvent_t> pev;
    if (kt) {
        std::memset(kt, 0, sizeof(*kt));
        pev.resize(3 * K + 2);
        for (auto& e : pev) cudaEventCreate(&e);
    }
    // batches: the host time at which the block holding each instance's last
    // check was seen complete (its status copied back after every block)
    const bool track = insts.size() > 1 && !kt;
    std::vector<double> fin_ms(insts.size(), -1.0);
    // live[q]: the pair at position q of the work tables (batches drop their
    // finished pairs from the tables as they go, see below)
    std::vector<int> live(insts.size());
    for (size_t q = 0; q < insts.size(); ++q) live[q] = (int)q;
    long long launches = 0;
    const auto th0 = std::chrono::steady_clock::now();
    auto note_finished = [&](const int* sts) {
        const double now = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - th0).count();
        for (size_t q = 0; q < live.size(); ++q)
            if (fin_ms[live[q]] < 0.0 && sts[q] != ST_RUNNING) fin_ms[live[q]] = now;
    };
    cudaEventRecord(t0, st);
    for (;;) {
        if (!kt) {
            if (B.launch_block(st, nb) != HOT_OK) {
                err = HOT_ECUDA;
                break;
            }
            launches += launches_per_block(fp64, (int)K, B.ninst == 1) + kLaunchesBlockEnd;
            cudaMemcpyAsync(&B.h_running[1 + (nb & 1)], B.d_running, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (track)
                cudaMemcpyAsync(B.h_stb + (size_t)(nb & 1) * B.cap, B.d_st, sizeof(int) * live.size(),
                                cudaMemcpyDeviceToHost, st);
            cudaEventRecord(ev[nb & 1], st);
            if (nb >= 1) {
                cudaEventSynchronize(ev[(nb - 1) & 1]);
                if (track) note_finished(B.h_stb + (size_t)((nb - 1) & 1) * B.cap);
                // Tail of a batch: once at most a quarter of the table still
                // runs, rebuild the tables with the running pairs alone, so that
                // the kernels stop walking the finished pairs' items (and a last
                // pair runs the single-instance kernels).  Every pair keeps its
                // own state, so its iterates do not change.
                const int run_prev = B.h_running[1 + ((nb - 1) & 1)];
                if (track && live.size() > 1 && run_prev > 0 && (size_t)run_prev * 4 <= live.size()) {
                    cudaEventSynchronize(ev[nb & 1]);            // block nb and its status copy
                    const int* sts = B.h_stb + (size_t)(nb & 1) * B.cap;
                    note_finished(sts);
                    std::vector<Inst*> keep;
                    std::vector<int> keep_idx;
                    for (size_t q = 0; q < live.size(); ++q)
                        if (sts[q] == ST_RUNNING) {
                            keep.push_back(insts[live[q]]);
                            keep_idx.push_back(live[q]);
                        }
                    if (keep.empty()) {
                        ++nb;
                        break;
                    }
                    if (B.set_instances(keep, st) != HOT_OK || B.ensure_graph(0) != HOT_OK) {
                        err = HOT_ECUDA;
                        ++nb;
                        break;
                    }
                    live = keep_idx;
                    // block nb's statuses, now at the new positions (all running)
                    int* stn = B.h_stb + (size_t)(nb & 1) * B.cap;
                    for (size_t q = 0; q < live.size(); ++q) stn[q] = ST_RUNNING;
                    ++nb;
                    continue;
                }
                if (timing) {
                    // block nb - 1 has finished; block nb runs on the other graph instance
                    float tms = 0.f;
                    const int p = (int)((nb - 1) & 1);
                    if (cudaEventElapsedTime(&tms, B.tev[p][0], B.tev[p][1]) == cudaSuccess) {
                        const Inst* I0 = insts[0];
                        ctx->st_ms += tms;
                        ctx->st_launches += 1;
                        ctx->st_bytes += (double)I0->m * I0->n * (I0->m + I0->n) * (fp64 ? 24.0 : 12.0);
                    } else {
                        cudaGetLastError();
                    }
                }
                if (B.h_running[1 + ((nb - 1) & 1)] <= 0) {
                    ++nb;
                    break;
                }
            }
        } else {
            for (int j = 0; j < K; ++j) {
                cudaEventRecord(pev[3 * j], st);
                launch_solve_kernels(B.d_work, B.ld, fp64, j, j == K - 1, insts.size() == 1, st);
                cudaEventRecord(pev[3 * j + 1], st);
                launch_sweep(B.d_work, B.ld, fp64, j, j == K - 1, B.pad != 0, st);
                cudaEventRecord(pev[3 * j + 2], st);
            }
            launch_block_end(B.d_work, B.ld, fp64, (int)K, B.a1, B.a2, B.a3, st);
            cudaEventRecord(pev[3 * K], st);
            cudaMemcpyAsync(&B.h_running[1], B.d_running, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (cudaStreamSynchronize(st) != cudaSuccess) {
                err = HOT_ECUDA;
                break;
            }
            for (int j = 0; j < K; ++j) {
                float a = 0.f, b = 0.f;
                cudaEventElapsedTime(&a, pev[3 * j], pev[3 * j + 1]);
                cudaEventElapsedTime(&b, pev[3 * j + 1], pev[3 * j + 2]);
                kt->solve_ms += a;
                kt->solve_launches += launches_per_iteration(fp64, insts.size() == 1) - 1;
                if (j == K - 1) {
                    kt->sweep_check_ms += b;
                    kt->sweep_check_launches += 1;
                } else {
                    kt->sweep_ms += b;
                    kt->sweep_launches += 1;
                }
            }
            float c = 0.f;
            cudaEventElapsedTime(&c, pev[3 * K - 1], pev[3 * K]);
            kt->block_end_ms += c;
            kt->block_end_launches += kLaunchesBlockEnd;
            if (B.h_running[1] <= 0) {
                ++nb;
                break;
            }
        }
        ++nb;
        if (nb > max_blocks) break;   // every instance hits its cap before this
    }
    cudaEventRecord(t1, st);
    cudaError_t e = cudaStreamSynchronize(st);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    for (auto& ee : pev) cudaEventDestroy(ee);
    if (kt) {
        double vb = 0.0;
        for (Inst* I : insts) vb += (double)I->m * I->n * (I->m + I->n) * (fp64 ? 24.0 : 12.0);
        kt->sweep_bytes = vb;
    }
    if (e != cudaSuccess || err != HOT_OK) {
        set_error(std::string("solve failed on the device: ") + cudaGetErrorString(e != cudaSuccess ? e : cudaGetLastError()));
        cleanup();
        return HOT_ECUDA;
    }
    if (kt) launches = nb * (launches_per_block(fp64, (int)K, insts.size() == 1) + kLaunchesBlockEnd);
    for (size_t q = 0; q < insts.size(); ++q) {
        Inst* I = insts[q];
        cudaMemcpy(&I->ctl_host, I->desc.ctl, sizeof(HotCtl), cudaMemcpyDeviceToHost);
        fill_result(I, &out[q]);
        // a batch reports each instance's own completion (host-observed, from
        // the start of the batch); a single solve the device time of the solve
        out[q].solve_ms = track ? (fin_ms[q] >= 0.0 ? fin_ms[q] : (double)ms) : ms;
        out[q].kernel_launches = launches;
        out[q].blocks = nb;
        if (keep) {
            const unsigned long long id = ctx->next_id++;
            ctx->solutions[id].inst = I;
            out[q].solution_id = id;
        } else {
            inst_destroy(I, st);
        }
    }
    insts.clear();
    return HOT_OK;
}

}  // namespace hot
