// HOT iteration kernels for sm_103a (GB300).
//
// One iteration of Algorithm 2 (arXiv 2408.00598) on a batch of instances is
// three launches in FP32 bulk mode:
//   k_vec32   -- slab totals and cross-slab row sums of the state (inputs of
//                the marginals that Prop. 3 needs);
//   k_alpha32 -- Prop. 3: the right-hand side R of eq. (update:y) from the
//                slab sums, its closed-form solution y-bar, and the per-slab
//                broadcast vectors alpha/beta of A^T y-bar; elementwise over
//                the pieces, in chunks;
//   k_sweep   -- Steps 2-4 fused into one streaming pass over the flow state:
//                x-bar, z-bar = Pi_+(...), the Halpern update, and the slab
//                row/column sums of the new state (the A v products of the
//                next iteration); on check iterations also the KKT partial
//                sums of eq. (kkt_res).
// FP64 mode runs the same solve as k_vec, k_marg (instance-wide vectors, one
// CTA per instance) and k_alpha, in FP64.
// A block of K iterations ends with the KKT check, the restart rule, and the
// restart itself (new anchor), see launch_block_end.
//
// FP32 bulk mode stores the anchor u (= v0 - sigma g0) and the delta d in FP32
// and forms every element from small quantities (see hot_internal.h):
// g - v/sigma = -(dA) - (u + d)/sigma with dA = A^T(y-bar - y0), and
// x-bar = u + d + sigma dA.  The reduced cost g = c - A^T y-bar itself (needed
// where z-bar = 0, i.e. on the support of the plan, where it tends to 0) is an
// unevaluated float pair: A^T y-bar is split per slab row/column into a hi
// part on the exact grid 2^-E of the scaled cost, so c - alpha_hi - beta_hi is
// exact in FP32, plus an FP32 lo part.  FP64 arithmetic runs at a small
// fraction of the FP32 rate on this part, so the per-iteration sums and the
// Prop. 3 solve use double-float pairs (two FP32 values, about 48 bits);
// FP64 is left to once-per-cycle work (restart, anchor sums).
#include "hot_internal.h"
#include "hot_df.cuh"

#include <algorithm>
#include <cstdint>
#include <type_traits>

namespace hot {

// ---------------------------------------------------------------- helpers --

__device__ __forceinline__ int find_inst(const int* __restrict__ pre, int n, int t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh) {
    // deterministic: fixed shuffle tree, then warp partials summed in order
#pragma unroll
    for (int q = 0; q < NV; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) sh[q * 32 + warp] = v[q];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double x = lane < nw ? sh[q * 32 + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            v[q] = x;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) sh[q * 32] = v[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = sh[q * 32];
    __syncthreads();
}

__device__ __forceinline__ float block_max(float v, float* sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    float r = 0.f;
    if (threadIdx.x == 0)
        for (int q = 0; q < nw; ++q) r = fmaxf(r, sh[q]);
    __syncthreads();
    return r;  // valid in thread 0
}

__device__ __forceinline__ double sum_f64_strided(const double* p, int count, int stride) {
    double acc = 0.0;
    for (int q = 0; q < count; ++q) acc += p[q * stride];
    return acc;
}

// Column total over a slab's bands: init + p[0] + p[stride] + ... (nb terms,
// added left to right in band order), the loads issued four at a time so that
// nb bands cost about nb / 4 round trips instead of nb.
template <typename T>
__device__ __forceinline__ T sum_bands(const T* p, size_t stride, int nb, T init = T(0)) {
    T acc = init;
    for (int b0 = 0; b0 < nb; b0 += 4) {
        T v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = b0 + u < nb ? p[(size_t)(b0 + u) * stride] : T(0);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (b0 + u < nb) acc += v[u];
    }
    return acc;
}

// deterministic block sum of NV pairs; every thread receives the totals
template <int NV>
__device__ __forceinline__ void block_sum_df(DF (&v)[NV], float2* sh) {
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = warp_sum_df(v[q]);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) sh[q * 32 + warp] = df_st(v[q]);
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            DF x = lane < nw ? df_ld(sh[q * 32 + lane]) : DF{0.f, 0.f};
            x = warp_sum_df(x);
            if (lane == 0) sh[q * 32] = df_st(x);
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = df_ld(sh[q * 32]);
    __syncthreads();
}


// ------------------------------------------------------ per-tile parameters --

struct P64 {
    double is, s, rho, trs, h;
};

// Step 4 on the delta d = v - v0 of v = x + sigma z, with v-bar - v = sigma r:
//   Halpern (Algorithm 2): d' = rho_k d + 2 rho_k sigma r, rho_k = (k+1)/(k+2);
//   generalized ADMM:      d' = d + rho sigma r          (w' = (1-rho) w + rho w-bar).
// Both are d' = rho d + trs r.
__device__ __forceinline__ P32 make_p32(double sigma, int k, double h, int gadmm = 0, double relax = 1.0) {
    P32 p{};
    p.sih = (float)(1.0 / sigma);
    p.sf = (float)sigma;
    const double rho = gadmm ? 1.0 : (k + 1.0) / (k + 2.0);
    p.rho = (float)rho;
    p.trs = (float)(gadmm ? relax * sigma : 2.0 * rho * sigma);
    p.h = (float)h;
    return p;
}
__device__ __forceinline__ P64 make_p64(double sigma, int k, double h, int gadmm = 0, double relax = 1.0) {
    P64 p;
    p.is = 1.0 / sigma;
    p.s = sigma;
    p.rho = gadmm ? 1.0 : (k + 1.0) / (k + 2.0);
    p.trs = gadmm ? relax * sigma : 2.0 * p.rho * sigma;
    p.h = h;
    return p;
}

// (x_r - x_c)^2 of two FP32 coordinates as a pair (the difference exact by a
// two-sum, its square by fma), and a product with an FP32 value as a pair:
// the objective's parts in FP32 mode with real-valued coordinates.
__device__ __forceinline__ DF cost_pair(float xr, float xc) {
    const float d = xr - xc;
    const float bv = d - xr;
    const float de = (xr - (d - bv)) + (-xc - bv);          // two-sum error of xr + (-xc)
    const float c = d * d;
    return DF{c, fmaf(d, d, -c) + 2.f * d * de};
}
__device__ __forceinline__ DF cost_times(DF c, float v) {
    const float p = c.hi * v;
    return DF{p, fmaf(c.hi, v, -p) + c.lo * v};
}

// The reduced cost g = c - alpha_r - beta_c of an element as an unevaluated
// pair (Gh, Gl), from its row piece a and column piece b.  Integer
// coordinates: Gh = h (x_r - x_c)^2 - alpha_hi - beta_hi is exact on the grid
// 2^-E, Gl = -(alpha_lo + beta_lo).  Real coordinates (pieces P_r, Q_c as
// pairs): g = P_r + Q_c - 2 h x_r x_c by two exact two-sums and the product's
// fma error.
__device__ __forceinline__ void reduced_cost(const float4& a, const float4& b, float h, int coord_real, float& Gh,
                                             float& Gl) {
    const float m2hr = -2.f * h * a.w;                       // exact
    if (coord_real) {
        const float t = a.x + b.x;
        const float tb = t - a.x;
        const float te = (a.x - (t - tb)) + (b.x - tb);      // two-sum error of P_hi + Q_hi
        const float ph = m2hr * b.w;
        const float pe = fmaf(m2hr, b.w, -ph);               // exact error of the product
        Gh = t + ph;
        const float sb = Gh - t;
        const float se = (t - (Gh - sb)) + (ph - sb);        // two-sum error of t + ph
        Gl = se + ((te + pe) + (a.y + b.y));
    } else {
        Gh = fmaf(m2hr, b.w, fmaf(a.w * a.w, h, -a.x) + fmaf(b.w * b.w, h, -b.x));
        Gl = -(a.y + b.y);
    }
}

// Element math of Steps 2-3.  Inputs: anchor u, delta d, cost cq = (r-c)^2
// (unscaled integer), the slab row/column pieces of A^T y-bar (hi, lo) and of
// dA = A^T(y-bar - y0).  Outputs: w = g - v/sigma, mg = -g and
// r = z-bar - g = max(-g, g - v/sigma), the dual residual entry.
struct E32 {
    float Gh, Gl, D, s, w, mg, r;
};
__device__ __forceinline__ E32 elem32(float u, float d, float cq, const float4& a, const float4& b, const P32& p,
                                      int coord_real = 0) {
    E32 e;
    if (coord_real) {
        reduced_cost(a, b, p.h, 1, e.Gh, e.Gl);
    } else {
        e.Gh = fmaf(cq, p.h, -a.x) - b.x;   // exact: every term is on the grid 2^-E
        e.Gl = -(a.y + b.y);
    }
    e.D = a.z + b.z;                        // A^T (y-bar - y0)
    e.s = u + d;
    e.w = fmaf(-e.s, p.sih, -e.D);          // g - v/sigma
    e.mg = -(e.Gh + e.Gl);                  // -g
    e.r = fmaxf(e.w, e.mg);
    return e;
}
// x-bar = v - sigma g = u + d + sigma dA and z-bar = max(0, 2g - v/sigma).
__device__ __forceinline__ void xz32(const E32& e, const P32& p, float& xb, float& zb) {
    zb = (e.w > e.mg) ? ((e.Gh + e.Gl) + e.w) : 0.f;
    xb = fmaf(p.sf, e.D, e.s);
}

struct E64 {
    double g, D, s, w, r;
};
__device__ __forceinline__ E64 elem64(double u, double d, double cq, double a, double b, double da, double db,
                                      const P64& p) {
    E64 e;
    e.g = cq * p.h - a - b;
    e.D = da + db;
    e.s = u + d;
    e.w = -e.D - e.s * p.is;
    e.r = fmax(e.w, -e.g);
    return e;
}
__device__ __forceinline__ void xz64(const E64& e, const P64& p, double& xb, double& zb) {
    zb = (e.w > -e.g) ? (e.g + e.w) : 0.0;
    xb = e.s + p.s * e.D;
}

template <typename T> struct VecT;
template <> struct VecT<float> {
    using type = float4;
    static constexpr int N = 4;
    __device__ static void ld(const float* p, float (&x)[4]) {
        const float4 t = __ldcs(reinterpret_cast<const float4*>(p));
        x[0] = t.x; x[1] = t.y; x[2] = t.z; x[3] = t.w;
    }
    __device__ static void st(float* p, const float (&x)[4]) {
        __stcs(reinterpret_cast<float4*>(p), make_float4(x[0], x[1], x[2], x[3]));
    }
};
template <> struct VecT<double> {
    using type = double2;
    static constexpr int N = 2;
    __device__ static void ld(const double* p, double (&x)[2]) {
        const double2 t = __ldcs(reinterpret_cast<const double2*>(p));
        x[0] = t.x; x[1] = t.y;
    }
    __device__ static void st(double* p, const double (&x)[2]) {
        __stcs(reinterpret_cast<double2*>(p), make_double2(x[0], x[1]));
    }
};

// Asynchronous global -> shared copies (16 B per thread, cached in L2 only).
// A thread waits only for its own copies (cp.async.wait_group), so a pipeline
// in which every thread reads back only what it copied needs no barrier.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16_ef(void* smem, const void* gmem, unsigned long long pol) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "l"(pol) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Stages of the FP32 sweep pipeline: each holds one pass of P rows
// (one float4 of u and one of the delta per thread).
constexpr int kStages = 4;
constexpr int kStageBytes = 2 * kThreads * 16;
// k_sweep32 dynamic shared memory: the pass ring, plus on check iterations
// the x-bar row partials, column partials and per-warp row pairs
constexpr int kSweepSmem = kStages * kStageBytes;
constexpr int kSweepSmemChk = kSweepSmem + (kRowSmemBytes + 256 * 4) + kThreads * 4 * 4 + (kThreads / 32) * kMaxTR * 8;

struct TileCtx {
    int inst, slab, band;
};

// Resolve tile t of the batch; returns false (block-uniform) if the instance
// is not running.
__device__ __forceinline__ bool resolve_tile(const WorkDev* __restrict__ W, int t, TileCtx& tc, int* s_tile) {
    if (threadIdx.x == 0) {
        const int i = find_inst(W->pre_tile, W->ninst, t);
        s_tile[0] = i;
        s_tile[1] = t - W->pre_tile[i];
        s_tile[2] = W->inst[i].ctl->status;
        s_tile[3] = W->inst[i].ctl->restart_pending;
    }
    __syncthreads();
    tc.inst = s_tile[0];
    g_tile_slab(W->inst[tc.inst], s_tile[1], tc.slab, tc.band);
    return true;
}

// Programmatic dependent launch: the kernels of the iteration chain are
// launched with programmatic stream serialisation, so the launch of a kernel
// is prepared while its predecessor runs.  Each one first waits for the
// predecessor grid to complete and its memory to be visible (everything
// below then sees stream order).  No kernel triggers its successor early:
// CTAs placed ahead of time and left waiting cost more than they saved.
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// ----------------------------------------------------------------- k_vec --
// T1[j] = sum_k rowsum(f1 slab j)[k] (j < n), T2[k] = sum_j rowsum(f2 slab k)[j]
// (k < m), P1[k] = sum_j rowsum(f1 slab j)[k], P2[j] = sum_k rowsum(f2 slab k)[j];
// row sums are those of u + d (the slab sums of u are kept separately).  One
// warp per output; outputs at vecs[which * L + index], L = max(m, n).
__global__ void __launch_bounds__(kThreads) k_vec(const WorkDev* __restrict__ W) {
    pdl_enter();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ninst = W->ninst;
    const int nitems = W->pre_vec[ninst];
    for (int base = blockIdx.x * (kThreads / 32); base < nitems; base += gridDim.x * (kThreads / 32)) {
        const int item = base + warp;
        if (item >= nitems) continue;
        const int i = find_inst(W->pre_vec, ninst, item);
        const HotInst& I = W->inst[i];
        if (I.ctl->status != ST_RUNNING) continue;
        const int m = I.m, n = I.n, L = g_L(I);
        int q = item - W->pre_vec[i];
        int which;
        if (q < n) which = 0;
        else if ((q -= n) < m) which = 1;
        else if ((q -= m) < m) which = 2;
        else {
            q -= m;
            which = 3;
        }
        const double* __restrict__ rs = I.rs;
        const double* __restrict__ rs0 = I.rs0;
        const size_t f2 = (size_t)n * m;               // first row of the f2 half
        double acc = 0.0;
        if (which == 0) {                              // T1[j]: f1 slab j, its m rows
            for (int t = lane; t < m; t += 32) acc += rs[(size_t)q * m + t] + rs0[(size_t)q * m + t];
        } else if (which == 1) {                       // T2[k]: f2 slab k, its n rows
            for (int t = lane; t < n; t += 32) acc += rs[f2 + (size_t)q * n + t] + rs0[f2 + (size_t)q * n + t];
        } else if (which == 2) {                       // P1[k]: row k of every f1 slab
            for (int t = lane; t < n; t += 32) acc += rs[(size_t)t * m + q] + rs0[(size_t)t * m + q];
        } else {                                       // P2[j]: row j of every f2 slab
            for (int t = lane; t < m; t += 32) acc += rs[f2 + (size_t)t * n + q] + rs0[f2 + (size_t)t * n + q];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) I.vecs[which * L + q] = acc;
    }
}

// ---------------------------------------------------------- k_marg/k_alpha --
// Prop. 3 on R' = (b - A(u + d))/sigma, the right-hand side whose solution is
// dy = y-bar - y0: with v = sigma g0 + u + d, the right-hand side of
// eq. (update:y) is R = b/sigma - A(v/sigma - c) = AA^T y0 + R'.  R' comes
// from the slab sums of u + d.  With j < n and k < m:
//   a_j = sum_k R1(k,j), bb_j = sum_i R2(i,j), r3_k = sum_l R3(k,l), T3 = sum r3,
//   y1-hat(k,j) = (R1(k,j) + a_j/n - (1/m+1/n) bb_j + r3_k/n + T3/n^2)/(m+n),
//   s_k = sum_j y1-hat(k,j),  t = W-hat s,  y1^a = t + (1^T t / n) 1,
//   y1 = y1-hat - y1^a,  y2(i,j) = (R2(i,j) - sum_k y1(k,j))/m,
//   y3(k,l) = (R3(k,l) + sum_j y1(k,j))/n.
// k_marg (one CTA per instance) forms the O(m + n) vectors shared by all
// slabs, at mv[w * L + index], L = max(m, n):
//   w = 0: a_j / n - (1/m + 1/n) bb_j        (column part of y1-hat), j < n
//   w = 1: r3_k / n + T3 / n^2 - (m+n) y1^a_k (row part of y1, times m+n), k < m
//   w = 2: sum_k y1(k,j)                      (for y2), j < n
//   w = 3: sum_j y1(k,j)                      (for y3), k < m
// k_alpha (one CTA per slab) then forms the slab's entries with products only
// (FP64 division is slow on this part; reciprocals are taken once).
__global__ void __launch_bounds__(kThreads) k_marg(const WorkDev* __restrict__ W) {
    pdl_enter();
    extern __shared__ double sv[];                   // 7 L: T1 T2 P1 P2 colmu1 rowmu2, then s
    __shared__ double s_red[4 * 32];
    const int ninst = W->ninst;
    for (int inst = blockIdx.x; inst < ninst; inst += gridDim.x) {
        const HotInst& I = W->inst[inst];
        if (I.ctl->status != ST_RUNNING) continue;     // block-uniform
        const int mi = I.m, ni = I.n, L = g_L(I);
        const double m = mi, n = ni;
        const double is = 1.0 / I.ctl->sigma;
        const double in_ = 1.0 / n, im = 1.0 / m, imn = 1.0 / (m + n);
        double* T1 = sv;
        double* T2 = sv + L;
        double* P1 = sv + 2 * L;
        double* P2 = sv + 3 * L;
        double* cm = sv + 4 * L;
        double* rm = sv + 5 * L;
        double* ss = sv + 6 * L;
        for (int q = threadIdx.x; q < 4 * L; q += blockDim.x) sv[q] = I.vecs[q];
        for (int q = threadIdx.x; q < ni; q += blockDim.x) cm[q] = I.colmu1[q];
        for (int q = threadIdx.x; q < mi; q += blockDim.x) rm[q] = I.rowmu2[q];
        // the dropped (m, n) row of eq. (7): column n-1 of the last f2 slab
        const int sl = g_nslab(I) - 1;
        const double kap_last =
            sum_bands(I.cs_part + g_colp(I, sl, 0) + (ni - 1), (size_t)ni, I.nb2, I.kapa[g_row(I, sl) + (ni - 1)]);
        const double mu_last = I.mu2[(size_t)(mi - 1) * ni + (ni - 1)];
        __syncthreads();
        auto A_ = [&](int j) { return -(T1[j] - P2[j]) * is; };
        auto B_ = [&](int j) { return (cm[j] - T1[j]) * is; };
        auto R3_ = [&](int k) {
            double r = (rm[k] - T2[k]) * is;
            if (k == mi - 1) r -= (mu_last - kap_last) * is;
            return r;
        };
        double red[4] = {0.0, 0.0, 0.0, 0.0};
        for (int j = threadIdx.x; j < ni; j += blockDim.x) {
            red[0] += A_(j);
            red[1] += B_(j);
        }
        for (int k = threadIdx.x; k < mi; k += blockDim.x) red[2] += R3_(k);
        block_sum<4>(red, s_red);
        const double Asum = red[0], Bsum = red[1], T3 = red[2];
        const double dl = (1.0 - in_) / (m + 1.0);
        const double iw = 1.0 / (im - dl);             // 1/w, w = 1/m - (1-1/n)/(m+1)
        red[0] = red[1] = red[2] = red[3] = 0.0;
        for (int k = threadIdx.x; k < mi; k += blockDim.x) {
            const double rowR1 = -(P1[k] - T2[k]) * is;
            const double s = (rowR1 + Asum * in_ - (im + in_) * Bsum + R3_(k) + T3 * in_) * imn;   // s_k
            ss[k] = s;
            red[0] += (k == mi - 1 ? dl : im) * s;
        }
        block_sum<4>(red, s_red);
        const double ds = red[0];
        red[0] = red[1] = red[2] = red[3] = 0.0;
        for (int k = threadIdx.x; k < mi; k += blockDim.x) {
            const double dq = (k == mi - 1 ? dl : im);
            red[0] += -dq * ss[k] - dq * ds * iw;       // 1^T W-hat s
        }
        block_sum<4>(red, s_red);
        const double tsum = red[0];
        const double yasum = tsum + m * tsum * in_;    // 1^T y1^a over k < m
        double* mv = I.mvec;
        for (int k = threadIdx.x; k < mi; k += blockDim.x) {
            const double dq = (k == mi - 1 ? dl : im);
            const double ya = -dq * ss[k] - dq * ds * iw + tsum * in_;   // y1^a_k
            mv[L + k] = R3_(k) * in_ + T3 * in_ * in_ - (m + n) * ya;
            mv[3 * L + k] = ss[k] - n * ya;
        }
        for (int j = threadIdx.x; j < ni; j += blockDim.x) {
            const double aq = A_(j), bq = B_(j);
            mv[j] = aq * in_ - (im + in_) * bq;
            mv[2 * L + j] = (aq - bq + T3 * in_) * in_ - yasum;
        }
        __syncthreads();
    }
}

// Per-slab entries of dy = A^T-pieces of y-bar - y0.  The anchor part of R
// (row sums and column totals of u) is precomputed once per cycle by
// k_anchor; here only the delta's sums enter.
template <bool CHECK>
__global__ void __launch_bounds__(kThreads) k_alpha(const WorkDev* __restrict__ W) {
    pdl_enter();
    __shared__ double s_red[4 * 32];
    __shared__ float s_max[32];
    __shared__ int s_t[4];
    const int ninst = W->ninst;
    const int nslab = W->pre_slab[ninst];
    for (int t = blockIdx.x; t < nslab; t += gridDim.x) {
        if (threadIdx.x == 0) {
            const int i = find_inst(W->pre_slab, ninst, t);
            s_t[0] = i;
            s_t[1] = t - W->pre_slab[i];
            s_t[2] = W->inst[i].ctl->status;
        }
        __syncthreads();
        if (s_t[2] != ST_RUNNING) {
            __syncthreads();
            continue;
        }
        const HotInst& I = W->inst[s_t[0]];
        const int slab = s_t[1];
        const int mi = I.m, ni = I.n, L = g_L(I), Ls = g_side(I, slab), nb = g_nb(I, slab);
        const double m = mi, n = ni;
        const double is = 1.0 / I.ctl->sigma;
        const double im = 1.0 / m, in_ = 1.0 / n, imn = 1.0 / (m + n);
        const double* __restrict__ rs = I.rs;
        const double* __restrict__ mv = I.mvec;
        const double* __restrict__ R1a = I.R1a + g_row(I, slab);
        const double* __restrict__ kapa = I.kapa + g_row(I, slab);
        const size_t o = 2 * g_row(I, slab);
        const size_t f2 = (size_t)ni * mi;            // first row of the f2 half
        float ymax = 0.f;
        double dob = 0.0;
        // idx < Ls: alpha (row) entries, idx >= Ls: beta (column) entries; returns the full piece
        auto put = [&](int idx, double dv) -> double {
            I.dab64[o + idx] = dv;
            const double full = I.ab0[o + idx] + dv;
            I.ab64[o + idx] = full;
            if (CHECK) ymax = fmaxf(ymax, fabsf((float)full));
            return full;
        };
        auto kap_delta = [&](int c) -> double {           // column total of the delta over the bands
            double k = 0.0;
            k += sum_bands(I.cs_part + g_colp(I, slab, 0) + c, (size_t)Ls, nb);
            return k;
        };
        if (slab < ni) {
            const int j = slab;
            const double colj = mv[j];
            for (int k = threadIdx.x; k < mi; k += blockDim.x) {
                const double R1 = R1a[k] - (rs[(size_t)j * mi + k] - rs[f2 + (size_t)k * ni + j]) * is;
                put(k, (R1 + colj + mv[L + k]) * imn);        // y1(k, j)
            }
            const double sy = mv[2 * L + j];
            for (int i = threadIdx.x; i < mi; i += blockDim.x) {
                const double kap = kapa[i] + kap_delta(i);
                const double mu = I.mu1[(size_t)i * ni + j];
                const double full = put(Ls + i, ((mu - kap) * is - sy) * im);  // y2(i, j)
                if (CHECK) dob += mu * full;                                    // <b, y>: mu1 . y2
            }
        } else {
            const int k = slab - ni;
            const double rowk = mv[L + k];
            for (int j = threadIdx.x; j < ni; j += blockDim.x) {
                const double R1 = R1a[j] - (rs[(size_t)j * mi + k] - rs[f2 + (size_t)k * ni + j]) * is;
                put(j, -(R1 + mv[j] + rowk) * imn);            // -y1(k, j): A2 = -1_n^T kron I_M
            }
            const double sp = mv[3 * L + k];
            for (int l = threadIdx.x; l < ni; l += blockDim.x) {
                if (k == mi - 1 && l == ni - 1) {
                    put(Ls + l, 0.0);                          // no row: y3(m, n) = 0
                    continue;
                }
                const double kap = kapa[l] + kap_delta(l);
                const double mu = I.mu2[(size_t)k * ni + l];
                const double full = put(Ls + l, ((mu - kap) * is + sp) * in_); // y3(k, l)
                if (CHECK) dob += mu * full;                                    // mu2 . y3
            }
        }
        if (CHECK) {
            double red[4] = {dob, 0.0, 0.0, 0.0};
            block_sum<4>(red, s_red);
            const float bm = block_max(ymax, s_max);
            if (threadIdx.x == 0) {
                I.dobj_part[slab] = red[0];
                atomicMax(&I.ctl->ymax_bits, __float_as_uint(bm));
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------- k_vec32/k_alpha32 --
// FP32 bulk mode.  The same Prop. 3 solve as k_vec/k_marg/k_alpha, with the
// per-iteration arithmetic on double-float pairs: FP64 throughput on this
// part is a small fraction of FP32, and pairs carry about 48 bits, far more
// than the FP32 row and column partial sums they combine.
//
// k_vec32: T1, T2, P1, P2 of u + d.  A work item is one CTA: for T1/T2 (sums
// along contiguous rows) 8 outputs, one warp each; for P1/P2 (sums down the
// columns of the row-sum matrices) 32 columns x kVecRows rows, one column per
// lane and kVecRows / 8 rows per warp, combined in a fixed order into one
// partial per row block (k_alpha32 adds the partials).  Every lane issues
// its loads before it adds, so an item costs about one L2 round trip.
constexpr int kVecRows = 64;

// Pieces of A^T(y-bar - y0) in FP32 mode: per slab its row pieces (alpha),
// then its column pieces (beta), slab after slab as in ab32, 4mn per instance.
// The inputs of one piece, loaded in one round before any is computed:
//   row piece e of f1 slab j (k = e) or f2 slab k (j = e): the row sums of
//     u + d of f2 slab k row j (x) and of f1 slab j row k (y);
//   column piece e: the sigma-scaled anchor constant K2 (x), the column total
//     of the delta over the slab's bands (y.x) and on check iterations the
//     marginal entry (mu).
struct PieceIn {
    float2 a0;            // anchor piece (hi, lo)
    float2 x, y, mu;
    float2 s0, s1;        // the stage entries the piece uses (k_stage32): row pieces mvA_j, mvS_k; column pieces sy_j or sp_k
    float xc;             // bin coordinate of the piece's row or column
};
__device__ __forceinline__ void piece_slab(const HotInst& I, int q, int& slab, int& idx) {
    const int m = I.m, n = I.n;
    const int h1 = 2 * m * n;                     // pieces of the f1 half: n slabs of 2m
    if (q < h1) {
        slab = q / (2 * m);
        idx = q - slab * 2 * m;
    } else {
        const int r = q - h1, t = r / (2 * n);
        slab = n + t;
        idx = r - t * 2 * n;
    }
}
__device__ __forceinline__ PieceIn piece_in(const HotInst& I, int slab, int idx, bool check) {
    const int m = I.m, n = I.n;
    const bool f1 = slab < n;
    const int Ls = f1 ? m : n;
    PieceIn p;
    p.a0 = I.ab0_32[2 * g_row(I, slab) + idx];
    p.mu = make_float2(0.f, 0.f);
    p.xc = I.X32[g_xbase(I, slab) + (idx < Ls ? idx : idx - Ls)];
    const int L = g_L(I);
    const float2* __restrict__ sq = I.stg2;
    if (idx < Ls) {
        const float2* __restrict__ rs = I.rs2;
        const int j = f1 ? slab : idx, k = f1 ? idx : slab - n;
        p.x = rs[(size_t)n * m + (size_t)k * n + j];
        p.y = rs[(size_t)j * m + k];
        p.s0 = sq[j];                 // mvA_j
        p.s1 = sq[L + k];             // mvS_k
    } else {
        p.s0 = f1 ? sq[2 * L + slab] : sq[3 * L + slab - n];   // sy_j / sp_k
        p.s1 = make_float2(0.f, 0.f);
        const int e = idx - Ls, nb = f1 ? I.nb1 : I.nb2;
        p.x = I.K2[g_row(I, slab) + e];
        float kd = 0.f;
        kd += sum_bands(I.cs32 + g_colp(I, slab, 0) + e, (size_t)Ls, nb);
        p.y = make_float2(kd, 0.f);
        if (check) p.mu = f1 ? I.mu1f[(size_t)e * n + slab] : I.mu2f[(size_t)(slab - n) * n + e];
    }
    return p;
}

// Constants of the piece formula for the current cycle (from CycleK) and the
// cost grid 2^-E.
struct PieceK {
    DF is, imn, im, in, isim, isin;
    float grid, igrid;
};
__device__ __forceinline__ PieceK piece_consts(const HotInst& I) {
    const CycleK C = *I.cyc;
    PieceK K;
    K.is = df_ld(C.is);
    K.imn = df_ld(C.imn);
    K.im = df_ld(C.im);
    K.in = df_ld(C.in);
    K.isim = df_ld(C.isim);
    K.isin = df_ld(C.isin);
    K.igrid = (float)I.h;
    K.grid = 1.0f / K.igrid;                 // powers of two: exact
    return K;
}

// Piece idx of slab s of A^T(y-bar - y0) from its inputs and the stage sq of
// k_vec32 (Prop. 3): row pieces (idx < side) are y1(k, j) on f1 slab j row k
// and -y1(k, j) on f2 slab k row j, with
//   y1(k, j) = (R1(k, j) + mvA_j + mvS_k) / (m + n),
//   R1(k, j) = -(rowsum f1 slab j [k] - rowsum f2 slab k [j]) / sigma;
// column pieces are y2(i, j) on f1 slab j and y3(k, l) on f2 slab k (y3(m, n) = 0,
// the row dropped by eq. 7-8).  *zero is set for that last piece.
__device__ __forceinline__ DF piece_dv(const HotInst& I, const PieceK& K, int slab, int idx, const PieceIn& a,
                                      bool& zero) {
    const int m = I.m, n = I.n;
    const bool f1 = slab < n;
    const int Ls = f1 ? m : n;
    zero = false;
    if (idx < Ls) {
        const DF R1 = df_mul(df_sub(df_ld(a.x), df_ld(a.y)), K.is);
        const DF y1 = df_mul(df_add(df_add(R1, df_ld(a.s0)), df_ld(a.s1)), K.imn);
        return f1 ? y1 : df_neg(y1);
    }
    const int e = idx - Ls;
    zero = !f1 && slab == n + m - 1 && e == n - 1;
    if (zero) return DF{0.f, 0.f};
    const DF colc = f1 ? df_mul(df_ld(a.s0), df_neg(K.im)) : df_mul(df_ld(a.s0), K.in);
    const DF isc = f1 ? K.isim : K.isin;
    return df_add(df_sub(df_ld(a.x), df_mul(isc, a.y.x)), colc);
}

// The float4 the sweep reads for a piece: the full piece A^T y-bar = anchor +
// dv split into a part on the cost grid 2^-E (hi, so that c - hi_r - hi_c is
// exact in FP32) and an FP32 remainder, then dv itself, then the bin
// coordinate of the piece's row or column.  With real-valued coordinates
// (coord_real) the first two are instead the pair h x^2 - (anchor + dv), the
// piece's share of the separable cost h (x_r - x_c)^2 = h x_r^2 + h x_c^2 -
// 2 h x_r x_c less the piece itself (x^2 exact as a pair by fma; h a power of 2).
__device__ __forceinline__ float4 piece_pack(const PieceIn& a, DF dv, const PieceK& K, int coord_real) {
    const float df = df_f(dv);
    if (coord_real) {
        const float x2 = a.xc * a.xc;
        const DF hx2{x2 * K.igrid, fmaf(a.xc, a.xc, -x2) * K.igrid};
        const DF P = df_sub(hx2, df_add(DF{a.a0.x, a.a0.y}, dv));
        return make_float4(P.hi, P.lo, df, a.xc);
    }
    const float dh = rintf(df * K.grid) * K.igrid;
    return make_float4(a.a0.x + dh, a.a0.y + (df - dh), df, a.xc);
}


// The instance-wide O(m + n) stage of Prop. 3: from T1, T2, P1, P2 (k_vec32)
// the vectors
//   mvA_j = a_j/n - (1/m + 1/n) bb_j      (column part of y1-hat), j < n
//   mvS_k = r3_k/n + T3/n^2 - (m+n) y1a_k (row part of y1, times m+n), k < m
//   sy_j  = sum_k y1(k, j)                (for y2)
//   sp_k  = sum_j y1(k, j)                (for y3)
// into rows 0-3 of sq (mvA at j, mvS at k, sy at j, sp at k), with
//   a_j = (P2_j - T1_j)/sigma, bb_j = (colmu1_j - T1_j)/sigma,
//   r3_k = (rowmu2_k - T2_k)/sigma (less the dropped (m, n) entry's share at k = m-1),
//   e_k = (T2_k - P1_k)/sigma + r3_k,  s_k = (e_k + cst)/(m+n).
// Every global scalar is fixed by the two half totals F1 = sum_j T1_j = sum_k P1_k
// and F2 = sum_k T2_k = sum_j P2_j (the state summed over the f1 and f2 slabs)
// and the k = m-1 entries:
//   sum a = (F2 - F1)/sigma,  sum bb = (sum mu1 - F1)/sigma,
//   T3 = sum r3 = (sum mu2 - F2)/sigma - (dropped entry),
//   sum d_k e_k = (1/m) ((F2 - F1)/sigma + T3) + (d_last - 1/m) e_{m-1}
// (d the diagonal of W-hat: 1/m, ..., 1/m, d_last).  F1 and F2 come from the
// per-item totals of k_vec32's T items (one block reduction); every thread
// loads the k = m-1 entries itself, so the only barrier is that reduction's.
struct StageIn {
    DF T1, P2, cm;        // column quantities at j = q < n (P2 summed over its row blocks)
    DF T2, P1, rm;        // row quantities at k = q < m (P1 summed over its row blocks)
};
// sum of the row-block partials at column q of rows first, first + 1, ...
__device__ __forceinline__ DF sum_partials(const float2* __restrict__ v, int L, int first, int count, int q) {
    DF acc{0.f, 0.f};
    for (int b0 = 0; b0 < count; b0 += 4) {
        float2 pp[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            pp[u] = b0 + u < count ? __ldcg(v + (size_t)(first + b0 + u) * L + q) : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 4; ++u) acc = df_add(acc, df_ld(pp[u]));
    }
    return acc;
}
__device__ __forceinline__ StageIn stage_in(const HotInst& I, int q) {
    const int m = I.m, n = I.n, L = g_L(I);
    const float2* __restrict__ v = I.vec2;
    const int r1 = (n + kVecRows - 1) / kVecRows, r2 = (m + kVecRows - 1) / kVecRows;
    StageIn s{};
    if (q < n) {
        s.T1 = df_ld(__ldcg(v + q));
        s.P2 = sum_partials(v, L, 2 + r1, r2, q);
        s.cm = df_ld(I.cm2[q]);
    }
    if (q < m) {
        s.T2 = df_ld(__ldcg(v + L + q));
        s.P1 = sum_partials(v, L, 2, r1, q);
        s.rm = df_ld(I.rm2[q]);
    }
    return s;
}

// Every thread of the calling CTA takes part; the results are stored to sq
// (global) by the thread of each index.
__device__ void alpha32_stage(const HotInst& I, float2* __restrict__ sq, float2* s_red) {
    const int m = I.m, n = I.n, L = g_L(I);
    const CycleK C = *I.cyc;
    const float2* __restrict__ v = I.vec2;
    const int r1 = (n + kVecRows - 1) / kVecRows, r2 = (m + kVecRows - 1) / kVecRows;
    const int t1 = (n + 7) / 8, t2 = (m + 7) / 8;        // T items of k_vec32
    const float2* __restrict__ tp = v + (size_t)(2 + r1 + r2) * L;
    // F1, F2 from the T items' totals (t1 + t2 <= L <= 4 * kThreads)
    DF red[2] = {DF{0.f, 0.f}, DF{0.f, 0.f}};
    for (int q = threadIdx.x; q < t1 + t2; q += blockDim.x) {
        const DF x = df_ld(__ldcg(tp + q));
        if (q < t1) red[0] = df_add(red[0], x);
        else red[1] = df_add(red[1], x);
    }
    // the k = m-1 entries (every thread), and the entries of this thread's first index
    const StageIn last = stage_in(I, m - 1);
    const int sl = g_nslab(I) - 1;
    const float kdl = sum_bands(I.cs32 + g_colp(I, sl, 0) + (n - 1), (size_t)n, I.nb2);
    const StageIn own = stage_in(I, threadIdx.x);
    block_sum_df<2>(red, s_red);
    const DF F1 = red[0], F2 = red[1];
    const DF is = df_ld(C.is), im = df_ld(C.im), in = df_ld(C.in), imn = df_ld(C.imn), imin = df_ld(C.imin);
    const DF dl = df_ld(C.dl), sumd = df_ld(C.sumd), iw = df_ld(C.iw);
    // the dropped (m, n) row of eq. (7): column n-1 of the last f2 slab
    const DF drop = df_mul(df_add(df_ld(C.mk), -kdl), is);
    const DF dF = df_mul(df_sub(F2, F1), is);
    const DF suma = dF;
    const DF sumbb = df_mul(df_sub(df_from(I.sum_mu1), F1), is);
    const DF T3 = df_sub(df_mul(df_sub(df_from(I.sum_mu2), F2), is), drop);
    const DF R3l = df_sub(df_mul(df_sub(last.rm, last.T2), is), drop);
    const DF el = df_add(df_mul(df_sub(last.T2, last.P1), is), R3l);
    const DF sde = df_add(df_mul(df_add(dF, T3), im), df_mul(el, df_sub(dl, im)));     // sum d_k e_k
    const DF cst = df_add(df_sub(df_mul(suma, in), df_mul(sumbb, imin)), df_mul(T3, in));
    const DF ds = df_mul(df_add(sde, df_mul(cst, sumd)), imn);                          // sum d_k s_k
    const DF dsiw = df_mul(ds, iw);
    const DF tsum = df_neg(df_add(ds, df_mul(dsiw, sumd)));                            // 1^T W-hat s
    const DF tin = df_mul(tsum, in);
    const DF yasum = df_add(tsum, df_mul(tin, (float)m));                              // 1^T y1a over k < m
    const DF T3in = df_mul(T3, in);
    const DF T3in2 = df_mul(T3in, in);
    const float mpn = (float)(m + n);
    const int top = m > n ? m : n;
    for (int q = threadIdx.x; q < top; q += blockDim.x) {
        const StageIn s = q == (int)threadIdx.x ? own : stage_in(I, q);
        if (q < n) {
            const DF A = df_mul(df_sub(s.P2, s.T1), is);                                 // a_j
            const DF B = df_mul(df_sub(s.cm, s.T1), is);                                 // bb_j
            sq[0 * (size_t)L + q] = df_st(df_sub(df_mul(A, in), df_mul(B, imin)));                   // mvA_j
            sq[2 * (size_t)L + q] = df_st(df_sub(df_mul(df_add(df_sub(A, B), T3in), in), yasum));    // sy_j
        }
        if (q < m) {
            DF R3 = df_mul(df_sub(s.rm, s.T2), is);                                      // r3_k
            if (q == m - 1) R3 = df_sub(R3, drop);
            const DF e = df_add(df_mul(df_sub(s.T2, s.P1), is), R3);
            const DF sk = df_mul(df_add(e, cst), imn);                                   // s_k
            const DF ya = df_add(df_neg(df_mul(df_add(sk, dsiw), q == m - 1 ? dl : im)), tin);   // y1a_k
            sq[1 * (size_t)L + q] = df_st(df_sub(df_add(df_mul(R3, in), T3in2), df_mul(ya, mpn)));  // mvS_k
            sq[3 * (size_t)L + q] = df_st(df_sub(sk, df_mul(ya, (float)n)));                        // sp_k
        }
    }
}

// SINGLE (a batch of one instance): the CTA that finishes the instance's last
// item also forms its Prop. 3 stage (k_stage32's work), which saves a kernel
// on the single-instance path; batches of many instances launch k_stage32,
// since there every item would pay the count's atomic and barriers.
template <bool SINGLE>
__global__ void __launch_bounds__(kThreads) k_vec32(const WorkDev* __restrict__ W, int j) {
    pdl_enter();
    constexpr int kW = kThreads / 32;
    constexpr int kRW = kVecRows / kW;               // rows per warp in a P item
    __shared__ float2 s_p[kThreads];
    __shared__ float2 s_red[SINGLE ? 2 * 32 : 1];
    __shared__ int s_t[4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ninst = W->ninst;
    const int nitems = W->pre_vec[ninst];
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        if (threadIdx.x == 0) {
            const int i = find_inst(W->pre_vec, ninst, it);
            s_t[0] = i;
            s_t[1] = it - W->pre_vec[i];
            s_t[2] = W->inst[i].ctl->status;
        }
        __syncthreads();
        if (s_t[2] == ST_RUNNING) {
            const HotInst I = W->inst[s_t[0]];
            const int m = I.m, n = I.n, L = g_L(I);
            const int t1 = (n + 7) / 8, t2 = (m + 7) / 8;
            const int c1 = (m + 31) / 32, r1 = (n + kVecRows - 1) / kVecRows;   // P1: columns k, rows j
            const int c2 = (n + 31) / 32, r2 = (m + kVecRows - 1) / kVecRows;   // P2: columns j, rows k
            const size_t f2 = (size_t)n * m;                 // first row of the f2 half
            int item = s_t[1];
            const float2* __restrict__ rs = I.rs2;           // row sums of u + d
            if (item < t1 + t2) {
                // T1[j]: the m rows of f1 slab j; T2[k]: the n rows of f2 slab k
                const int which = item < t1 ? 0 : 1;
                const int q = (which ? item - t1 : item) * 8 + warp;
                const int cnt = which ? m : n, len = which ? n : m;
                if (q < cnt) {                                // warp-uniform
                    const float2* row = rs + (which ? f2 + (size_t)q * n : (size_t)q * m);
                    DF acc{0.f, 0.f};
                    for (int t0 = 0; t0 < len; t0 += 8 * 32) {
                        float2 v[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int t = t0 + u * 32 + lane;
                            v[u] = t < len ? row[t] : make_float2(0.f, 0.f);
                        }
#pragma unroll
                        for (int u = 0; u < 8; ++u) acc = df_add(acc, df_ld(v[u]));
                    }
                    acc = warp_sum_df(acc);
                    if (lane == 0) I.vec2[which * L + q] = df_st(acc);
                    if (lane == 0) s_p[warp] = df_st(acc);
                } else if (lane == 0) {
                    s_p[warp] = make_float2(0.f, 0.f);
                }
                // the item's total, for the half totals F1, F2 of the stage
                __syncthreads();
                if (threadIdx.x == 0) {
                    DF tot = df_ld(s_p[0]);
                    for (int w = 1; w < kW; ++w) tot = df_add(tot, df_ld(s_p[w]));
                    I.vec2[(size_t)(2 + r1 + r2) * L + item] = df_st(tot);
                }
            } else {
                item -= t1 + t2;
                // P1[k] = sum_j rs(f1 slab j)[k]; P2[j] = sum_k rs(f2 slab k)[j]:
                // 32 columns x kVecRows rows per item, one partial per row block
                const int which = item < c1 * r1 ? 0 : 1;
                if (which) item -= c1 * r1;
                const int ncol = which ? n : m, nrow = which ? m : n, nc = which ? c2 : c1;
                const int part = item / nc;
                const int q = (item - part * nc) * 32 + lane;
                const int t0 = part * kVecRows + warp * kRW;
                float2 v[kRW];
#pragma unroll
                for (int u = 0; u < kRW; ++u) {
                    const int t = t0 + u;
                    const size_t idx = which ? f2 + (size_t)t * n + q : (size_t)t * m + q;
                    v[u] = (q < ncol && t < nrow) ? rs[idx] : make_float2(0.f, 0.f);
                }
                DF acc{0.f, 0.f};
#pragma unroll
                for (int u = 0; u < kRW; ++u) acc = df_add(acc, df_ld(v[u]));
                s_p[threadIdx.x] = df_st(acc);
                __syncthreads();
                if (warp == 0 && q < ncol) {
                    DF tot = df_ld(s_p[lane]);
                    for (int w = 1; w < kW; ++w) tot = df_add(tot, df_ld(s_p[w * 32 + lane]));
                    I.vec2[(size_t)(2 + (which ? r1 : 0) + part) * L + q] = df_st(tot);
                }
            }
            if constexpr (SINGLE) {
                // The barrier orders this CTA's writes of the item before thread
                // 0's fence, which makes them visible device-wide before the
                // count (the pattern of a grid-wide barrier); the last CTA reads
                // the others' through L2 (__ldcg in stage_in).
                __syncthreads();
                if (threadIdx.x == 0) {
                    __threadfence();
                    const unsigned int done = atomicAdd(I.vcount, 1u) + 1u;
                    s_t[3] = done == (unsigned int)vec32_items_dev(m, n);
                    if (s_t[3]) __threadfence();
                }
                __syncthreads();
                if (s_t[3]) {
                    alpha32_stage(I, I.stg2, s_red);
                    if (threadIdx.x == 0) {
                        *I.vcount = 0u;                           // for the next launch
                        *I.p32 = make_p32(I.ctl->sigma, I.ctl->k + j, I.h, I.gadmm, I.relax);
                    }
                }
            }
        }
        __syncthreads();
    }
}

// k_stage32: the instance-wide Prop. 3 stage (alpha32_stage) from k_vec32's
// sums, one CTA per instance, and the element constants of the iteration.
// (A kernel of its own: forming it in the CTA that finishes an instance's
// last k_vec32 item cost every item an atomic and a barrier, which batches of
// many small instances paid many times over.)
__global__ void __launch_bounds__(kThreads) k_stage32(const WorkDev* __restrict__ W, int j) {
    pdl_enter();
    __shared__ float2 s_red[2 * 32];
    const int ninst = W->ninst;
    for (int i = blockIdx.x; i < ninst; i += gridDim.x) {
        const HotInst I = W->inst[i];
        if (I.ctl->status != ST_RUNNING) continue;   // block-uniform
        alpha32_stage(I, I.stg2, s_red);
        if (threadIdx.x == 0) *I.p32 = make_p32(I.ctl->sigma, I.ctl->k + j, I.h, I.gadmm, I.relax);
        __syncthreads();
    }
}

// k_alpha32: the pieces of y-bar - y0 (pairs, kept for the restart), their
// FP32 split for the sweep, and on check iterations the partial sums of
// <b, y>, of <c, A^T(y-bar - y0)> and max |A^T y|.  An instance's 4mn pieces
// are cut into chunks of kAlphaChunk (kAPT per thread, consecutive threads on
// consecutive pieces); a CTA takes chunks in a grid-stride loop and loads the
// inputs of all its pieces of a chunk before it computes any.  The
// instance-wide O(m + n) stage of Prop. 3 comes from k_stage32 (stg2), so a
// piece is a few loads and double-float operations.  The descriptor is copied
// into registers: the stores below cannot then force reloads of its fields.
// Per-chunk partial sums sit at the chunk's index (dobj_part, cD_part;
// k_check adds them in order).
template <bool CHECK>
__global__ void __launch_bounds__(kThreads, 2) k_alpha32(const WorkDev* __restrict__ W, int j) {
    pdl_enter();
    __shared__ float2 s_red[2 * 32];
    __shared__ float s_max[32];
    const int ninst = W->ninst;
    const int nchunk = W->pre_achunk[ninst];
    const int tid = threadIdx.x;
    for (int c = blockIdx.x; c < nchunk; c += gridDim.x) {
        // every thread resolves the chunk itself (uniform, no barrier)
        const int inst = find_inst(W->pre_achunk, ninst, c);
        const HotInst I = W->inst[inst];
        const int m = I.m, n = I.n;
        const int cl = c - W->pre_achunk[inst];
        const int npieces = 4 * m * n;
        // every input is loaded before the status is known (the instance's
        // memory is valid either way), so the chunk costs one round trip less
        int ps[kAPT], pi[kAPT];
        PieceIn pin[kAPT];
#pragma unroll
        for (int u = 0; u < kAPT; ++u) {
            const int q = cl * kAlphaChunk + u * kThreads + tid;
            ps[u] = -1;
            if (q < npieces) {
                piece_slab(I, q, ps[u], pi[u]);
                pin[u] = piece_in(I, ps[u], pi[u], CHECK);
            }
        }
        const PieceK K = piece_consts(I);
        if (I.ctl->status != ST_RUNNING) continue;
        float2* __restrict__ dab2 = I.dab2;
        float4* __restrict__ ab32 = I.ab32;
        float ymax = 0.f;
        DF dob{0.f, 0.f};
        // <c, A^T(y-bar - y0)>: the cost is separable, so a slab contributes
        // sum_r dalpha_r C(r) + sum_c dbeta_c C(c), C(x) = sum_y (X_x - X_y)^2
        DF cdd{0.f, 0.f};
#pragma unroll
        for (int u = 0; u < kAPT; ++u) {
            if (ps[u] < 0) continue;
            const int slab = ps[u], idx = pi[u];
            const int Ls = slab < n ? m : n;
            const PieceIn& a = pin[u];
            bool zero;
            const DF dv = piece_dv(I, K, slab, idx, a, zero);
            const bool col = idx >= Ls;
            const size_t o = 2 * g_row(I, slab) + idx;
            dab2[o] = df_st(dv);
            ab32[o] = piece_pack(a, dv, K, I.coord_real);
            if (CHECK) {
                const DF full = df_add(DF{a.a0.x, a.a0.y}, dv);
                ymax = fmaxf(ymax, fabsf(full.hi));
                const float2* csum = I.csum2 + g_xbase(I, slab);
                cdd = df_add(cdd, df_mul(dv, df_ld(csum[col ? idx - Ls : idx])));
                if (col && !zero) dob = df_add(dob, df_mul(df_ld(a.mu), full));
            }
        }
        if (CHECK) {
            DF red[2] = {dob, cdd};
            block_sum_df<2>(red, s_red);
            const float bm = block_max(ymax, s_max);
            if (tid == 0) {
                reinterpret_cast<float2*>(I.dobj_part)[cl] = df_st(red[0]);
                reinterpret_cast<float2*>(I.cD_part)[cl] = df_st(red[1]);
                atomicMax(&I.ctl->ymax_bits, __float_as_uint(bm));
            }
        }
    }
}

// Once per cycle (after a restart, and at the start): the anchor parts of the
// right-hand side, per slab: R1a along the slab's rows and the column totals
// of u.  One CTA per slab.
__device__ __forceinline__ void anchor_slab(const HotInst& I, int slab, double sigma) {
    const int mi = I.m, ni = I.n, Ls = g_side(I, slab), nb = g_nb(I, slab);
    const double is = 1.0 / sigma;
    const size_t f2 = (size_t)ni * mi;                // first row of the f2 half
    if (!I.fp64 && slab == 0 && threadIdx.x == 0) {
        const double m = mi, n = ni;
        const double dl = (1.0 - 1.0 / n) / (m + 1.0);
        CycleK& K = *I.cyc;
        K.is = df_st(df_from(is));
        K.in = df_st(df_from(1.0 / n));
        K.im = df_st(df_from(1.0 / m));
        K.imn = df_st(df_from(1.0 / (m + n)));
        K.imin = df_st(df_from(1.0 / m + 1.0 / n));
        K.iw = df_st(df_from(1.0 / (1.0 / m - dl)));       // 1/w, w = 1/m - (1-1/n)/(m+1)
        K.dl = df_st(df_from(dl));
        K.sumd = df_st(df_from((mi - 1) / m + dl));
        K.isim = df_st(df_from(is / m));
        K.isin = df_st(df_from(is / n));
    }
    const bool last = slab == g_nslab(I) - 1;
    const size_t ro = g_row(I, slab);
    for (int q = threadIdx.x; q < Ls; q += blockDim.x) {
        // f1 slab j: rows k, R1(k, j); f2 slab k: rows j, R1(k, j)
        const int j = slab < ni ? slab : q;
        const int k = slab < ni ? q : slab - ni;
        I.R1a[ro + q] = -(I.rs0[(size_t)j * mi + k] - I.rs0[f2 + (size_t)k * ni + j]) * is;
        double kap = 0.0;
        kap += sum_bands(I.cs0_part + g_colp(I, slab, 0) + q, (size_t)Ls, nb);
        I.kapa[ro + q] = kap;
        if (!I.fp64) {
            // pairs for the FP32-mode solve: the row sums of u (also those of
            // u + d, d = 0 at the anchor); K2 is the sigma-scaled anchor part
            // of y2 (f1 slab j, column i) resp. y3 (f2 slab k, column l)
            const float2 r0 = df_st(df_from(I.rs0[ro + q]));
            I.rs02[ro + q] = r0;
            I.rs2[ro + q] = r0;
            if (last && q == ni - 1) I.cyc->mk = df_st(df_from(I.mu2[(size_t)(mi - 1) * ni + (ni - 1)] - kap));
            double k2;
            if (slab < ni) k2 = (I.mu1[(size_t)q * ni + slab] - kap) * is / mi;
            else if (last && q == ni - 1) k2 = 0.0;
            else k2 = (I.mu2[(size_t)(slab - ni) * ni + q] - kap) * is / ni;
            I.K2[ro + q] = df_st(df_from(k2));
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_anchor(const WorkDev* __restrict__ W) {
    pdl_enter();
    __shared__ int s_t[4];
    const int ninst = W->ninst;
    const int nslab = W->pre_slab[ninst];
    int any = 0;
    for (int i = threadIdx.x; i < ninst; i += blockDim.x) {
        const HotCtl* C = W->inst[i].ctl;
        any |= (C->status == ST_RUNNING && C->restart_pending != 0);
    }
    if (!__syncthreads_or(any)) return;
    for (int t = blockIdx.x; t < nslab; t += gridDim.x) {
        if (threadIdx.x == 0) {
            const int i = find_inst(W->pre_slab, ninst, t);
            s_t[0] = i;
            s_t[1] = t - W->pre_slab[i];
            s_t[2] = (W->inst[i].ctl->status == ST_RUNNING) && W->inst[i].ctl->restart_pending;
        }
        __syncthreads();
        if (s_t[2]) anchor_slab(W->inst[s_t[0]], s_t[1], W->inst[s_t[0]].ctl->sigma);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads) k_anchor_one(HotInst I, double sigma) {
    for (int slab = blockIdx.x; slab < g_nslab(I); slab += gridDim.x) anchor_slab(I, slab, sigma);
}

// --------------------------------------------------------------- k_sweep --
// FP64 mode: Steps 2-4 of Algorithm 2 on one tile (TR rows of one slab) per
// loop trip.
__global__ void __launch_bounds__(kThreads, 2) k_sweep64(const WorkDev* __restrict__ W, int j, int check) {
    pdl_enter();
    constexpr int NV = 2;
    constexpr int kRowN = kRowSmemBytes / sizeof(double) + 256;
    __shared__ __align__(16) double s_row[kRowN];
    __shared__ __align__(16) double s_col[kThreads * NV];
    __shared__ __align__(16) double s_xrow[kRowN];
    __shared__ __align__(16) double s_xcol[kThreads * NV];
    __shared__ double s_red[kNK * 32];
    __shared__ int s_tile[4];
    __shared__ P64 s_p64;
    const int ninst = W->ninst;
    const int ntiles = W->pre_tile[ninst];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        TileCtx tc;
        resolve_tile(W, t, tc, s_tile);
        if (s_tile[2] != ST_RUNNING) {
            __syncthreads();
            continue;
        }
        const HotInst& I = W->inst[tc.inst];
        const int slab = tc.slab, band = tc.band;
        const int S = g_side(I, slab), Sp = g_pitch(I, slab), TR = I.TR;   // this slab's side and row pitch
        const int NC = Sp / NV;
        const int P = kThreads / NC;
        const int cg = threadIdx.x % NC, ro = threadIdx.x / NC;
        const bool active = ro < P;
        const int r0 = band * TR, r1 = min(S, r0 + TR);
        const size_t off = g_elem(I, slab);
        const double* __restrict__ u = (const double*)I.u + off;
        const double* __restrict__ din = (const double*)((j & 1) ? I.d1 : I.d0) + off;
        double* __restrict__ dout = (double*)((j & 1) ? I.d0 : I.d1) + off;
        if (threadIdx.x == 0) s_p64 = make_p64(I.ctl->sigma, I.ctl->k + j, I.h, I.gadmm, I.relax);
        __syncthreads();
        const int c0 = cg * NV;
        double cacc[NV], xacc[NV];
#pragma unroll
        for (int e = 0; e < NV; ++e) cacc[e] = xacc[e] = 0.0;
        double k64[kNK] = {0.0, 0.0, 0.0, 0.0, 0.0};
        const P64 p = s_p64;
        const double* ab = I.ab64 + 2 * g_row(I, slab);
        const double* dab = I.dab64 + 2 * g_row(I, slab);
        const double* X = I.X64 + g_xbase(I, slab);            // bin coordinates of this half
        double bb[NV], db[NV], cf[NV];
        const int nval = S - c0;                                // columns inside the slab (pad after)
#pragma unroll
        for (int e = 0; e < NV; ++e) {
            bb[e] = active && e < nval ? ab[S + c0 + e] : 0.0;
            db[e] = active && e < nval ? dab[S + c0 + e] : 0.0;
            cf[e] = active && e < nval ? X[c0 + e] : 0.0;
        }
        if (active) {
            for (int r = r0 + ro; r < r1; r += P) {
                const double a = ab[r], da = dab[r];
                const double rf = X[r];
                double uu[NV], dd[NV], out[NV], xo[NV];
                VecT<double>::ld(u + (size_t)r * Sp + c0, uu);
                VecT<double>::ld(din + (size_t)r * Sp + c0, dd);
#pragma unroll
                for (int e = 0; e < NV; ++e) {
                    const double dc = rf - cf[e];
                    const double cq = dc * dc;
                    const E64 el = elem64(uu[e], dd[e], cq, a, bb[e], da, db[e], p);
                    out[e] = p.rho * dd[e] + p.trs * el.r;
                    xo[e] = 0.0;
                    if (e >= nval) {
                        out[e] = 0.0;                               // pad columns stay 0
                        continue;
                    }
                    if (check) {
                        double xb, zb;
                        xz64(el, p, xb, zb);
                        xo[e] = xb;
                        const double mn = fmin(xb, zb);
                        k64[0] += el.r * el.r;
                        k64[1] += mn * mn;
                        k64[2] += xb * xb;
                        k64[3] += zb * zb;
                        k64[4] += cq * xb;
                        xacc[e] += xb;
                    }
                    cacc[e] += out[e];
                }
                VecT<double>::st(dout + (size_t)r * Sp + c0, out);
                s_row[(r - r0) * (NC + 1) + cg] = out[0] + out[1];
                if (check) s_xrow[(r - r0) * (NC + 1) + cg] = xo[0] + xo[1];
            }
        }
        __syncthreads();
        if (active) {
#pragma unroll
            for (int e = 0; e < NV; ++e) {
                s_col[ro * Sp + c0 + e] = cacc[e];
                if (check) s_xcol[ro * Sp + c0 + e] = xacc[e];
            }
        }
        __syncthreads();
        const size_t cbase = g_colp(I, slab, band);
        for (int c = threadIdx.x; c < S; c += blockDim.x) {
            I.cs_part[cbase + c] = sum_f64_strided(s_col + c, P, Sp);
            if (check) I.xcs_part[cbase + c] = sum_f64_strided(s_xcol + c, P, Sp);
        }
        for (int rr = threadIdx.x; rr < r1 - r0; rr += blockDim.x) {
            I.rs[g_row(I, slab) + r0 + rr] = sum_f64_strided(s_row + rr * (NC + 1), NC, 1);
            if (check) I.xrs[g_row(I, slab) + r0 + rr] = sum_f64_strided(s_xrow + rr * (NC + 1), NC, 1);
        }
        if (check) {
            block_sum<kNK>(k64, s_red);
            if (threadIdx.x == 0) {
                double* o = I.tile_kkt + (size_t)g_tile(I, slab, band) * kNK;
#pragma unroll
                for (int q = 0; q < kNK; ++q) o[q] = k64[q];
            }
        }
        __syncthreads();
    }
}

// -------------------------------------------------------------- k_sweep32 --
// FP32 bulk mode: Steps 2-4 of Algorithm 2 as one streaming pass over the
// flow state.  A CTA takes the tiles blockIdx.x, blockIdx.x + G, ... (TR rows
// of one slab each) and streams their passes (P rows: every thread one float4
// of u and one of the delta) through a kStages-deep cp.async ring that is not
// drained between tiles, so the next tile's loads are in flight while the
// current tile's row and column sums are reduced.  The rows' alpha pieces
// travel in the group of each tile's first pass into a ring of their own, and
// thread 0 leaves each tile's descriptor in a third ring for the compute side.
//
// The scaled cost is separable, h (x_r - x_c)^2 = h x_r^2 + h x_c^2 - 2 h x_r x_c
// (x the bin coordinates of the slab's half, integers in FP32 mode), so the
// grid part of the reduced cost is Gh = (A_r + B_c) - 2 h x_r x_c with
// A_r = h x_r^2 - alpha_hi (per row) and B_c = h x_c^2 - beta_hi (per column):
// every term is an integer multiple of 2^-E, so Gh is exact in FP32.  The
// coordinates travel in the w component of the alpha/beta pieces (k_alpha32),
// so the sweep reads no coordinate array.  A tile's offsets in the per-slab
// arrays are resolved once, by the issue side, into its descriptor.
// Zeros in place of a tile's delta: a tile spans TR * pitch <= kMaxTileElems
// floats (checked when the instance is created); zero-initialised at module load.
__device__ __align__(16) float g_zero_tile[kMaxTileElems];

struct TileD {
    int inst, slab, band, S, NC, P, r0, r1, npass;   // NC: column groups of the row pitch (S rounded up to 4)
    int row;          // g_row: first row entry of the slab
    int tile;         // g_tile: index of the tile within its instance
    int colp;         // g_colp: first column-partial entry of (slab, band)
    int dz;           // the delta read is zero (first iteration after an FP32 restart): no loads
    long long elem;   // g_elem: first flow variable of the slab
};

// Resolve tile t; npass = 0 marks a tile of an instance that is not running,
// or t past the end.  PAD = false: every side of the batch is a multiple of 4,
// so the pitch is the side.
template <bool PAD>
__device__ __forceinline__ TileD tile_desc(const WorkDev* __restrict__ W, int t, int ntiles, bool first) {
    TileD d{};
    if (t >= ntiles) return d;
    const int i = find_inst(W->pre_tile, W->ninst, t);
    const HotInst& I = W->inst[i];
    const int loc = t - W->pre_tile[i];
    d.inst = i;
    g_tile_slab(I, loc, d.slab, d.band);
    d.S = g_side(I, d.slab);
    d.NC = (PAD ? g_pitch(I, d.slab) : d.S) / 4;
    d.P = kThreads / d.NC;
    d.r0 = d.band * I.TR;
    d.r1 = min(d.S, d.r0 + I.TR);
    d.row = (int)g_row(I, d.slab);
    d.tile = g_tile(I, d.slab, d.band);
    d.colp = (int)g_colp(I, d.slab, d.band);
    d.elem = PAD ? (long long)g_elem(I, d.slab)
                 : (d.slab < I.n ? (long long)d.slab * I.m * I.m
                                 : (long long)I.n * I.m * I.m + (long long)(d.slab - I.n) * I.n * I.n);
    if (I.ctl->status == ST_RUNNING) d.npass = (d.r1 - d.r0 + d.P - 1) / d.P;
    if (first) d.dz = I.ctl->dzero;
    return d;
}

// PAD: some slab side of the batch is not a multiple of 4, so a thread's
// last column group may reach into the pad columns, which are masked (a
// variant of its own: the masks cost the unpadded sweep registers).
// FIRST (the first iteration of a block, never a check): a tile whose delta
// is known to be zero copies it from the zero tile (a variant of its own, so
// the other iterations' sweep carries none of it).
template <bool CHECK, bool PAD, bool FIRST = false>
__global__ void __launch_bounds__(kThreads, CHECK ? 2 : 3) k_sweep32(const WorkDev* __restrict__ W, int j) {
    pdl_enter();
    constexpr int NV = 4;
    constexpr int kW = kThreads / 32;
    constexpr int kRowN = kRowSmemBytes / sizeof(float) + 256;
    __shared__ __align__(16) float s_row[kRowN];
    __shared__ __align__(16) float s_col[kThreads * NV];
    __shared__ __align__(16) float4 s_alpha[kStages][kMaxTR];
    __shared__ __align__(16) float2 s_rdf[kW][kMaxTR];            // per-warp row partial pairs
    __shared__ TileD s_td[kStages];
    __shared__ float2 s_red[kNK * 32];
    // dynamic: the pass ring [kStages][2][kThreads] float4, then (check
    // iterations) the x-bar row and column partials
    extern __shared__ float4 s_stage[];
    float* s_xrow = reinterpret_cast<float*>(s_stage + kStages * 2 * kThreads);
    float* s_xcol = s_xrow + kRowN;
    float2 (*s_xdf)[kMaxTR] = reinterpret_cast<float2 (*)[kMaxTR]>(s_xcol + kThreads * NV);
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int G = gridDim.x;
    const int ntiles = W->pre_tile[W->ninst];

    // ---- issue side: every thread walks the same tile sequence
    struct Cur {
        const float* u;            // this thread's source of the next pass (u)
        const float* d;            // and of the delta
        const float4* a;           // alpha piece of this thread's row of the tile (tid < tile rows)
        int step;                  // P rows, in floats
        int mine;                  // passes of the tile left in which this thread copies a row
        int left, it, ik;          // passes left, tile, tiles started
        bool acopy;                // the next pass is the tile's first and this thread copies an alpha piece
    } c;
    // a state larger than L2: odd iterations take the tiles in reverse order,
    // so a sweep starts on the tiles whose state the previous sweep touched
    // last (still in L2)
    const bool rev = (j & 1) && W->alternate;
    auto set_tile = [&](int t) {
        TileD d = tile_desc<PAD>(W, rev && t < ntiles ? ntiles - 1 - t : t, ntiles, FIRST);
        while (t < ntiles && d.npass == 0) {
            t += G;
            d = tile_desc<PAD>(W, rev && t < ntiles ? ntiles - 1 - t : t, ntiles, FIRST);
        }
        c.it = t;
        if (t < ntiles) {
            const HotInst& I = W->inst[d.inst];
            const int ro = tid / d.NC, cg = tid - ro * d.NC;
            const int sp = PAD ? (d.S + 3) & ~3 : d.S;   // row pitch (without padded slabs, the side)
            const size_t base = (size_t)d.elem + ((size_t)d.r0 + ro) * sp + (size_t)cg * NV;
            c.u = (const float*)I.u + base;
            // a delta known to be zero (first iteration after an FP32 restart,
            // which stores none) is copied from a zero tile: L2 hits, no HBM read
            c.d = (FIRST && d.dz) ? g_zero_tile + ((size_t)ro * sp + (size_t)cg * NV)
                                  : (const float*)((j & 1) ? I.d1 : I.d0) + base;
            const int nr = d.r1 - d.r0;
            c.a = I.ab32 + 2 * (size_t)d.row + d.r0 + tid;
            c.step = d.P * sp;
            // rows ro, ro + P, ... below nr (threads past P rows copy nothing)
            c.mine = ro < d.P && ro < nr ? (nr - ro + d.P - 1) / d.P : 0;
            c.left = d.npass;
            c.acopy = tid < nr;
            if (tid == 0) s_td[c.ik % kStages] = d;
        }
    };
    c.ik = 0;
    unsigned long long pol_ef;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol_ef));
    set_tile(blockIdx.x);
    // one commit group per call: the copies of global pass n (ring slot n % kStages)
    auto issue = [&](int n) {
        if (c.it < ntiles) {
            if (c.mine > 0) {
                float4* su = s_stage + (size_t)(n % kStages) * 2 * kThreads + tid;
                cp_async16_ef(su, c.u, pol_ef);
                cp_async16_ef(su + kThreads, c.d, pol_ef);
                --c.mine;
            }
            if (c.acopy) {
                cp_async16(&s_alpha[c.ik % kStages][tid], c.a);
                c.acopy = false;
            }
            c.u += c.step;
            c.d += c.step;
            if (--c.left == 0) {
                ++c.ik;
                set_tile(c.it + G);
            }
        }
        cp_async_commit();
    };
#pragma unroll 1
    for (int q = 0; q < kStages - 1; ++q) issue(q);

    // ---- compute side
    // per column of this thread: B_c = h x_c^2 - beta_hi (exact), beta_lo,
    // dbeta, x_c; loaded for the next tile during the current tile's epilogue
    float4 bq[NV];
    P32 p;
    auto load_cols = [&](const TileD& d) {
        const HotInst& I = W->inst[d.inst];
        const int ro = tid / d.NC, c0 = (tid - ro * d.NC) * NV;
        p = *I.p32;
        const float4* ab = I.ab32 + 2 * (size_t)d.row + d.S;
#pragma unroll
        for (int e = 0; e < NV; ++e)
            bq[e] = ro < d.P && (!PAD || c0 + e < d.S) ? ab[c0 + e] : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    bool have = false;                           // bq, p hold the current tile's values
    int n = 0;                                   // global index of the next pass to compute
    for (int ck = 0;; ++ck) {
        // the tile's alpha pieces and its descriptor: group n (its first pass)
        // and thread 0's store, both complete before this barrier
        cp_async_wait<kStages - 2>();
        __syncthreads();
        // the issue side has started every tile this CTA still has (it runs ahead)
        if (c.it >= ntiles && ck >= c.ik) break;
        const TileD dc = s_td[ck % kStages];
        if (!have) load_cols(dc);
        const HotInst& I = W->inst[dc.inst];
        const int S = dc.S, Sp = PAD ? (dc.S + 3) & ~3 : dc.S, NC = dc.NC, P = dc.P;
        const int r0 = dc.r0, nr = dc.r1 - dc.r0;
        const int ro = tid / NC, cg = tid - ro * NC;
        const bool active = ro < P;
        const int c0 = cg * NV;
        const int nval = PAD ? S - c0 : NV;       // columns of this thread's group inside the slab (pad after)
        const int cr = PAD ? I.coord_real : 0;    // real-valued coordinates (general variant only)
        const float h = p.h;
        if (!cr) {
#pragma unroll
            for (int e = 0; e < NV; ++e) {
                const float cf = bq[e].w;                      // column coordinate x_c
                bq[e] = make_float4(fmaf(cf * cf, h, -bq[e].x), bq[e].y, bq[e].z, cf);
            }
        }
        const float4* sa = s_alpha[ck % kStages];
        float* __restrict__ dout = (float*)((j & 1) ? I.d0 : I.d1) + dc.elem + ((size_t)r0 + ro) * Sp + c0;
        const int ostep = P * Sp;
        float* srow = s_row + ro * (NC + 1) + cg;
        float* sxrow = s_xrow + (CHECK ? ro * (NC + 1) + cg : 0);
        const int rstep = P * (NC + 1);
        float cacc[NV], xacc[NV];
#pragma unroll
        for (int e = 0; e < NV; ++e) cacc[e] = xacc[e] = 0.f;
        // KKT partials: FP32 chains of at most 64 terms per thread and tile
        // (a tile has TR * S / 1024 <= 16 passes), summed over the CTA in pairs.
        // The objective's share <c, d> is not formed here: it only reports the
        // value, so the pass that ends an instance forms it once (MODE 2)
        float k32[kNK - 1] = {0.f, 0.f, 0.f, 0.f};
        int rr = ro;                              // this thread's row, relative to r0
#pragma unroll 1
        for (int q = 0; q < dc.npass; ++q, ++n) {
            issue(n + kStages - 1);
            cp_async_wait<kStages - 1>();         // this thread's pass-n copies are in
            if (active && rr < nr) {
                const float4* su = s_stage + (size_t)(n % kStages) * 2 * kThreads + tid;
                const float4 U = su[0], D = su[kThreads];
                const float uu[NV] = {U.x, U.y, U.z, U.w};
                const float dd[NV] = {D.x, D.y, D.z, D.w};
                const float4 a = sa[rr];
                const float rf = a.w;                         // row coordinate x_r
                const float Ar = fmaf(rf * rf, h, -a.x);      // h x_r^2 - alpha_hi (exact)
                const float m2hr = -2.f * h * rf;             // exact
                float out[NV], xo[NV];
#pragma unroll
                for (int e = 0; e < NV; ++e) {
                    const float4 b = bq[e];
                    float Gh, Gl;
                    if (PAD && cr) {
                        reduced_cost(a, b, h, 1, Gh, Gl);          // pieces h x^2 - alpha, h x^2 - beta as pairs
                    } else {
                        Gh = fmaf(m2hr, b.w, Ar + b.x);            // h (x_r-x_c)^2 - alpha_hi - beta_hi
                        Gl = -(a.y + b.y);
                    }
                    const float Dv = a.z + b.z;                  // A^T (y-bar - y0)
                    const float s = uu[e] + dd[e];
                    const float w = fmaf(-s, p.sih, -Dv);        // g - v/sigma
                    const float mg = -(Gh + Gl);                 // -g
                    const float r = fmaxf(w, mg);                // z-bar - g
                    out[e] = !PAD || e < nval ? fmaf(p.trs, r, p.rho * dd[e]) : 0.f;   // pad columns stay 0
                    if constexpr (CHECK) {
                        xo[e] = 0.f;
                        if (!PAD || e < nval) {
                            const float zb = (w > mg) ? ((Gh + Gl) + w) : 0.f;
                            const float xb = fmaf(p.sf, Dv, s);
                            xo[e] = xb;
                            const float mn = fminf(xb, zb);
                            k32[0] = fmaf(r, r, k32[0]);
                            k32[1] = fmaf(mn, mn, k32[1]);
                            k32[2] = fmaf(xb, xb, k32[2]);
                            k32[3] = fmaf(zb, zb, k32[3]);
                            xacc[e] += xb;
                        }
                    }
                    cacc[e] += out[e];
                }
                __stcs(reinterpret_cast<float4*>(dout), make_float4(out[0], out[1], out[2], out[3]));
                *srow = (out[0] + out[1]) + (out[2] + out[3]);
                if constexpr (CHECK) *sxrow = (xo[0] + xo[1]) + (xo[2] + xo[3]);
            }
            dout += ostep;
            srow += rstep;
            if constexpr (CHECK) sxrow += rstep;
            rr += P;
        }
        // ---- tile epilogue: column and row sums as double-float pairs
        if (active) {
            *reinterpret_cast<float4*>(&s_col[ro * Sp + c0]) = make_float4(cacc[0], cacc[1], cacc[2], cacc[3]);
            if constexpr (CHECK)
                *reinterpret_cast<float4*>(&s_xcol[ro * Sp + c0]) = make_float4(xacc[0], xacc[1], xacc[2], xacc[3]);
        }
        __syncthreads();
        // the next tile's column values (thread 0 stored its descriptor while
        // issuing its first pass, before this barrier); the loads complete
        // under the reductions below
        have = !(c.it >= ntiles && ck + 1 >= c.ik);
        if (have) load_cols(s_td[(ck + 1) % kStages]);
        const size_t cbase = dc.colp;
        for (int cc = tid; cc < S; cc += kThreads) {
            DF a{0.f, 0.f}, x{0.f, 0.f};
            for (int qq = 0; qq < P; ++qq) {
                a = df_add(a, s_col[qq * Sp + cc]);
                if constexpr (CHECK) x = df_add(x, s_xcol[qq * Sp + cc]);
            }
            I.cs32[cbase + cc] = df_f(a);
            if constexpr (CHECK) I.xcs_part[cbase + cc] = df_val(x);
        }
        // rows: warp w sums partials [w NC/8, (w+1) NC/8) of rows lane, lane + 32, ...
        // (row stride NC + 1 keeps the lanes on distinct banks), then the 8
        // pairs of each row are combined in warp order
        {
            const int w0 = (warp * NC) / kW, w1 = ((warp + 1) * NC) / kW;
            for (int r = lane; r < nr; r += 32) {
                DF a{0.f, 0.f}, x{0.f, 0.f};
                for (int cc = w0; cc < w1; ++cc) {
                    a = df_add(a, s_row[r * (NC + 1) + cc]);
                    if constexpr (CHECK) x = df_add(x, s_xrow[r * (NC + 1) + cc]);
                }
                s_rdf[warp][r] = df_st(a);
                if constexpr (CHECK) s_xdf[warp][r] = df_st(x);
            }
        }
        if constexpr (CHECK) {
            DF kd[kNK - 1];
#pragma unroll
            for (int qq = 0; qq < kNK - 1; ++qq) kd[qq] = DF{k32[qq], 0.f};
            block_sum_df<kNK - 1>(kd, s_red);    // its barriers also publish s_rdf
            if (tid == 0) {
                float2* o = reinterpret_cast<float2*>(I.tile_kkt) + (size_t)dc.tile * kNK;
#pragma unroll
                for (int qq = 0; qq < kNK - 1; ++qq) o[qq] = df_st(kd[qq]);
            }
        } else {
            __syncthreads();
        }
        for (int r = tid; r < nr; r += kThreads) {
            DF a = df_ld(s_rdf[0][r]), x{0.f, 0.f};
            if constexpr (CHECK) x = df_ld(s_xdf[0][r]);
#pragma unroll
            for (int w = 1; w < kW; ++w) {
                a = df_add(a, df_ld(s_rdf[w][r]));
                if constexpr (CHECK) x = df_add(x, df_ld(s_xdf[w][r]));
            }
            a = df_add(a, df_ld(I.rs02[dc.row + r0 + r]));      // + row sum of u
            I.rs2[dc.row + r0 + r] = df_st(a);
            if constexpr (CHECK) I.xrs[dc.row + r0 + r] = df_val(x);
        }
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------- restart tiles --
// MODE 0: partial ||x-bar - x_r||^2, ||z-bar - z_r||^2 of the check iteration.
// MODE 1: restart at the check iteration: anchor and iterate <- w-bar, i.e.
//         v0 = x-bar + sigma_new z-bar and y0 = y-bar, stored as
//         u = v0 - sigma_new g-bar = x-bar + sigma_new r (r = z-bar - g-bar);
//         (x_r, z_r) = (x-bar, z-bar); delta = 0; FP64 slab sums of u;
//         A^T y0 pieces <- those of y-bar.
// MODE 2: x-bar of the final check iteration into x_r (the solution), and
//         (FP32 mode) the tile's share of <c, d> of that iteration, which
//         completes the reported objective (k_block_end).
// The check iteration (index K-1, odd) read delta buffer d1.
template <typename T, int MODE>
__device__ __forceinline__ void restart_tile(const HotInst& I, int slab, int band, double* s_row, double* s_col,
                                             double* s_red) {
    using V = VecT<T>;
    constexpr int NV = V::N;
    constexpr bool F32 = std::is_same<T, float>::value;
    const int S = g_side(I, slab), Sp = g_pitch(I, slab), TR = I.TR;   // this slab's side and row pitch
    const int NC = Sp / NV;
    const int P = kThreads / NC;
    const int cg = threadIdx.x % NC, ro = threadIdx.x / NC;
    const bool active = ro < P;
    const int r0 = band * TR, r1 = min(S, r0 + TR);
    const size_t off = g_elem(I, slab);
    T* u = (T*)I.u + off;
    const T* d1 = (const T*)I.d1 + off;
    T* d0 = (T*)I.d0 + off;
    T* xr = (T*)I.xr + off;
    T* zr = (T*)I.zr + off;
    // x-bar, z-bar need the check iteration's sigma; MODE 1 runs after
    // k_restart_sigma has replaced it (kept in sigma_old)
    const double sig_old = (MODE == 1) ? I.ctl->sigma_old : I.ctl->sigma;
    const double sig_new = I.ctl->sigma;
    const int c0 = cg * NV;
    const int nval = S - c0;                         // columns inside the slab (pad columns after)
    const int cr = F32 ? I.coord_real : 0;           // real-valued coordinates: the cost term in pairs
    const int xb0 = g_xbase(I, slab);                // bin coordinates of this slab's half
    // sums that feed later iterations: FP64 (FP64 mode) or double-float (FP32 mode)
    double racc[2] = {0.0, 0.0};
    DF fr[2] = {DF{0.f, 0.f}, DF{0.f, 0.f}};
    double ccol[NV];
    DF fcol[NV];
#pragma unroll
    for (int e = 0; e < NV; ++e) {
        ccol[e] = 0.0;
        fcol[e] = DF{0.f, 0.f};
    }
    if (active) {
        // loop invariants of the tile, read once: the check iteration's
        // constants, this thread's column pieces and column coordinates, and
        // the arrays behind restrict-qualified locals (the stores below then
        // force no reloads of the descriptor)
        const P32 p32 = make_p32(sig_old, 0, I.h);
        const P64 p64 = make_p64(sig_old, 0, I.h);
        const float4* __restrict__ ab32 = F32 ? I.ab32 + 2 * g_row(I, slab) : nullptr;
        const double* __restrict__ ab64 = F32 ? nullptr : I.ab64 + 2 * g_row(I, slab);
        const double* __restrict__ dab64 = F32 ? nullptr : I.dab64 + 2 * g_row(I, slab);
        const float* __restrict__ X32 = I.X32 + xb0;
        const double* __restrict__ X64 = I.X64 + xb0;
        float4 bq[NV];
        T xc[NV], bb[NV], db[NV];
#pragma unroll
        for (int e = 0; e < NV; ++e) {
            const bool v = e < nval;
            if constexpr (F32) {
                bq[e] = v ? ab32[S + c0 + e] : make_float4(0.f, 0.f, 0.f, 0.f);
                xc[e] = v ? X32[c0 + e] : 0.f;
            } else {
                bb[e] = v ? ab64[S + c0 + e] : 0.0;
                db[e] = v ? dab64[S + c0 + e] : 0.0;
                xc[e] = v ? X64[c0 + e] : 0.0;
            }
        }
        const float fsig = (float)sig_new;
        // two rows in flight per thread: the pass streams 16-24 B per variable
        // and needs the loads of several rows outstanding to reach HBM speed
#pragma unroll 2
        for (int r = r0 + ro; r < r1; r += P) {
            T uu[NV], dd[NV], xbv[NV], zbv[NV], rv[NV];
            V::ld(u + (size_t)r * Sp + c0, uu);
            V::ld(d1 + (size_t)r * Sp + c0, dd);
            if constexpr (F32) {
                const float4 a = ab32[r];
                const float xrow = X32[r];
#pragma unroll
                for (int e = 0; e < NV; ++e) {
                    const float dc = xrow - xc[e];
                    const E32 el = elem32(uu[e], dd[e], dc * dc, a, bq[e], p32, cr);
                    xz32(el, p32, xbv[e], zbv[e]);
                    rv[e] = el.r;
                }
            } else {
                const double a = ab64[r], da = dab64[r];
                const double xrow = X64[r];
#pragma unroll
                for (int e = 0; e < NV; ++e) {
                    const double dc = xrow - xc[e];
                    const E64 el = elem64(uu[e], dd[e], dc * dc, a, bb[e], da, db[e], p64);
                    xz64(el, p64, xbv[e], zbv[e]);
                    rv[e] = el.r;
                }
            }
#pragma unroll
            for (int e = 0; e < NV; ++e)
                if (e >= nval) xbv[e] = zbv[e] = rv[e] = T(0);   // pad columns: zero in every array
            if constexpr (MODE == 0) {
                T xo[NV], zo[NV];
                V::ld(xr + (size_t)r * Sp + c0, xo);
                V::ld(zr + (size_t)r * Sp + c0, zo);
#pragma unroll
                for (int e = 0; e < NV; ++e) {
                    if constexpr (F32) {
                        // (a - b)^2 exactly as a pair: the difference is exact to
                        // rounding, its square split by fma
                        const float dx = xbv[e] - xo[e], dz = zbv[e] - zo[e];
                        const float px = dx * dx, pz = dz * dz;
                        fr[0] = df_add(fr[0], DF{px, fmaf(dx, dx, -px)});
                        fr[1] = df_add(fr[1], DF{pz, fmaf(dz, dz, -pz)});
                    } else {
                        const double dx = xbv[e] - xo[e], dz = zbv[e] - zo[e];
                        racc[0] += dx * dx;
                        racc[1] += dz * dz;
                    }
                }
            } else if constexpr (MODE == 1) {
                // the slab sums of u enter every later right-hand side of Prop. 3,
                // where they cancel against b: FP64-level accuracy is needed
                T nu_[NV], zero[NV];
                DF rsf{0.f, 0.f};
                double rsd = 0.0;
                (void)rsd;
#pragma unroll
                for (int e = 0; e < NV; ++e) {
                    if constexpr (F32) nu_[e] = fmaf(fsig, rv[e], xbv[e]);
                    else nu_[e] = xbv[e] + sig_new * rv[e];
                    zero[e] = T(0);
                    if constexpr (F32) {
                        rsf = df_add(rsf, (float)nu_[e]);
                        fcol[e] = df_add(fcol[e], (float)nu_[e]);
                        // <c, u>: (r-c)^2 u exactly as a pair (the integer cost is exact in FP32)
                        if (cr) {
                            fr[0] = df_add(fr[0], cost_times(cost_pair(X32[r], xc[e]), (float)nu_[e]));
                        } else {
                            const float dc = X32[r] - xc[e], cq = dc * dc;
                            const float p = cq * (float)nu_[e];
                            fr[0] = df_add(fr[0], DF{p, fmaf(cq, (float)nu_[e], -p)});
                        }
                    } else {
                        rsd += nu_[e];
                        ccol[e] += nu_[e];
                    }
                }
                V::st(u + (size_t)r * Sp + c0, nu_);
                V::st(xr + (size_t)r * Sp + c0, xbv);
                V::st(zr + (size_t)r * Sp + c0, zbv);
                if constexpr (!F32) V::st(d0 + (size_t)r * Sp + c0, zero);   // FP32: dzero instead
                if constexpr (F32) reinterpret_cast<float2*>(s_row)[(r - r0) * NC + cg] = df_st(rsf);
                else s_row[(r - r0) * NC + cg] = rsd;
            } else {
                V::st(xr + (size_t)r * Sp + c0, xbv);
                if constexpr (F32) {
                    // <c, d> of the final check iteration: (r-c)^2 d exactly as a pair
                    // (real-valued coordinates: the cost itself as a pair)
#pragma unroll
                    for (int e = 0; e < NV; ++e) {
                        if (e >= nval) continue;
                        if (cr) {
                            fr[0] = df_add(fr[0], cost_times(cost_pair(X32[r], xc[e]), (float)dd[e]));
                        } else {
                            const float dc = X32[r] - xc[e], cq = dc * dc;
                            const float pd = cq * (float)dd[e];
                            fr[0] = df_add(fr[0], DF{pd, fmaf(cq, (float)dd[e], -pd)});
                        }
                    }
                }
            }
        }
    }
    // FP32 mode: the tile's sums as double-float pairs (GB300 runs FP64 at a
    // small fraction of the FP32 rate); FP64 mode: FP64
    if constexpr (MODE == 0) {
        if constexpr (F32) {
            block_sum_df<2>(fr, reinterpret_cast<float2*>(s_red));
            if (threadIdx.x == 0) {
                float2* o = reinterpret_cast<float2*>(I.rst_part) + (size_t)g_tile(I, slab, band) * 2;
                o[0] = df_st(fr[0]);
                o[1] = df_st(fr[1]);
            }
        } else {
            block_sum<2>(racc, s_red);
            if (threadIdx.x == 0) {
                double* o = I.rst_part + (size_t)g_tile(I, slab, band) * 2;
                o[0] = racc[0];
                o[1] = racc[1];
            }
        }
    } else if constexpr (MODE == 2) {
        if constexpr (F32) {
            DF cd[1] = {fr[0]};                           // <c, d> of this thread's share
            block_sum_df<1>(cd, reinterpret_cast<float2*>(s_red));
            if (threadIdx.x == 0)
                reinterpret_cast<float2*>(I.tile_kkt)[(size_t)g_tile(I, slab, band) * kNK + kNK - 1] = df_st(cd[0]);
        }
    } else if constexpr (MODE == 1) {
        if constexpr (F32) {
            DF cu[1] = {fr[0]};                           // <c, u> of this thread's share
            block_sum_df<1>(cu, reinterpret_cast<float2*>(s_red));
            if (threadIdx.x == 0) reinterpret_cast<float2*>(I.cu_part)[g_tile(I, slab, band)] = df_st(cu[0]);
        }
        __syncthreads();
        if (active)
#pragma unroll
            for (int e = 0; e < NV; ++e) {
                if constexpr (F32) reinterpret_cast<float2*>(s_col)[ro * Sp + c0 + e] = df_st(fcol[e]);
                else s_col[ro * Sp + c0 + e] = ccol[e];
            }
        __syncthreads();
        const size_t cbase = g_colp(I, slab, band);
        for (int c = threadIdx.x; c < S; c += blockDim.x) {
            if constexpr (F32) {
                const float2* sc = reinterpret_cast<const float2*>(s_col) + c;
                DF a{0.f, 0.f};
                for (int q = 0; q < P; ++q) a = df_add(a, df_ld(sc[(size_t)q * Sp]));
                I.cs0_part[cbase + c] = df_val(a);
            } else {
                I.cs0_part[cbase + c] = sum_f64_strided(s_col + c, P, Sp);
            }
            I.cs_part[cbase + c] = 0.0;
            I.cs32[cbase + c] = 0.f;
        }
        // y0 <- y-bar: A^T y0 pieces of this tile's rows (and, for band 0, columns)
        const size_t o = 2 * g_row(I, slab);
        const double ih = 1.0 / I.h;                         // a power of two: exact
        auto set_anchor = [&](int idx) {
            const double a0 = I.ab0[o + idx] + (F32 ? df_val(df_ld(I.dab2[o + idx])) : I.dab64[o + idx]);
            I.ab0[o + idx] = a0;
            if (I.ab0_32) {
                // integer coordinates: hi on the grid 2^-E (the reduced cost is then
                // exact in FP32); real ones form it in pairs and take a plain
                // double-float split, whose lo part keeps 2^-24 of hi, not of 2^-E
                const double hi = I.coord_real ? (double)(float)a0 : rint(a0 * ih) * I.h;
                I.ab0_32[o + idx] = make_float2((float)hi, (float)(a0 - hi));
            }
        };
        for (int rr = threadIdx.x; rr < r1 - r0; rr += blockDim.x) {
            if constexpr (F32) {
                const float2* sr = reinterpret_cast<const float2*>(s_row) + (size_t)rr * NC;
                DF a{0.f, 0.f};
                for (int q = 0; q < NC; ++q) a = df_add(a, df_ld(sr[q]));
                I.rs0[g_row(I, slab) + r0 + rr] = df_val(a);
            } else {
                I.rs0[g_row(I, slab) + r0 + rr] = sum_f64_strided(s_row + rr * NC, NC, 1);
            }
            if (!F32) I.rs[g_row(I, slab) + r0 + rr] = 0.0;      // FP32: k_anchor resets rs2
            set_anchor(r0 + rr);
        }
        if (band == 0)
            for (int c = threadIdx.x; c < S; c += blockDim.x) set_anchor(S + c);
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads, 3) k_restart(const WorkDev* __restrict__ W) {
    pdl_enter();
    __shared__ double s_row[MODE == 1 ? kRowSmemBytes / 8 * 2 : 1];
    __shared__ double s_col[MODE == 1 ? kThreads * 4 : 1];
    __shared__ double s_red[2 * 32];
    __shared__ int s_tile[4];
    const int ninst = W->ninst;
    const int ntiles = W->pre_tile[ninst];
    // most blocks end without a restart: leave at once unless some instance needs this pass
    int any = 0;
    for (int i = threadIdx.x; i < ninst; i += blockDim.x) {
        const HotCtl* C = W->inst[i].ctl;
        any |= (MODE == 2) ? (C->just_finished != 0) : (C->status == ST_RUNNING && C->restart_pending != 0);
    }
    if (!__syncthreads_or(any)) return;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        TileCtx tc;
        resolve_tile(W, t, tc, s_tile);
        const HotInst& I = W->inst[tc.inst];
        bool go;
        if (MODE == 2) go = I.ctl->just_finished != 0;
        else go = (s_tile[2] == ST_RUNNING) && (s_tile[3] != 0);
        if (go) restart_tile<T, MODE>(I, tc.slab, tc.band, s_row, s_col, s_red);
        __syncthreads();
    }
}

// Initial point w0 = 0 of a new instance: v0 = 0 and y0 = 0, so
// u = v0 - sigma0 (c - A^T y0) = -sigma0 c; d = 0; x_r = z_r = 0; FP64 slab
// sums of u.  One launch per instance (descriptor by value).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_init(HotInst I, double sigma0) {
    using V = VecT<T>;
    constexpr int NV = V::N;
    __shared__ double s_row[kRowSmemBytes / 8 * 2];
    __shared__ double s_col[kThreads * 4];
    __shared__ double s_red[32];
    const int TR = I.TR;
    for (int t = blockIdx.x; t < g_ntiles(I); t += gridDim.x) {
        int slab, band;
        g_tile_slab(I, t, slab, band);
        const int S = g_side(I, slab), Sp = g_pitch(I, slab);   // this slab's side and row pitch
        const int NC = Sp / NV;
        const int P = kThreads / NC;
        const int cg = threadIdx.x % NC, ro = threadIdx.x / NC;
        const bool active = ro < P;
        const int c0 = cg * NV;
        const int r0 = band * TR, r1 = min(S, r0 + TR);
        const size_t off = g_elem(I, slab);
        DF cuf{0.f, 0.f};
        double ccol[NV];
        DF fcol[NV];
#pragma unroll
        for (int e = 0; e < NV; ++e) {
            ccol[e] = 0.0;
            fcol[e] = DF{0.f, 0.f};
        }
        if (active) {
            for (int r = r0 + ro; r < r1; r += P) {
                T uu[NV], zero[NV];
                DF rsf{0.f, 0.f};
                double rs = 0.0;
#pragma unroll
                for (int e = 0; e < NV; ++e) {
                    const int xb0 = g_xbase(I, slab);
                    const bool v = c0 + e < S;                 // pad columns: 0
                    const double dc = v ? I.X64[xb0 + r] - I.X64[xb0 + c0 + e] : 0.0;
                    uu[e] = v ? (T)(-sigma0 * (dc * dc * I.h)) : T(0);
                    zero[e] = T(0);
                    if constexpr (std::is_same<T, float>::value) {
                        rsf = df_add(rsf, (float)uu[e]);
                        fcol[e] = df_add(fcol[e], (float)uu[e]);
                        if (I.coord_real) {                                     // <c, u> with the FP32 positions
                            const float* X32 = I.X32 + xb0;
                            if (v) cuf = df_add(cuf, cost_times(cost_pair(X32[r], X32[c0 + e]), (float)uu[e]));
                        } else {
                            const float cq = (float)(dc * dc), p = cq * (float)uu[e];
                            cuf = df_add(cuf, DF{p, fmaf(cq, (float)uu[e], -p)});   // <c, u>
                        }
                    } else {
                        rs += (double)uu[e];
                        ccol[e] += (double)uu[e];
                    }
                }
                if constexpr (std::is_same<T, float>::value) rs = df_val(rsf);
                V::st((T*)I.u + off + (size_t)r * Sp + c0, uu);
                V::st((T*)I.d0 + off + (size_t)r * Sp + c0, zero);
                V::st((T*)I.xr + off + (size_t)r * Sp + c0, zero);
                V::st((T*)I.zr + off + (size_t)r * Sp + c0, zero);
                s_row[(r - r0) * NC + cg] = rs;
            }
        }
        if constexpr (std::is_same<T, float>::value)
#pragma unroll
            for (int e = 0; e < NV; ++e) ccol[e] = df_val(fcol[e]);
        __syncthreads();
        if (active)
#pragma unroll
            for (int e = 0; e < NV; ++e) s_col[ro * Sp + c0 + e] = ccol[e];
        __syncthreads();
        const size_t cbase = g_colp(I, slab, band);
        for (int c = threadIdx.x; c < S; c += blockDim.x) I.cs0_part[cbase + c] = sum_f64_strided(s_col + c, P, Sp);
        for (int rr = threadIdx.x; rr < r1 - r0; rr += blockDim.x)
            I.rs0[g_row(I, slab) + r0 + rr] = sum_f64_strided(s_row + rr * NC, NC, 1);
        if constexpr (std::is_same<T, float>::value) {
            DF cu[1] = {cuf};
            block_sum_df<1>(cu, reinterpret_cast<float2*>(s_red));
            if (threadIdx.x == 0) reinterpret_cast<float2*>(I.cu_part)[g_tile(I, slab, band)] = df_st(cu[0]);
        }
        __syncthreads();
    }
}

// --------------------------------------------------------------- k_kkt1 --
// Partial sums of ||A x-bar - b||^2 from the x-bar slab sums.  F32 (FP32 bulk
// mode): the partials are double-float pairs, like every per-block partial of
// that mode (tile KKT sums, <c, u>, <b, y>, the restart norms): GB300 runs FP64
// at a small fraction of the FP32 rate, and FP64 block reductions dominated
// these small kernels.  FP64 mode keeps FP64 throughout.
template <bool F32>
__global__ void __launch_bounds__(kThreads) k_kkt1(const WorkDev* __restrict__ W) {
    pdl_enter();
    __shared__ double s_red[32];
    __shared__ int s_t[3];
    const int ninst = W->ninst;
    const int nchunks = W->pre_k1[ninst];
    for (int t = blockIdx.x; t < nchunks; t += gridDim.x) {
        if (threadIdx.x == 0) {
            const int i = find_inst(W->pre_k1, ninst, t);
            s_t[0] = i;
            s_t[1] = t - W->pre_k1[i];
            s_t[2] = W->inst[i].ctl->status;
        }
        __syncthreads();
        if (s_t[2] != ST_RUNNING) {
            __syncthreads();
            continue;
        }
        const HotInst& I = W->inst[s_t[0]];
        const int m = I.m, n = I.n;
        const int MN = m * n;
        const int q = s_t[1] * kThreads + threadIdx.x;
        double res = 0.0;
        if (q < 3 * MN - 1) {
            if (q < MN) {                                  // conservation rows (k, j)
                const int j = q / m, k = q % m;
                res = I.xrs[(size_t)j * m + k] - I.xrs[(size_t)MN + (size_t)k * n + j];
            } else if (q < 2 * MN) {                       // mu1 rows (i, j)
                const int j = (q - MN) / m, i = (q - MN) % m;
                double kap = 0.0;
                kap += sum_bands(I.xcs_part + g_colp(I, j, 0) + i, (size_t)m, I.nb1);
                res = kap - I.mu1[(size_t)i * n + j];
            } else {                                       // mu2 rows (k, l), the last one dropped
                const int k = (q - 2 * MN) / n, l = (q - 2 * MN) % n;
                double kap = 0.0;
                kap += sum_bands(I.xcs_part + g_colp(I, n + k, 0) + l, (size_t)n, I.nb2);
                res = kap - I.mu2[(size_t)k * n + l];
            }
        }
        if constexpr (F32) {
            const DF r = df_from(res);
            DF v[1] = {df_mul(r, r)};
            block_sum_df<1>(v, reinterpret_cast<float2*>(s_red));
            if (threadIdx.x == 0) reinterpret_cast<float2*>(I.k1_part)[s_t[1]] = df_st(v[0]);
        } else {
            double v[1] = {res * res};
            block_sum<1>(v, s_red);
            if (threadIdx.x == 0) I.k1_part[s_t[1]] = v[0];
        }
        __syncthreads();
    }
}

// Sum of count pairs p[0], p[stride], ... of this thread's share (q = threadIdx.x,
// q + blockDim.x, ...), the loads issued four at a time.
__device__ __forceinline__ DF sum_pairs(const float2* __restrict__ p, int count, int stride) {
    DF acc{0.f, 0.f};
    for (int q0 = threadIdx.x; q0 < count; q0 += 4 * blockDim.x) {
        float2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = q0 + u * blockDim.x;
            v[u] = q < count ? p[(size_t)q * stride] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) acc = df_add(acc, df_ld(v[u]));
    }
    return acc;
}

// --------------------------------------------------------------- k_check --
// Stopping rule eq. (kkt_res) and the restart rule, one CTA per instance.
template <bool F32>
__global__ void __launch_bounds__(kThreads) k_check(const WorkDev* __restrict__ W, int K, double a1, double a2,
                                                    double a3) {
    pdl_enter();
    __shared__ double s_red[8 * 32];
    const int ninst = W->ninst;
    for (int i = blockIdx.x; i < ninst; i += gridDim.x) {
        const HotInst& I = W->inst[i];
        HotCtl* C = I.ctl;
        if (C->status != ST_RUNNING) continue;   // block-uniform
        const int ntile = g_ntiles(I), nslab = g_nslab(I);
        double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if constexpr (F32) {
            // pairs: the check sweep's per-tile KKT sums, <c, u> per tile, the
            // ||A x - b||^2 chunks and k_alpha32's <b, y> and <c, A^T(y-bar - y0)>
            // per chunk (the objective's <c, d> share is added when the
            // instance ends: only the reported value needs it)
            // (every load of a round is issued before the adds: the sums cost
            // a few round trips, not one per array)
            const float2* tk = reinterpret_cast<const float2*>(I.tile_kkt);
            const float2* cu = reinterpret_cast<const float2*>(I.cu_part);
            DF w[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) w[e] = DF{0.f, 0.f};
            for (int q0 = threadIdx.x; q0 < ntile; q0 += 4 * blockDim.x) {
                float2 t[4][kNK + 1];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int q = q0 + u * blockDim.x;
#pragma unroll
                    for (int e = 0; e < kNK - 1; ++e) t[u][e] = q < ntile ? tk[(size_t)q * kNK + e] : make_float2(0.f, 0.f);
                    t[u][kNK - 1] = make_float2(0.f, 0.f);
                    t[u][kNK] = q < ntile ? cu[q] : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
#pragma unroll
                    for (int e = 0; e < kNK; ++e) w[e] = df_add(w[e], df_ld(t[u][e]));
                    w[7] = df_add(w[7], df_ld(t[u][kNK]));
                }
            }
            w[5] = sum_pairs(reinterpret_cast<const float2*>(I.k1_part), I.n_k1, 1);
            w[6] = sum_pairs(reinterpret_cast<const float2*>(I.dobj_part), I.n_achunk, 1);
            const DF cD = sum_pairs(reinterpret_cast<const float2*>(I.cD_part), I.n_achunk, 1);
            w[4] = df_add(w[4], df_mul(cD, df_from(C->sigma)));
            block_sum_df<8>(w, reinterpret_cast<float2*>(s_red));
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = df_val(w[e]);
        } else {
            for (int q = threadIdx.x; q < ntile; q += blockDim.x)
                for (int e = 0; e < kNK; ++e) v[e] += I.tile_kkt[(size_t)q * kNK + e];
            for (int q = threadIdx.x; q < I.n_k1; q += blockDim.x) v[5] += I.k1_part[q];
            // partial sums of <b, y>: one per slab
            for (int q = threadIdx.x; q < nslab; q += blockDim.x) v[6] += I.dobj_part[q];
            block_sum<8>(v, s_red);
        }
        if (threadIdx.x == 0) {
            // FP32 mode: <c, x-bar> = <c, u> + <c, d> + sigma <c, A^T(y-bar - y0)>
            // from exact per-tile and per-slab parts (the per-element x-bar is
            // rounded where u + d nearly cancels); <c, d> joins at the end
            // (restart pass MODE 2, k_block_end)
            const double r2 = v[0], mn2 = v[1], x2 = v[2], z2 = v[3], cx = v[4] + v[7], ax2 = v[5], dob = v[6];
            const double scale = 1.0 / I.h;
            const double rel_dual = sqrt(r2) / (1.0 + I.norm_c);
            const double rel_comp = sqrt(mn2) / (1.0 + sqrt(x2) + sqrt(z2));
            const double rel_primal = sqrt(ax2) / (1.0 + I.norm_b);
            const double rel = fmax(rel_dual, fmax(rel_comp, rel_primal));
            const double absk = fmax(sqrt(r2), fmax(sqrt(mn2), sqrt(ax2)));      // Table VI
            C->abs_kkt = absk;
            C->rel_dual = rel_dual;
            C->rel_comp = rel_comp;
            C->rel_primal = rel_primal;
            C->rel_kkt = rel;
            C->pobj = cx;                 // sum (r-c)^2 x-bar: unscaled <c, x-bar>
            C->dzero = 0;                 // this block's first sweep has read it
            C->dobj = dob * scale;
            const long long total = C->total + K;
            const int kcheck = C->k + K - 1;
            C->total = total;
            int fin = 0;
            if (!(rel == rel) || isinf(rel) || !(cx == cx) || isinf(cx)) {
                C->status = ST_NUMERIC;
                fin = 1;
            } else if (C->cancel) {
                C->status = ST_CANCELLED;
                fin = 1;
            } else if ((I.stop_abs ? absk : rel) <= C->tol) {
                C->status = ST_CONVERGED;
                fin = 1;
            } else if (total >= C->max_iter) {
                C->status = ST_CAPPED;
                fin = 1;
            } else {
                const double r = sqrt(C->sigma) * sqrt(r2);     // ||w - w-bar||_M = sqrt(sigma) ||z-bar - g||
                C->res_norm = r;
                if (C->r0 < 0.0) C->r0 = r;
                const bool rs = (r <= a1 * C->r0) || (C->rprev >= 0.0 && r <= a2 * C->r0 && r > C->rprev) ||
                                ((double)kcheck >= a3 * (double)total);
                C->rprev = r;
                if (rs) C->restart_pending = 1;
                else C->k = C->k + K;
            }
            if (fin) {
                C->just_finished = 1;
                atomicSub(W->n_running, 1);
            }
            W->st_out[i] = C->status;
        }
        __syncthreads();
    }
}

// Sigma update at a restart: sigma <- sqrt(sigma ||x-bar - x_r|| / ||z-bar - z_r||) on the grid 2^(j/16).
template <bool F32>
__global__ void __launch_bounds__(kThreads) k_restart_sigma(const WorkDev* __restrict__ W) {
    pdl_enter();
    __shared__ double s_red[2 * 32];
    const int ninst = W->ninst;
    for (int i = blockIdx.x; i < ninst; i += gridDim.x) {
        const HotInst& I = W->inst[i];
        HotCtl* C = I.ctl;
        if (C->status != ST_RUNNING || !C->restart_pending) continue;
        const int ntile = g_ntiles(I);
        double v[2] = {0.0, 0.0};
        if constexpr (F32) {
            const float2* rp = reinterpret_cast<const float2*>(I.rst_part);
            DF w[2] = {sum_pairs(rp, ntile, 2), sum_pairs(rp + 1, ntile, 2)};
            block_sum_df<2>(w, reinterpret_cast<float2*>(s_red));
            v[0] = df_val(w[0]);
            v[1] = df_val(w[1]);
        } else {
            for (int q = threadIdx.x; q < ntile; q += blockDim.x) {
                v[0] += I.rst_part[(size_t)q * 2];
                v[1] += I.rst_part[(size_t)q * 2 + 1];
            }
            block_sum<2>(v, s_red);
        }
        if (threadIdx.x == 0) {
            const double dx = sqrt(v[0]), dz = sqrt(v[1]);
            const double old = C->sigma;
            C->dx2 = v[0];
            C->dz2 = v[1];
            C->sigma_old = old;
            // geometric mean of the old sigma and the movement ratio, rounded
            // to the grid 2^(j/16) (so rounding noise in dx, dz does not move it)
            if (dx > 0.0 && dz > 0.0 && isfinite(dx / dz)) C->sigma = exp2(rint(log2(sqrt(old * (dx / dz))) * 16.0) / 16.0);
            C->k = 0;
            C->r0 = -1.0;
            C->rprev = -1.0;
            C->restarts += 1;
            if constexpr (F32) C->dzero = 1;   // MODE 1 stores no zero delta; the next first sweep reads none
        }
        __syncthreads();
    }
}

// End of a block: an FP32 instance that finished in it adds the <c, d> share
// of its final check iteration (per-tile pairs from the restart pass MODE 2,
// summed in tile order) to its objective; every instance's flags reset.
// One CTA per instance.
__global__ void __launch_bounds__(kThreads) k_block_end(const WorkDev* __restrict__ W) {
    pdl_enter();
    __shared__ float2 s_red[32];
    const int ninst = W->ninst;
    for (int i = blockIdx.x; i < ninst; i += gridDim.x) {
        const HotInst& I = W->inst[i];
        HotCtl* C = I.ctl;
        if (C->just_finished && !I.fp64) {                // block-uniform
            DF cd[1] = {sum_pairs(reinterpret_cast<const float2*>(I.tile_kkt) + (kNK - 1), g_ntiles(I), kNK)};
            block_sum_df<1>(cd, s_red);
            if (threadIdx.x == 0) C->pobj += df_val(cd[0]);
        }
        if (threadIdx.x == 0) {
            C->restart_pending = 0;
            C->just_finished = 0;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------- launchers --

// SM count x resident CTAs per SM (at most cap) of one kernel at kThreads
template <typename F>
static int occ_grid(F kernel, int sms, size_t dyn_smem, int cap) {
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kThreads, dyn_smem) != cudaSuccess || per < 1)
        per = 1;
    return sms * (per < cap ? per : cap);
}

LaunchDims make_launch_dims(int device, int fp64) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (sms <= 0) sms = 1;
    LaunchDims d;
    if (fp64) {
        d.grid_tile = occ_grid(k_sweep64, sms, 0, 8);
        d.grid_tile_chk = d.grid_tile;
        d.grid_rst = std::min(occ_grid(k_restart<double, 0>, sms, 0, 8), occ_grid(k_restart<double, 1>, sms, 0, 8));
        d.grid_slab = occ_grid(k_alpha<true>, sms, 0, 4);
        d.grid_alpha = d.grid_slab;
        d.grid_vec = occ_grid(k_vec, sms, 0, 4);
        d.grid_vec1 = d.grid_vec;
    } else {
        d.grid_tile = occ_grid(k_sweep32<false, false>, sms, kSweepSmem, 8);
        d.grid_tile_chk = occ_grid(k_sweep32<true, false>, sms, kSweepSmemChk, 8);
        d.grid_rst = std::min(occ_grid(k_restart<float, 0>, sms, 0, 8), occ_grid(k_restart<float, 1>, sms, 0, 8));
        d.grid_slab = occ_grid(k_anchor, sms, 0, 4);
        d.grid_alpha = occ_grid(k_alpha32<true>, sms, 0, 2);
        d.grid_vec = occ_grid(k_vec32<false>, sms, 0, 4);
        d.grid_vec1 = occ_grid(k_vec32<true>, sms, 0, 4);
    }
    d.grid_k1 = occ_grid(k_kkt1<true>, sms, 0, 6);
    d.grid_inst = sms * 2;
    return d;
}

int sweep_grid(int fp64) {
    static int cache[2][64];                 // per precision and device ordinal; 0 = not yet queried
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 0;
    int& c = cache[fp64 ? 1 : 0][dev];
    if (c == 0) c = make_launch_dims(dev, fp64).grid_tile;
    return c;
}

void launch_init(const HotInst& I, double sigma0, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tiles = g_ntiles(I);
    const int grid = tiles < sms * 4 ? tiles : sms * 4;
    if (I.fp64) k_init<double><<<grid, kThreads, 0, st>>>(I, sigma0);
    else k_init<float><<<grid, kThreads, 0, st>>>(I, sigma0);
    k_anchor_one<<<g_nslab(I) < sms * 4 ? g_nslab(I) : sms * 4, kThreads, 0, st>>>(I, sigma0);
}

cudaError_t kernels_init(int device) {
    (void)device;
    cudaError_t e = cudaFuncSetAttribute(k_sweep32<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSweepSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep32<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSweepSmemChk);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep32<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSweepSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep32<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSweepSmemChk);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep32<false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSweepSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep32<false, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSweepSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_marg, cudaFuncAttributeMaxDynamicSharedMemorySize, 7 * kMaxS * 8);
    return e;
}

// One launch of the chain (cudaLaunchKernelEx keeps every call site in one form),
// programmatically dependent on the previous kernel (pdl_enter in every kernel).
template <typename... KArgs, typename... Args>
static void launch(const LaunchDims&, void (*k)(KArgs...), int grid, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, args...);
}

void launch_solve_kernels(const WorkDev* w, const LaunchDims& ld, int fp64, int j, bool check, bool single,
                          cudaStream_t st) {
    if (fp64) {
        launch(ld, k_vec, ld.grid_vec, 0, st, w);
        launch(ld, k_marg, ld.grid_inst, 7 * kMaxS * 8, st, w);
        launch(ld, check ? k_alpha<true> : k_alpha<false>, ld.grid_slab, 0, st, w);
    } else {
        if (single) {
            launch(ld, k_vec32<true>, ld.grid_vec1, 0, st, w, j);
        } else {
            launch(ld, k_vec32<false>, ld.grid_vec, 0, st, w, j);
            launch(ld, k_stage32, ld.grid_inst, 0, st, w, j);
        }
        launch(ld, check ? k_alpha32<true> : k_alpha32<false>, ld.grid_alpha, 0, st, w, j);
    }
}

void launch_sweep(const WorkDev* w, const LaunchDims& ld, int fp64, int j, bool check, bool pad, cudaStream_t st) {
    if (fp64)
        launch(ld, k_sweep64, check ? ld.grid_tile_chk : ld.grid_tile, 0, st, w, j, check ? 1 : 0);
    else if (check)
        launch(ld, pad ? k_sweep32<true, true> : k_sweep32<true, false>, ld.grid_tile_chk, kSweepSmemChk, st, w, j);
    else if (j == 0)
        launch(ld, pad ? k_sweep32<false, true, true> : k_sweep32<false, false, true>, ld.grid_tile, kSweepSmem, st, w, j);
    else
        launch(ld, pad ? k_sweep32<false, true> : k_sweep32<false, false>, ld.grid_tile, kSweepSmem, st, w, j);
}

void launch_block_end(const WorkDev* w, const LaunchDims& ld, int fp64, int K, double a1, double a2, double a3,
                      cudaStream_t st) {
    if (fp64) {
        launch(ld, k_kkt1<false>, ld.grid_k1, 0, st, w);
        launch(ld, k_check<false>, ld.grid_inst, 0, st, w, K, a1, a2, a3);
        launch(ld, k_restart<double, 0>, ld.grid_rst, 0, st, w);
        launch(ld, k_restart_sigma<false>, ld.grid_inst, 0, st, w);
        launch(ld, k_restart<double, 1>, ld.grid_rst, 0, st, w);
        launch(ld, k_anchor, ld.grid_slab, 0, st, w);
        launch(ld, k_restart<double, 2>, ld.grid_rst, 0, st, w);
    } else {
        launch(ld, k_kkt1<true>, ld.grid_k1, 0, st, w);
        launch(ld, k_check<true>, ld.grid_inst, 0, st, w, K, a1, a2, a3);
        launch(ld, k_restart<float, 0>, ld.grid_rst, 0, st, w);
        launch(ld, k_restart_sigma<true>, ld.grid_inst, 0, st, w);
        launch(ld, k_restart<float, 1>, ld.grid_rst, 0, st, w);
        launch(ld, k_anchor, ld.grid_slab, 0, st, w);
        launch(ld, k_restart<float, 2>, ld.grid_rst, 0, st, w);
    }
    launch(ld, k_block_end, ld.grid_inst, 0, st, w);
}

}  // namespace hot
