// HOT iteration kernels for sm_103a (GB300).
//
// One iteration of Algorithm 2 (arXiv 2408.00598) on a batch of instances is
// three launches:
//   k_vec    -- slab totals and cross-slab row sums of the state (inputs of the
//               marginals that Prop. 3 needs), one warp per output;
//   k_alpha  -- Prop. 3: the right-hand side R of eq. (update:y) from the slab
//               sums, its closed-form solution y-bar, and the per-slab
//               broadcast vectors alpha/beta of A^T y-bar; one CTA per slab;
//   k_sweep  -- Steps 2-4 fused into one streaming pass over the flow state:
//               x-bar, z-bar = Pi_+(...), the Halpern update, and the slab row/
//               column sums of the new state (the A v products of the next
//               iteration); on check iterations also the KKT partial sums of
//               eq. (kkt_res).
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
// exact in FP32, plus an FP32 lo part.  Reductions use short FP32 chains
// combined in FP64.
#include "hot_internal.h"

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

// FP32 sums of up to 8 terms, accumulated in FP64 (fixed order).
__device__ __forceinline__ double sum_f32_strided(const float* p, int count, int stride) {
    double acc = 0.0;
    for (int q0 = 0; q0 < count; q0 += 8) {
        float g = 0.f;
        const int q1 = min(count, q0 + 8);
        for (int q = q0; q < q1; ++q) g += p[q * stride];
        acc += (double)g;
    }
    return acc;
}
__device__ __forceinline__ double sum_f64_strided(const double* p, int count, int stride) {
    double acc = 0.0;
    for (int q = 0; q < count; ++q) acc += p[q * stride];
    return acc;
}

// Double-float accumulator: an unevaluated pair (hi, lo) of FP32 values whose
// sum carries about twice the FP32 precision; each add is an exact two-sum
// followed by renormalisation (FP32 arithmetic only).  Used where a sum
// must be accurate to FP64 level but FP64 per element would be too slow.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_add(DF a, float b) {
    const float s = a.hi + b;
    const float bb = s - a.hi;
    const float e = ((a.hi - (s - bb)) + (b - bb)) + a.lo;
    const float h = s + e;
    return DF{h, e - (h - s)};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    DF r = df_add(a, b.hi);
    return df_add(r, b.lo);
}
__device__ __forceinline__ double df_val(DF a) { return (double)a.hi + (double)a.lo; }

// ------------------------------------------------------ per-tile parameters --

struct P32 {
    float sih;        // 1/sigma
    float sf;         // sigma
    float rho, trs;   // Halpern: rho = (k+1)/(k+2), trs = 2 rho sigma
    float h;          // 2^-E
};
struct P64 {
    double is, s, rho, trs, h;
};

__device__ __forceinline__ P32 make_p32(double sigma, int k, double h) {
    P32 p;
    p.sih = (float)(1.0 / sigma);
    p.sf = (float)sigma;
    const double rho = (k + 1.0) / (k + 2.0);
    p.rho = (float)rho;
    p.trs = (float)(2.0 * rho * sigma);
    p.h = (float)h;
    return p;
}
__device__ __forceinline__ P64 make_p64(double sigma, int k, double h) {
    P64 p;
    p.is = 1.0 / sigma;
    p.s = sigma;
    p.rho = (k + 1.0) / (k + 2.0);
    p.trs = 2.0 * p.rho * sigma;
    p.h = h;
    return p;
}

// Element math of Steps 2-3.  Inputs: anchor u, delta d, cost cq = (r-c)^2
// (unscaled integer), the slab row/column pieces of A^T y-bar (hi, lo) and of
// dA = A^T(y-bar - y0).  Outputs: w = g - v/sigma, mg = -g and
// r = z-bar - g = max(-g, g - v/sigma), the dual residual entry.
struct E32 {
    float Gh, Gl, D, s, w, mg, r;
};
__device__ __forceinline__ E32 elem32(float u, float d, float cq, const float4& a, const float4& b, const P32& p) {
    E32 e;
    e.Gh = fmaf(cq, p.h, -a.x) - b.x;       // exact: every term is on the grid 2^-E
    e.Gl = -(a.y + b.y);
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
        const float4 t = __ldg(reinterpret_cast<const float4*>(p));
        x[0] = t.x; x[1] = t.y; x[2] = t.z; x[3] = t.w;
    }
    __device__ static void st(float* p, const float (&x)[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
    }
};
template <> struct VecT<double> {
    using type = double2;
    static constexpr int N = 2;
    __device__ static void ld(const double* p, double (&x)[2]) {
        const double2 t = __ldg(reinterpret_cast<const double2*>(p));
        x[0] = t.x; x[1] = t.y;
    }
    __device__ static void st(double* p, const double (&x)[2]) {
        *reinterpret_cast<double2*>(p) = make_double2(x[0], x[1]);
    }
};

// Asynchronous global -> shared copies (16 B per thread, cached in L2 only).
// A thread waits only for its own copies (cp.async.wait_group), so a pipeline
// in which every thread reads back only what it copied needs no barrier.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
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
    const HotInst& I = W->inst[tc.inst];
    tc.slab = s_tile[1] / I.nb;
    tc.band = s_tile[1] % I.nb;
    return true;
}

// ----------------------------------------------------------------- k_vec --
// T1[j] = sum_k rowsum(f1 slab j)[k], T2[k] = sum_j rowsum(f2 slab k)[j],
// P1[k] = sum_j rowsum(f1 slab j)[k], P2[j] = sum_k rowsum(f2 slab k)[j];
// row sums are those of u + d (the slab sums of u are kept separately).
__global__ void __launch_bounds__(kThreads) k_vec(const WorkDev* __restrict__ W) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ninst = W->ninst;
    const int nitems = W->pre_vec[ninst];
    for (int base = blockIdx.x * (kThreads / 32); base < nitems; base += gridDim.x * (kThreads / 32)) {
        const int item = base + warp;
        if (item >= nitems) continue;
        const int i = find_inst(W->pre_vec, ninst, item);
        const HotInst& I = W->inst[i];
        if (I.ctl->status != ST_RUNNING) continue;
        const int S = I.S;
        const int q = item - W->pre_vec[i];
        const int which = q / S, idx = q % S;
        const double* __restrict__ rs = I.rs;
        const double* __restrict__ rs0 = I.rs0;
        double acc = 0.0;
        if (which == 0) {
            for (int t = lane; t < S; t += 32) acc += rs[idx * S + t] + rs0[idx * S + t];
        } else if (which == 1) {
            for (int t = lane; t < S; t += 32) acc += rs[(S + idx) * S + t] + rs0[(S + idx) * S + t];
        } else if (which == 2) {
            for (int t = lane; t < S; t += 32) acc += rs[t * S + idx] + rs0[t * S + idx];
        } else {
            for (int t = lane; t < S; t += 32) acc += rs[(S + t) * S + idx] + rs0[(S + t) * S + idx];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) I.vecs[which * S + idx] = acc;
    }
}

// ---------------------------------------------------------- k_marg/k_alpha --
// Prop. 3 on R' = (b - A(u + d))/sigma, the right-hand side whose solution is
// dy = y-bar - y0: with v = sigma g0 + u + d, the right-hand side of
// eq. (update:y) is R = b/sigma - A(v/sigma - c) = AA^T y0 + R'.  R' comes
// from the slab sums of u + d.  With m = n = S:
//   a_j = sum_k R1(k,j), bb_j = sum_i R2(i,j), r3_k = sum_l R3(k,l), T3 = sum r3,
//   y1-hat(k,j) = (R1(k,j) + a_j/n - (1/m+1/n) bb_j + r3_k/n + T3/n^2)/(m+n),
//   s_k = sum_j y1-hat(k,j),  t = W-hat s,  y1^a = t + (1^T t / n) 1,
//   y1 = y1-hat - y1^a,  y2(i,j) = (R2(i,j) - sum_k y1(k,j))/m,
//   y3(k,l) = (R3(k,l) + sum_j y1(k,j))/n.
// k_marg (one CTA per instance) forms the O(S) vectors shared by all slabs:
//   mv[0..S)   a_j / n - (1/m + 1/n) bb_j        (column part of y1-hat)
//   mv[S..2S)  r3_k / n + T3 / n^2 - (m+n) y1^a_k (row part of y1, times m+n)
//   mv[2S..3S) sum_k y1(k,j)                      (for y2)
//   mv[3S..4S) sum_j y1(k,j)                      (for y3)
// k_alpha (one CTA per slab) then forms the slab's entries with products only
// (FP64 division is slow on this part; reciprocals are taken once).
__global__ void __launch_bounds__(kThreads) k_marg(const WorkDev* __restrict__ W) {
    extern __shared__ double sv[];                   // 7 * S: T1 T2 P1 P2 colmu1 rowmu2, then s
    __shared__ double s_red[4 * 32];
    const int ninst = W->ninst;
    for (int inst = blockIdx.x; inst < ninst; inst += gridDim.x) {
        const HotInst& I = W->inst[inst];
        if (I.ctl->status != ST_RUNNING) continue;     // block-uniform
        const int S = I.S, nb = I.nb;
        const double m = S, n = S;
        const double is = 1.0 / I.ctl->sigma;
        const double in_ = 1.0 / n, im = 1.0 / m, imn = 1.0 / (m + n);
        double* T1 = sv;
        double* T2 = sv + S;
        double* P1 = sv + 2 * S;
        double* P2 = sv + 3 * S;
        double* cm = sv + 4 * S;
        double* rm = sv + 5 * S;
        double* ss = sv + 6 * S;
        for (int q = threadIdx.x; q < 4 * S; q += blockDim.x) sv[q] = I.vecs[q];
        for (int q = threadIdx.x; q < S; q += blockDim.x) {
            cm[q] = I.colmu1[q];
            rm[q] = I.rowmu2[q];
        }
        // column S-1 of the last f2 slab: the dropped (m, n) row of eq. (7)
        double kap_last = I.kapa[(size_t)(2 * S - 1) * S + (S - 1)];
        {
            const int sl = 2 * S - 1;
            if (I.fp64)
                for (int b = 0; b < nb; ++b) kap_last += I.cs_part[((size_t)sl * nb + b) * S + (S - 1)];
            else
                for (int b = 0; b < nb; ++b) kap_last += (double)I.cs32[((size_t)sl * nb + b) * S + (S - 1)];
        }
        const double mu_last = I.mu2[(size_t)(S - 1) * S + (S - 1)];
        __syncthreads();
        auto A_ = [&](int q) { return -(T1[q] - P2[q]) * is; };
        auto B_ = [&](int q) { return (cm[q] - T1[q]) * is; };
        auto R3_ = [&](int q) {
            double r = (rm[q] - T2[q]) * is;
            if (q == S - 1) r -= (mu_last - kap_last) * is;
            return r;
        };
        double red[4] = {0.0, 0.0, 0.0, 0.0};
        for (int q = threadIdx.x; q < S; q += blockDim.x) {
            red[0] += A_(q);
            red[1] += B_(q);
            red[2] += R3_(q);
        }
        block_sum<4>(red, s_red);
        const double Asum = red[0], Bsum = red[1], T3 = red[2];
        const double dl = (1.0 - in_) / (m + 1.0);
        const double iw = 1.0 / (im - dl);             // 1/w, w = 1/m - (1-1/n)/(m+1)
        red[0] = red[1] = red[2] = red[3] = 0.0;
        for (int q = threadIdx.x; q < S; q += blockDim.x) {
            const double rowR1 = -(P1[q] - T2[q]) * is;
            const double s = (rowR1 + Asum * in_ - (im + in_) * Bsum + R3_(q) + T3 * in_) * imn;   // s_k
            ss[q] = s;
            red[0] += (q == S - 1 ? dl : im) * s;
        }
        block_sum<4>(red, s_red);
        const double ds = red[0];
        red[0] = red[1] = red[2] = red[3] = 0.0;
        for (int q = threadIdx.x; q < S; q += blockDim.x) {
            const double dq = (q == S - 1 ? dl : im);
            red[0] += -dq * ss[q] - dq * ds * iw;       // 1^T W-hat s
        }
        block_sum<4>(red, s_red);
        const double tsum = red[0];
        red[0] = red[1] = red[2] = red[3] = 0.0;
        for (int q = threadIdx.x; q < S; q += blockDim.x) {
            const double dq = (q == S - 1 ? dl : im);
            red[0] += -dq * ss[q] - dq * ds * iw + tsum * in_;
        }
        block_sum<4>(red, s_red);
        const double yasum = red[0];
        double* mv = I.mvec;
        for (int q = threadIdx.x; q < S; q += blockDim.x) {
            const double dq = (q == S - 1 ? dl : im);
            const double ya = -dq * ss[q] - dq * ds * iw + tsum * in_;   // y1^a
            const double aq = A_(q), bq = B_(q);
            mv[q] = aq * in_ - (im + in_) * bq;
            mv[S + q] = R3_(q) * in_ + T3 * in_ * in_ - (m + n) * ya;
            mv[2 * S + q] = (aq - bq + T3 * in_) * in_ - yasum;
            mv[3 * S + q] = ss[q] - n * ya;
        }
        __syncthreads();
    }
}

// Per-slab entries of dy = A^T-pieces of y-bar - y0.  The anchor part of R
// (row sums and column totals of u) is precomputed once per cycle by
// k_anchor; here only the delta's sums enter.  FP32 mode splits each full
// piece a0 + dy into a part on the grid 2^-E and a remainder using FP32
// arithmetic on top of the per-cycle split of a0.
template <bool CHECK>
__global__ void __launch_bounds__(kThreads) k_alpha(const WorkDev* __restrict__ W) {
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
        const int S = I.S, nb = I.nb;
        const double m = S, n = S;
        const double is = 1.0 / I.ctl->sigma;
        const double im = 1.0 / m, in_ = 1.0 / n, imn = 1.0 / (m + n);
        const double* __restrict__ rs = I.rs;
        const double* __restrict__ mv = I.mvec;
        const double* __restrict__ R1a = I.R1a + (size_t)slab * S;
        const double* __restrict__ kapa = I.kapa + (size_t)slab * S;
        const size_t o = (size_t)slab * 2 * S;
        const bool fp32 = I.ab32 != nullptr;
        const float grid = (float)(1.0 / I.h), igrid = (float)I.h;
        float ymax = 0.f;
        double dob = 0.0;
        // idx < S: alpha (row) entries, idx >= S: beta (column) entries; returns the full piece
        auto put = [&](int idx, double dv) -> double {
            I.dab64[o + idx] = dv;
            double full;
            if (fp32) {
                const float df = (float)dv;
                const float dh = rintf(df * grid) * igrid;      // on the grid 2^-E
                const float2 a0 = I.ab0_32[o + idx];
                I.ab32[o + idx] = make_float4(a0.x + dh, a0.y + (df - dh), df, 0.f);
                full = CHECK ? I.ab0[o + idx] + dv : 0.0;
            } else {
                full = I.ab0[o + idx] + dv;
                I.ab64[o + idx] = full;
            }
            if (CHECK) ymax = fmaxf(ymax, fabsf((float)full));
            return full;
        };
        auto kap_delta = [&](int c) -> double {           // column total of the delta over the bands
            if (fp32) {
                float k = 0.f;
                for (int b = 0; b < nb; ++b) k += I.cs32[((size_t)slab * nb + b) * S + c];
                return (double)k;
            }
            double k = 0.0;
            for (int b = 0; b < nb; ++b) k += I.cs_part[((size_t)slab * nb + b) * S + c];
            return k;
        };
        if (slab < S) {
            const int j = slab;
            const double colj = mv[j];
            for (int k = threadIdx.x; k < S; k += blockDim.x) {
                const double R1 = R1a[k] - (rs[(size_t)j * S + k] - rs[(size_t)(S + k) * S + j]) * is;
                put(k, (R1 + colj + mv[S + k]) * imn);         // y1(k, j)
            }
            const double sy = mv[2 * S + j];
            for (int i = threadIdx.x; i < S; i += blockDim.x) {
                const double kap = kapa[i] + kap_delta(i);
                const double mu = I.mu1[(size_t)i * S + j];
                const double full = put(S + i, ((mu - kap) * is - sy) * im);   // y2(i, j)
                if (CHECK) dob += mu * full;                                    // <b, y>: mu1 . y2
            }
        } else {
            const int k = slab - S;
            const double rowk = mv[S + k];
            for (int j = threadIdx.x; j < S; j += blockDim.x) {
                const double R1 = R1a[j] - (rs[(size_t)j * S + k] - rs[(size_t)(S + k) * S + j]) * is;
                put(j, -(R1 + mv[j] + rowk) * imn);            // -y1(k, j): A2 = -1_n^T kron I_M
            }
            const double sp = mv[3 * S + k];
            for (int l = threadIdx.x; l < S; l += blockDim.x) {
                if (k == S - 1 && l == S - 1) {
                    put(S + l, 0.0);                           // no row: y3(m, n) = 0
                    continue;
                }
                const double kap = kapa[l] + kap_delta(l);
                const double mu = I.mu2[(size_t)k * S + l];
                const double full = put(S + l, ((mu - kap) * is + sp) * in_);  // y3(k, l)
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

// Once per cycle (after a restart, and at the start): the anchor parts of the
// right-hand side, per slab: R1a along the slab's rows and the column totals
// of u.  One CTA per slab.
__device__ __forceinline__ void anchor_slab(const HotInst& I, int slab, double sigma) {
    const int S = I.S, nb = I.nb;
    const double is = 1.0 / sigma;
    for (int q = threadIdx.x; q < S; q += blockDim.x) {
        // f1 slab j: rows k, R1(k, j); f2 slab k: rows j, R1(k, j)
        const int j = slab < S ? slab : q;
        const int k = slab < S ? q : slab - S;
        I.R1a[(size_t)slab * S + q] = -(I.rs0[(size_t)j * S + k] - I.rs0[(size_t)(S + k) * S + j]) * is;
        double kap = 0.0;
        for (int b = 0; b < nb; ++b) kap += I.cs0_part[((size_t)slab * nb + b) * S + q];
        I.kapa[(size_t)slab * S + q] = kap;
    }
}

__global__ void __launch_bounds__(kThreads) k_anchor(const WorkDev* __restrict__ W) {
    __shared__ int s_t[4];
    const int ninst = W->ninst;
    const int nslab = W->pre_slab[ninst];
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
    for (int slab = blockIdx.x; slab < 2 * I.S; slab += gridDim.x) anchor_slab(I, slab, sigma);
}

// --------------------------------------------------------------- k_sweep --
// Steps 2-4 of Algorithm 2 on one tile (TR rows of one slab).
template <typename T, bool CHECK>
__global__ void __launch_bounds__(kThreads) k_sweep(const WorkDev* __restrict__ W, int j) {
    using V = VecT<T>;
    constexpr int NV = V::N;
    // row partials, one padded row of NC+1 entries per tile row (conflict-free
    // on the write, where a warp spans columns, and on the reduction, where it
    // spans rows)
    constexpr int kRowN = kRowSmemBytes / sizeof(float) / (sizeof(T) / sizeof(float)) + 256;
    __shared__ __align__(16) T s_row[kRowN];
    __shared__ __align__(16) T s_col[kThreads * NV];
    __shared__ __align__(16) T s_xrow[CHECK ? kRowN : 1];
    __shared__ __align__(16) T s_xcol[CHECK ? kThreads * NV : 1];
    __shared__ double s_red[kNK * 32];
    __shared__ int s_tile[4];
    __shared__ P32 s_p32;
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
        const int S = I.S, nb = I.nb, TR = I.TR;
        const int slab = tc.slab, band = tc.band;
        const int NC = S / NV;
        const int P = kThreads / NC;
        const int cg = threadIdx.x % NC, ro = threadIdx.x / NC;
        const bool active = ro < P;
        const int r0 = band * TR, r1 = min(S, r0 + TR);
        const size_t off = (size_t)slab * S * S;
        const T* __restrict__ u = (const T*)I.u + off;
        const T* __restrict__ din = (const T*)((j & 1) ? I.d1 : I.d0) + off;
        T* __restrict__ dout = (T*)((j & 1) ? I.d0 : I.d1) + off;
        // per-tile constants (FP64 divisions are slow here: one thread forms them)
        if (threadIdx.x == 0) {
            const int kc = I.ctl->k + j;
            if constexpr (std::is_same<T, float>::value) s_p32 = make_p32(I.ctl->sigma, kc, I.h);
            else s_p64 = make_p64(I.ctl->sigma, kc, I.h);
        }
        __syncthreads();
        const int c0 = cg * NV;
        T cacc[NV], xacc[NV];
#pragma unroll
        for (int e = 0; e < NV; ++e) cacc[e] = xacc[e] = T(0);
        float k32[kNK] = {0.f, 0.f, 0.f, 0.f, 0.f};
        double k64[kNK] = {0.0, 0.0, 0.0, 0.0, 0.0};

        if constexpr (std::is_same<T, float>::value) {
            const P32 p = s_p32;
            const float4* ab = I.ab32 + (size_t)slab * 2 * S;
            float4 bq[NV];
            float cf[NV];
#pragma unroll
            for (int e = 0; e < NV; ++e) {
                bq[e] = active ? ab[S + c0 + e] : make_float4(0.f, 0.f, 0.f, 0.f);
                cf[e] = (float)(c0 + e);
            }
            if (active) {
                int nrow = 0;
                auto row = [&](int r, const float (&uu)[NV], const float (&dd)[NV]) {
                    const float4 a = ab[r];
                    const float rf = (float)r;
                    float out[NV], xo[NV];
#pragma unroll
                    for (int e = 0; e < NV; ++e) {
                        const float dc = rf - cf[e];
                        const float cq = dc * dc;
                        const E32 el = elem32(uu[e], dd[e], cq, a, bq[e], p);
                        out[e] = fmaf(p.trs, el.r, p.rho * dd[e]);
                        if constexpr (CHECK) {
                            float xb, zb;
                            xz32(el, p, xb, zb);
                            xo[e] = xb;
                            const float mn = fminf(xb, zb);
                            k32[0] = fmaf(el.r, el.r, k32[0]);
                            k32[1] = fmaf(mn, mn, k32[1]);
                            k32[2] = fmaf(xb, xb, k32[2]);
                            k32[3] = fmaf(zb, zb, k32[3]);
                            k32[4] = fmaf(cq, xb, k32[4]);
                            xacc[e] += xb;
                        }
                        cacc[e] += out[e];
                    }
                    V::st(dout + (size_t)r * S + c0, out);
                    s_row[(r - r0) * (NC + 1) + cg] = (out[0] + out[1]) + (out[2] + out[3]);
                    if constexpr (CHECK) {
                        s_xrow[(r - r0) * (NC + 1) + cg] = (xo[0] + xo[1]) + (xo[2] + xo[3]);
                        // FP32 chains of 64 terms, combined in FP64
                        if ((++nrow & 15) == 0) {
#pragma unroll
                            for (int q = 0; q < kNK; ++q) {
                                k64[q] += (double)k32[q];
                                k32[q] = 0.f;
                            }
                        }
                    }
                };
                // kStages-deep cp.async pipeline over the passes of this tile:
                // pass q covers row r0 + ro + q P of every active thread
                extern __shared__ float4 s_stage[];          // [kStages][2][kThreads]
                const int npass = (r1 - r0 + P - 1) / P;
                auto issue = [&](int q) {
                    const int r = r0 + ro + q * P;
                    if (r < r1) {
                        float4* su = s_stage + (size_t)(q % kStages) * 2 * kThreads + threadIdx.x;
                        cp_async16(su, u + (size_t)r * S + c0);
                        cp_async16(su + kThreads, din + (size_t)r * S + c0);
                    }
                    cp_async_commit();                       // empty groups keep the count aligned
                };
#pragma unroll
                for (int q = 0; q < kStages - 1; ++q) issue(q);
                for (int q = 0; q < npass; ++q) {
                    issue(q + kStages - 1);
                    cp_async_wait<kStages - 1>();            // this thread's pass-q copies are in
                    const int r = r0 + ro + q * P;
                    if (r < r1) {
                        const float4* su = s_stage + (size_t)(q % kStages) * 2 * kThreads + threadIdx.x;
                        const float4 U = su[0], D = su[kThreads];
                        const float uu[NV] = {U.x, U.y, U.z, U.w};
                        const float dd[NV] = {D.x, D.y, D.z, D.w};
                        row(r, uu, dd);
                    }
                }
                cp_async_wait<0>();
            }
#pragma unroll
            for (int q = 0; q < kNK; ++q) k64[q] += (double)k32[q];
        } else {
            const P64 p = s_p64;
            const double* ab = I.ab64 + (size_t)slab * 2 * S;
            const double* dab = I.dab64 + (size_t)slab * 2 * S;
            double bb[NV], db[NV], cf[NV];
#pragma unroll
            for (int e = 0; e < NV; ++e) {
                bb[e] = active ? ab[S + c0 + e] : 0.0;
                db[e] = active ? dab[S + c0 + e] : 0.0;
                cf[e] = (double)(c0 + e);
            }
            if (active) {
                for (int r = r0 + ro; r < r1; r += P) {
                    const double a = ab[r], da = dab[r];
                    const double rf = (double)r;
                    double uu[NV], dd[NV], out[NV], xo[NV];
                    V::ld(u + (size_t)r * S + c0, uu);
                    V::ld(din + (size_t)r * S + c0, dd);
#pragma unroll
                    for (int e = 0; e < NV; ++e) {
                        const double dc = rf - cf[e];
                        const double cq = dc * dc;
                        const E64 el = elem64(uu[e], dd[e], cq, a, bb[e], da, db[e], p);
                        out[e] = p.rho * dd[e] + p.trs * el.r;
                        if constexpr (CHECK) {
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
                    V::st(dout + (size_t)r * S + c0, out);
                    s_row[(r - r0) * (NC + 1) + cg] = out[0] + out[1];
                    if constexpr (CHECK) s_xrow[(r - r0) * (NC + 1) + cg] = xo[0] + xo[1];
                }
            }
        }
        __syncthreads();
        if (active) {
#pragma unroll
            for (int e = 0; e < NV; ++e) {
                s_col[ro * S + c0 + e] = cacc[e];
                if constexpr (CHECK) s_xcol[ro * S + c0 + e] = xacc[e];
            }
        }
        __syncthreads();
        const size_t cbase = ((size_t)slab * nb + band) * S;
        for (int c = threadIdx.x; c < S; c += blockDim.x) {
            if constexpr (std::is_same<T, float>::value) {
                I.cs32[cbase + c] = (float)sum_f32_strided(s_col + c, P, S);
                if constexpr (CHECK) I.xcs_part[cbase + c] = sum_f32_strided(s_xcol + c, P, S);
            } else {
                I.cs_part[cbase + c] = sum_f64_strided(s_col + c, P, S);
                if constexpr (CHECK) I.xcs_part[cbase + c] = sum_f64_strided(s_xcol + c, P, S);
            }
        }
        for (int rr = threadIdx.x; rr < r1 - r0; rr += blockDim.x) {
            if constexpr (std::is_same<T, float>::value) {
                I.rs[(size_t)slab * S + r0 + rr] = sum_f32_strided(s_row + rr * (NC + 1), NC, 1);
                if constexpr (CHECK) I.xrs[(size_t)slab * S + r0 + rr] = sum_f32_strided(s_xrow + rr * (NC + 1), NC, 1);
            } else {
                I.rs[(size_t)slab * S + r0 + rr] = sum_f64_strided(s_row + rr * (NC + 1), NC, 1);
                if constexpr (CHECK) I.xrs[(size_t)slab * S + r0 + rr] = sum_f64_strided(s_xrow + rr * (NC + 1), NC, 1);
            }
        }
        if constexpr (CHECK) {
            block_sum<kNK>(k64, s_red);
            if (threadIdx.x == 0) {
                double* o = I.tile_kkt + ((size_t)slab * nb + band) * kNK;
#pragma unroll
                for (int q = 0; q < kNK; ++q) o[q] = k64[q];
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------- restart tiles --
// MODE 0: partial ||x-bar - x_r||^2, ||z-bar - z_r||^2 of the check iteration.
// MODE 1: restart at the check iteration: anchor and iterate <- w-bar, i.e.
//         v0 = x-bar + sigma_new z-bar and y0 = y-bar, stored as
//         u = v0 - sigma_new g-bar = x-bar + sigma_new r (r = z-bar - g-bar);
//         (x_r, z_r) = (x-bar, z-bar); delta = 0; FP64 slab sums of u;
//         A^T y0 pieces <- those of y-bar.
// MODE 2: x-bar of the final check iteration into x_r (the solution).
// The check iteration (index K-1, odd) read delta buffer d1.
template <typename T, int MODE>
__device__ __forceinline__ void restart_tile(const HotInst& I, int slab, int band, double* s_row, double* s_col,
                                             double* s_red) {
    using V = VecT<T>;
    constexpr int NV = V::N;
    constexpr bool F32 = std::is_same<T, float>::value;
    const int S = I.S, nb = I.nb, TR = I.TR;
    const int NC = S / NV;
    const int P = kThreads / NC;
    const int cg = threadIdx.x % NC, ro = threadIdx.x / NC;
    const bool active = ro < P;
    const int r0 = band * TR, r1 = min(S, r0 + TR);
    const size_t off = (size_t)slab * S * S;
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
        for (int r = r0 + ro; r < r1; r += P) {
            T uu[NV], dd[NV], xbv[NV], zbv[NV], rv[NV];
            V::ld(u + (size_t)r * S + c0, uu);
            V::ld(d1 + (size_t)r * S + c0, dd);
            if constexpr (F32) {
                const P32 p = make_p32(sig_old, 0, I.h);
                const float4* ab = I.ab32 + (size_t)slab * 2 * S;
                const float4 a = ab[r];
#pragma unroll
                for (int e = 0; e < NV; ++e) {
                    const float dc = (float)r - (float)(c0 + e);
                    const E32 el = elem32(uu[e], dd[e], dc * dc, a, ab[S + c0 + e], p);
                    xz32(el, p, xbv[e], zbv[e]);
                    rv[e] = el.r;
                }
            } else {
                const P64 p = make_p64(sig_old, 0, I.h);
                const double* ab = I.ab64 + (size_t)slab * 2 * S;
                const double* dab = I.dab64 + (size_t)slab * 2 * S;
                const double a = ab[r], da = dab[r];
#pragma unroll
                for (int e = 0; e < NV; ++e) {
                    const double dc = (double)r - (double)(c0 + e);
                    const E64 el = elem64(uu[e], dd[e], dc * dc, a, ab[S + c0 + e], da, dab[S + c0 + e], p);
                    xz64(el, p, xbv[e], zbv[e]);
                    rv[e] = el.r;
                }
            }
            if constexpr (MODE == 0) {
                T xo[NV], zo[NV];
                V::ld(xr + (size_t)r * S + c0, xo);
                V::ld(zr + (size_t)r * S + c0, zo);
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
#pragma unroll
                for (int e = 0; e < NV; ++e) {
                    if constexpr (F32) nu_[e] = fmaf((float)sig_new, rv[e], xbv[e]);
                    else nu_[e] = xbv[e] + sig_new * rv[e];
                    zero[e] = T(0);
                    if constexpr (F32) {
                        rsf = df_add(rsf, (float)nu_[e]);
                        fcol[e] = df_add(fcol[e], (float)nu_[e]);
                    } else {
                        rsd += nu_[e];
                        ccol[e] += nu_[e];
                    }
                }
                V::st(u + (size_t)r * S + c0, nu_);
                V::st(xr + (size_t)r * S + c0, xbv);
                V::st(zr + (size_t)r * S + c0, zbv);
                V::st(d0 + (size_t)r * S + c0, zero);
                s_row[(r - r0) * NC + cg] = F32 ? df_val(rsf) : rsd;
            } else {
                V::st(xr + (size_t)r * S + c0, xbv);
            }
        }
    }
    if constexpr (F32) {
        racc[0] = df_val(fr[0]);
        racc[1] = df_val(fr[1]);
#pragma unroll
        for (int e = 0; e < NV; ++e) ccol[e] = df_val(fcol[e]);
    }
    if constexpr (MODE == 0) {
        block_sum<2>(racc, s_red);
        if (threadIdx.x == 0) {
            double* o = I.rst_part + ((size_t)slab * nb + band) * 2;
            o[0] = racc[0];
            o[1] = racc[1];
        }
    } else if constexpr (MODE == 1) {
        __syncthreads();
        if (active)
#pragma unroll
            for (int e = 0; e < NV; ++e) s_col[ro * S + c0 + e] = ccol[e];
        __syncthreads();
        const size_t cbase = ((size_t)slab * nb + band) * S;
        for (int c = threadIdx.x; c < S; c += blockDim.x) {
            I.cs0_part[cbase + c] = sum_f64_strided(s_col + c, P, S);
            I.cs_part[cbase + c] = 0.0;
            I.cs32[cbase + c] = 0.f;
        }
        // y0 <- y-bar: A^T y0 pieces of this tile's rows (and, for band 0, columns)
        const size_t o = (size_t)slab * 2 * S;
        auto set_anchor = [&](int idx) {
            const double a0 = I.ab0[o + idx] + I.dab64[o + idx];
            I.ab0[o + idx] = a0;
            if (I.ab0_32) {
                const double hi = rint(a0 / I.h) * I.h;          // on the grid 2^-E
                I.ab0_32[o + idx] = make_float2((float)hi, (float)(a0 - hi));
            }
        };
        for (int rr = threadIdx.x; rr < r1 - r0; rr += blockDim.x) {
            I.rs0[(size_t)slab * S + r0 + rr] = sum_f64_strided(s_row + rr * NC, NC, 1);
            I.rs[(size_t)slab * S + r0 + rr] = 0.0;
            set_anchor(r0 + rr);
        }
        if (band == 0)
            for (int c = threadIdx.x; c < S; c += blockDim.x) set_anchor(S + c);
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) k_restart(const WorkDev* __restrict__ W) {
    __shared__ double s_row[MODE == 1 ? kRowSmemBytes / 8 * 2 : 1];
    __shared__ double s_col[MODE == 1 ? kThreads * 4 : 1];
    __shared__ double s_red[2 * 32];
    __shared__ int s_tile[4];
    const int ninst = W->ninst;
    const int ntiles = W->pre_tile[ninst];
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
    const int S = I.S, nb = I.nb, TR = I.TR;
    const int NC = S / NV;
    const int P = kThreads / NC;
    const int cg = threadIdx.x % NC, ro = threadIdx.x / NC;
    const bool active = ro < P;
    const int c0 = cg * NV;
    for (int t = blockIdx.x; t < 2 * S * nb; t += gridDim.x) {
        const int slab = t / nb, band = t % nb;
        const int r0 = band * TR, r1 = min(S, r0 + TR);
        const size_t off = (size_t)slab * S * S;
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
                    const double dc = (double)(r - (c0 + e));
                    uu[e] = (T)(-sigma0 * (dc * dc * I.h));
                    zero[e] = T(0);
                    if constexpr (std::is_same<T, float>::value) {
                        rsf = df_add(rsf, (float)uu[e]);
                        fcol[e] = df_add(fcol[e], (float)uu[e]);
                    } else {
                        rs += (double)uu[e];
                        ccol[e] += (double)uu[e];
                    }
                }
                if constexpr (std::is_same<T, float>::value) rs = df_val(rsf);
                V::st((T*)I.u + off + (size_t)r * S + c0, uu);
                V::st((T*)I.d0 + off + (size_t)r * S + c0, zero);
                V::st((T*)I.xr + off + (size_t)r * S + c0, zero);
                V::st((T*)I.zr + off + (size_t)r * S + c0, zero);
                s_row[(r - r0) * NC + cg] = rs;
            }
        }
        if constexpr (std::is_same<T, float>::value)
#pragma unroll
            for (int e = 0; e < NV; ++e) ccol[e] = df_val(fcol[e]);
        __syncthreads();
        if (active)
#pragma unroll
            for (int e = 0; e < NV; ++e) s_col[ro * S + c0 + e] = ccol[e];
        __syncthreads();
        const size_t cbase = ((size_t)slab * nb + band) * S;
        for (int c = threadIdx.x; c < S; c += blockDim.x) I.cs0_part[cbase + c] = sum_f64_strided(s_col + c, P, S);
        for (int rr = threadIdx.x; rr < r1 - r0; rr += blockDim.x)
            I.rs0[(size_t)slab * S + r0 + rr] = sum_f64_strided(s_row + rr * NC, NC, 1);
        __syncthreads();
    }
}

// --------------------------------------------------------------- k_kkt1 --
// Partial sums of ||A x-bar - b||^2 from the x-bar slab sums.
__global__ void __launch_bounds__(kThreads) k_kkt1(const WorkDev* __restrict__ W) {
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
        const int S = I.S, nb = I.nb;
        const int SS = S * S;
        const int q = s_t[1] * kThreads + threadIdx.x;
        double v[1] = {0.0};
        if (q < 3 * SS - 1) {
            double res;
            if (q < SS) {
                const int j = q / S, k = q % S;
                res = I.xrs[(size_t)j * S + k] - I.xrs[(size_t)(S + k) * S + j];
            } else if (q < 2 * SS) {
                const int j = (q - SS) / S, i = (q - SS) % S;
                double kap = 0.0;
                for (int b = 0; b < nb; ++b) kap += I.xcs_part[((size_t)j * nb + b) * S + i];
                res = kap - I.mu1[(size_t)i * S + j];
            } else {
                const int k = (q - 2 * SS) / S, l = (q - 2 * SS) % S;
                double kap = 0.0;
                for (int b = 0; b < nb; ++b) kap += I.xcs_part[((size_t)(S + k) * nb + b) * S + l];
                res = kap - I.mu2[(size_t)k * S + l];
            }
            v[0] = res * res;
        }
        block_sum<1>(v, s_red);
        if (threadIdx.x == 0) I.k1_part[s_t[1]] = v[0];
        __syncthreads();
    }
}

// --------------------------------------------------------------- k_check --
// Stopping rule eq. (kkt_res) and the restart rule, one CTA per instance.
__global__ void __launch_bounds__(kThreads) k_check(const WorkDev* __restrict__ W, int K, double a1, double a2,
                                                    double a3) {
    __shared__ double s_red[8 * 32];
    const int ninst = W->ninst;
    for (int i = blockIdx.x; i < ninst; i += gridDim.x) {
        const HotInst& I = W->inst[i];
        HotCtl* C = I.ctl;
        if (C->status != ST_RUNNING) continue;   // block-uniform
        const int S = I.S, nb = I.nb;
        const int ntile = 2 * S * nb;
        double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int q = threadIdx.x; q < ntile; q += blockDim.x)
            for (int e = 0; e < kNK; ++e) v[e] += I.tile_kkt[(size_t)q * kNK + e];
        for (int q = threadIdx.x; q < I.n_k1; q += blockDim.x) v[5] += I.k1_part[q];
        for (int q = threadIdx.x; q < 2 * S; q += blockDim.x) v[6] += I.dobj_part[q];
        block_sum<8>(v, s_red);
        if (threadIdx.x == 0) {
            const double r2 = v[0], mn2 = v[1], x2 = v[2], z2 = v[3], cx = v[4], ax2 = v[5], dob = v[6];
            const double scale = 1.0 / I.h;
            const double rel_dual = sqrt(r2) / (1.0 + I.norm_c);
            const double rel_comp = sqrt(mn2) / (1.0 + sqrt(x2) + sqrt(z2));
            const double rel_primal = sqrt(ax2) / (1.0 + I.norm_b);
            const double rel = fmax(rel_dual, fmax(rel_comp, rel_primal));
            C->rel_dual = rel_dual;
            C->rel_comp = rel_comp;
            C->rel_primal = rel_primal;
            C->rel_kkt = rel;
            C->pobj = cx;                 // sum (r-c)^2 x-bar: unscaled <c, x-bar>
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
            } else if (rel <= C->tol) {
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

// Sigma update at a restart: sigma <- sqrt(sigma ||x-bar - x_r|| / ||z-bar - z_r||).
__global__ void __launch_bounds__(kThreads) k_restart_sigma(const WorkDev* __restrict__ W) {
    __shared__ double s_red[2 * 32];
    const int ninst = W->ninst;
    for (int i = blockIdx.x; i < ninst; i += gridDim.x) {
        const HotInst& I = W->inst[i];
        HotCtl* C = I.ctl;
        if (C->status != ST_RUNNING || !C->restart_pending) continue;
        const int ntile = 2 * I.S * I.nb;
        double v[2] = {0.0, 0.0};
        for (int q = threadIdx.x; q < ntile; q += blockDim.x) {
            v[0] += I.rst_part[(size_t)q * 2];
            v[1] += I.rst_part[(size_t)q * 2 + 1];
        }
        block_sum<2>(v, s_red);
        if (threadIdx.x == 0) {
            const double dx = sqrt(v[0]), dz = sqrt(v[1]);
            const double old = C->sigma;
            C->dx2 = v[0];
            C->dz2 = v[1];
            C->sigma_old = old;
            if (dx > 0.0 && dz > 0.0 && isfinite(dx / dz)) C->sigma = sqrt(old * (dx / dz));
            C->k = 0;
            C->r0 = -1.0;
            C->rprev = -1.0;
            C->restarts += 1;
        }
        __syncthreads();
    }
}

__global__ void k_block_end(const WorkDev* __restrict__ W) {
    const int ninst = W->ninst;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ninst; i += gridDim.x * blockDim.x) {
        HotCtl* C = W->inst[i].ctl;
        C->restart_pending = 0;
        C->just_finished = 0;
    }
}

// ------------------------------------------------------------- launchers --

LaunchDims make_launch_dims(int device) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (sms <= 0) sms = 1;
    LaunchDims d;
    d.grid_tile = sms * 4;
    d.grid_slab = sms * 4;
    d.grid_vec = sms * 4;
    d.grid_k1 = sms * 2;
    d.grid_inst = sms * 2;
    return d;
}

void launch_init(const HotInst& I, double sigma0, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tiles = 2 * I.S * I.nb;
    const int grid = tiles < sms * 4 ? tiles : sms * 4;
    if (I.fp64) k_init<double><<<grid, kThreads, 0, st>>>(I, sigma0);
    else k_init<float><<<grid, kThreads, 0, st>>>(I, sigma0);
    k_anchor_one<<<2 * I.S < sms * 4 ? 2 * I.S : sms * 4, kThreads, 0, st>>>(I, sigma0);
}

cudaError_t kernels_init(int device) {
    (void)device;
    cudaError_t e = cudaFuncSetAttribute(k_sweep<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kStages * kStageBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kStages * kStageBytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_marg, cudaFuncAttributeMaxDynamicSharedMemorySize, 7 * kMaxS * 8);
    return e;
}

void launch_solve_kernels(const WorkDev* w, const LaunchDims& ld, bool check, cudaStream_t st) {
    k_vec<<<ld.grid_vec, kThreads, 0, st>>>(w);
    k_marg<<<ld.grid_inst, kThreads, 7 * kMaxS * 8, st>>>(w);
    if (check) k_alpha<true><<<ld.grid_slab, kThreads, 0, st>>>(w);
    else k_alpha<false><<<ld.grid_slab, kThreads, 0, st>>>(w);
}

void launch_sweep(const WorkDev* w, const LaunchDims& ld, int fp64, int j, bool check, cudaStream_t st) {
    if (fp64) {
        if (check) k_sweep<double, true><<<ld.grid_tile, kThreads, 0, st>>>(w, j);
        else k_sweep<double, false><<<ld.grid_tile, kThreads, 0, st>>>(w, j);
    } else {
        if (check) k_sweep<float, true><<<ld.grid_tile, kThreads, kStages * kStageBytes, st>>>(w, j);
        else k_sweep<float, false><<<ld.grid_tile, kThreads, kStages * kStageBytes, st>>>(w, j);
    }
}

void launch_iteration(const WorkDev* w, const LaunchDims& ld, int fp64, int j, bool check, cudaStream_t st) {
    launch_solve_kernels(w, ld, check, st);
    launch_sweep(w, ld, fp64, j, check, st);
}

void launch_block_end(const WorkDev* w, const LaunchDims& ld, int fp64, int K, double a1, double a2, double a3,
                      cudaStream_t st) {
    k_kkt1<<<ld.grid_k1, kThreads, 0, st>>>(w);
    k_check<<<ld.grid_inst, kThreads, 0, st>>>(w, K, a1, a2, a3);
    if (fp64) {
        k_restart<double, 0><<<ld.grid_tile, kThreads, 0, st>>>(w);
        k_restart_sigma<<<ld.grid_inst, kThreads, 0, st>>>(w);
        k_restart<double, 1><<<ld.grid_tile, kThreads, 0, st>>>(w);
        k_anchor<<<ld.grid_slab, kThreads, 0, st>>>(w);
        k_restart<double, 2><<<ld.grid_tile, kThreads, 0, st>>>(w);
    } else {
        k_restart<float, 0><<<ld.grid_tile, kThreads, 0, st>>>(w);
        k_restart_sigma<<<ld.grid_inst, kThreads, 0, st>>>(w);
        k_restart<float, 1><<<ld.grid_tile, kThreads, 0, st>>>(w);
        k_anchor<<<ld.grid_slab, kThreads, 0, st>>>(w);
        k_restart<float, 2><<<ld.grid_tile, kThreads, 0, st>>>(w);
    }
    k_block_end<<<ld.grid_inst, kThreads, 0, st>>>(w);
}

}  // namespace hot
