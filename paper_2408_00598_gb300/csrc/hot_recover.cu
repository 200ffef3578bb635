// Algorithm 1 of arXiv 2408.00598 on the GPU: the transport plan from the
// reduced-model flows, one intermediate node (k, j) per warp ("parallelise the
// (k, j) loop", Remark after Prop. 1).
//
// For node (k, j), Algorithm 1's inner loops (i = 1..m, then l = 1..n, move
// min(f1_{i,k,j}, f2_{k,j,l}) and subtract it from both) are the north-west-
// corner coupling of the sources a_i = f1_{i,k,j} with the sinks
// b_l = f2_{k,j,l}: with exclusive prefix sums A_i, B_l, the mass moved from i
// to l is the overlap of [A_i, A_{i+1}) and [B_l, B_{l+1}), and mass beyond
// min(sum a, sum b) is left unassigned exactly as the sequential loop leaves
// it.  Each lane takes a set of sources i, finds its first sink by binary
// search and walks forward; entries are written in (node, i, l) order.
// Flows are clipped at 0 first (an approximate solution may have small
// negative entries).  In the slab layout both a and b are contiguous rows:
// a = row k of f1 slab j (m sources i), b = row j of f2 slab k (n sinks l).
// A plan entry runs from source bin (i, j), index i n + j of mu, to target bin
// (k, l), index k n + l of nu.
#include "hot_engine.h"
#include "hot_df.cuh"

namespace hot {

constexpr int kRecWarps = 8;

// shared memory of one warp in k_recover_df, in floats: a (m floats), b (n
// floats), padded to an even count, and the pairs A (m + 1), B (n + 1)
__host__ __device__ constexpr size_t recover_df_words(int m, int n) {
    return (size_t)m + n + ((m + n) & 1) + 2 * ((size_t)m + 1) + 2 * ((size_t)n + 1);
}
// the same for k_recover, in doubles
__host__ __device__ constexpr size_t recover_words(int m, int n) { return 2 * ((size_t)m + n) + 2; }

// first entries of f1 row k of slab j and of f2 row j of slab k; a slab's
// rows are stored at a pitch of its side rounded up to a multiple of 4
__host__ __device__ constexpr int row_pitch(int side) { return (side + 3) & ~3; }
__device__ __forceinline__ size_t node_row_a(int m, int k, int j) { return ((size_t)j * m + k) * row_pitch(m); }
__device__ __forceinline__ size_t node_row_b(int m, int n, int k, int j) {
    return (size_t)n * m * row_pitch(m) + ((size_t)k * n + j) * row_pitch(n);
}

template <typename T>
__device__ __forceinline__ void load_node(const T* __restrict__ x, int m, int n, int k, int j, double* a, double* b,
                                          double* A, double* B) {
    const int lane = threadIdx.x & 31;
    const T* ra = x + node_row_a(m, k, j);
    const T* rb = x + node_row_b(m, n, k, j);
    for (int t = lane; t < m; t += 32) a[t] = fmax((double)ra[t], 0.0);
    for (int t = lane; t < n; t += 32) b[t] = fmax((double)rb[t], 0.0);
    __syncwarp();
    // exclusive prefix sums, sequential per 32-chunk with a warp scan (FP64);
    // a tree scan's partial sums need not be ordered to the last bit, so a
    // running maximum keeps A and B non-decreasing (the walk relies on it)
    double carryA = 0.0, carryB = 0.0, runA = 0.0, runB = 0.0;
    const int L = m > n ? m : n;
    for (int base = 0; base < L; base += 32) {
        const int t = base + lane;
        double va = t < m ? a[t] : 0.0, vb = t < n ? b[t] : 0.0;
        double sa = va, sb = vb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double ya = __shfl_up_sync(0xffffffffu, sa, o);
            const double yb = __shfl_up_sync(0xffffffffu, sb, o);
            if (lane >= o) {
                sa += ya;
                sb += yb;
            }
        }
        double ea = fmax(carryA + sa - va, runA), eb = fmax(carryB + sb - vb, runB);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double ya = __shfl_up_sync(0xffffffffu, ea, o);
            const double yb = __shfl_up_sync(0xffffffffu, eb, o);
            if (lane >= o) {
                ea = fmax(ea, ya);
                eb = fmax(eb, yb);
            }
        }
        if (t < m) A[t] = ea;
        if (t < n) B[t] = eb;
        runA = __shfl_sync(0xffffffffu, ea, 31);
        runB = __shfl_sync(0xffffffffu, eb, 31);
        carryA += __shfl_sync(0xffffffffu, sa, 31);
        carryB += __shfl_sync(0xffffffffu, sb, 31);
    }
    if (lane == 0) {
        A[m] = fmax(carryA, runA);
        B[n] = fmax(carryB, runB);
    }
    __syncwarp();
}

// number of sinks (of n) overlapping source i (and optionally write them)
__device__ __forceinline__ int node_source(int n, int i, const double* A, const double* B, const double* a,
                                           const double* b, int32_t* src, int32_t* dst, double* mass, size_t pos,
                                           int src_id, int node_k) {
    if (!(a[i] > 0.0)) return 0;             // the loops move nothing out of an empty source
    const double lo = A[i];
    const double hi = fmin(A[i + 1], B[n]);
    if (!(hi > lo)) return 0;
    // first l with B[l+1] > lo
    int l0 = 0, l1 = n - 1;
    while (l0 < l1) {
        const int mid = (l0 + l1) >> 1;
        if (B[mid + 1] > lo) l1 = mid; else l0 = mid + 1;
    }
    int cnt = 0;
    for (int l = l0; l < n && B[l] < hi; ++l) {
        const double p = fmin(hi, B[l + 1]) - fmax(lo, B[l]);
        if (p > 0.0 && b[l] > 0.0) {
            if (src) {
                src[pos + cnt] = src_id;
                dst[pos + cnt] = node_k * n + l;
                mass[pos + cnt] = p;
            }
            ++cnt;
        }
    }
    return cnt;
}

template <typename T>
__global__ void __launch_bounds__(kRecWarps * 32) k_recover(const T* __restrict__ x, int m, int n, int count_only,
                                                            int* __restrict__ counts,
                                                            const long long* __restrict__ offs,
                                                            int32_t* __restrict__ src, int32_t* __restrict__ dst,
                                                            double* __restrict__ mass, double* __restrict__ marg1,
                                                            double* __restrict__ marg2) {
    extern __shared__ double sh[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    double* a = sh + (size_t)warp * recover_words(m, n);
    double* b = a + m;
    double* A = b + n;
    double* B = A + m + 1;
    const int nodes = m * n;
    for (int node = blockIdx.x * nw + warp; node < nodes; node += gridDim.x * nw) {
        const int k = node / n, j = node % n;    // k-major node order
        load_node(x, m, n, k, j, a, b, A, B);
        if (count_only) {
            int c = 0;
            for (int i = lane; i < m; i += 32) c += node_source(n, i, A, B, a, b, nullptr, nullptr, nullptr, 0, 0, k);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
            if (lane == 0) counts[node] = c;
            // marginals of the plan: source (i, j) gets min(a_i, max(0, Btot - A_i)),
            // target (k, l) gets min(b_l, max(0, Atot - B_l))
            for (int t = lane; t < m; t += 32) {
                const double ga = fmin(a[t], fmax(0.0, B[n] - A[t]));
                if (ga > 0.0) atomicAdd(&marg1[(size_t)t * n + j], ga);
            }
            for (int t = lane; t < n; t += 32) {
                const double gb = fmin(b[t], fmax(0.0, A[m] - B[t]));
                if (gb > 0.0) atomicAdd(&marg2[(size_t)k * n + t], gb);
            }
        } else {
            long long pos = offs[node];
            for (int base = 0; base < m; base += 32) {
                const int i = base + lane;
                int c = 0;
                if (i < m) c = node_source(n, i, A, B, a, b, nullptr, nullptr, nullptr, 0, 0, k);
                int incl = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                if (i < m && c > 0)
                    node_source(n, i, A, B, a, b, src, dst, mass, (size_t)(pos + incl - c), i * n + j, k);
                pos += __shfl_sync(0xffffffffu, incl, 31);
            }
        }
        __syncwarp();
    }
}

// FP32 bulk mode: the same node procedure with the prefix sums, comparisons
// and overlaps of the FP32 flows in double-float pairs (FP64 arithmetic runs
// at a small fraction of the FP32 rate on this part; a pair holds the sum of
// FP32 values to about 48 bits, as a running FP64 sum of them does).
__device__ __forceinline__ bool df_lt(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ DF df_min(DF a, DF b) { return df_lt(b, a) ? b : a; }
__device__ __forceinline__ DF df_max(DF a, DF b) { return df_lt(a, b) ? b : a; }
__device__ __forceinline__ bool df_pos(DF a) { return a.hi > 0.f || (a.hi == 0.f && a.lo > 0.f); }
__device__ __forceinline__ DF df_shfl_up(DF a, int o) {
    return DF{__shfl_up_sync(0xffffffffu, a.hi, o), __shfl_up_sync(0xffffffffu, a.lo, o)};
}
__device__ __forceinline__ DF df_shfl(DF a, int l) {
    return DF{__shfl_sync(0xffffffffu, a.hi, l), __shfl_sync(0xffffffffu, a.lo, l)};
}

__device__ __forceinline__ void load_node_df(const float* __restrict__ x, int m, int n, int k, int j, float* a,
                                             float* b, float2* A, float2* B) {
    const int lane = threadIdx.x & 31;
    const float* ra = x + node_row_a(m, k, j);
    const float* rb = x + node_row_b(m, n, k, j);
    for (int t = lane; t < m; t += 32) a[t] = fmaxf(ra[t], 0.f);
    for (int t = lane; t < n; t += 32) b[t] = fmaxf(rb[t], 0.f);
    __syncwarp();
    // prefix sums of non-negative entries never decrease, but the rounding of
    // sums formed in different orders (the scan tree) can make a later one
    // smaller by an ulp; a running maximum restores the order the merge walk
    // relies on (ma, mb: maxima of the chunks done so far)
    DF ca{0.f, 0.f}, cb{0.f, 0.f}, ma{0.f, 0.f}, mb{0.f, 0.f};
    const int L = m > n ? m : n;
    for (int base = 0; base < L; base += 32) {
        const int t = base + lane;
        DF sa{t < m ? a[t] : 0.f, 0.f}, sb{t < n ? b[t] : 0.f, 0.f};
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const DF ya = df_shfl_up(sa, o), yb = df_shfl_up(sb, o);
            if (lane >= o) {
                sa = df_add(sa, ya);
                sb = df_add(sb, yb);
            }
        }
        DF ea = df_shfl_up(sa, 1), eb = df_shfl_up(sb, 1);       // exclusive within the chunk
        if (lane == 0) ea = eb = DF{0.f, 0.f};
        DF pa = df_max(df_add(ca, ea), ma), pb = df_max(df_add(cb, eb), mb);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const DF ya = df_shfl_up(pa, o), yb = df_shfl_up(pb, o);
            if (lane >= o) {
                pa = df_max(pa, ya);
                pb = df_max(pb, yb);
            }
        }
        if (t < m) A[t] = df_st(pa);
        if (t < n) B[t] = df_st(pb);
        ma = df_shfl(pa, 31);
        mb = df_shfl(pb, 31);
        ca = df_add(ca, df_shfl(sa, 31));
        cb = df_add(cb, df_shfl(sb, 31));
    }
    if (lane == 0) {
        A[m] = df_st(df_max(ca, ma));
        B[n] = df_st(df_max(cb, mb));
    }
    __syncwarp();
}

// The node's coupling as a merge of the source ends A[1..m] with the sink
// ends B[1..n] (ties: source first).  After the first d merged ends the walk
// stands at source p, sink q = d - p; the step from there moves the overlap
// min(A[p+1], B[q+1]) - max(A[p], B[q]) from source p to sink q (an entry
// when positive and both the source and the sink hold mass) and passes the
// nearer end.  These are the pairs and masses of the north-west-corner loops
// of Algorithm 1, in (i, l) order.  A lane takes a
// contiguous range of steps and finds its start by a binary search on the
// merge diagonal (merge path), so a node costs about log2(m + n) +
// (m + n)/32 steps per lane.
__device__ __forceinline__ int merge_split(const float2* A, const float2* B, int m, int n, int d) {
    int lo = d - n > 0 ? d - n : 0, hi = d < m ? d : m;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        // source end mid + 1 is among the first d ends iff it is <= sink end d - mid
        if (!df_lt(df_ld(B[d - mid]), df_ld(A[mid + 1]))) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ int merge_walk(const float2* A, const float2* B, const float* a, const float* b, int m,
                                          int n, int p, int q, int steps, int32_t* src, int32_t* dst, double* mass,
                                          size_t pos, int j, int k) {
    int cnt = 0;
    for (int t = 0; t < steps && p < m && q < n; ++t) {
        const DF ae = df_ld(A[p + 1]), be = df_ld(B[q + 1]);
        const DF ov = df_sub(df_min(ae, be), df_max(df_ld(A[p]), df_ld(B[q])));
        if (df_pos(ov) && a[p] > 0.f && b[q] > 0.f) {
            if (src) {
                src[pos + cnt] = p * n + j;
                dst[pos + cnt] = k * n + q;
                mass[pos + cnt] = df_val(ov);
            }
            ++cnt;
        }
        if (!df_lt(be, ae)) ++p;
        else ++q;
    }
    return cnt;
}

__global__ void __launch_bounds__(kRecWarps * 32) k_recover_df(const float* __restrict__ x, int m, int n,
                                                               int count_only,
                                                               int* __restrict__ counts,
                                                               const long long* __restrict__ offs,
                                                               int32_t* __restrict__ src, int32_t* __restrict__ dst,
                                                               double* __restrict__ mass, double* __restrict__ marg1,
                                                               double* __restrict__ marg2) {
    extern __shared__ float4 shdf[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    const size_t per = recover_df_words(m, n);           // floats per warp
    float* a = reinterpret_cast<float*>(shdf) + (size_t)warp * per;
    float* b = a + m;
    float2* A = reinterpret_cast<float2*>(b + n + ((m + n) & 1));
    float2* B = A + m + 1;
    const int nodes = m * n;
    const int span = (m + n + 31) / 32;                  // merge steps per lane
    const int d0 = lane * span < m + n ? lane * span : m + n;
    const int d1 = d0 + span < m + n ? d0 + span : m + n;
    for (int node = blockIdx.x * nw + warp; node < nodes; node += gridDim.x * nw) {
        const int k = node / n, j = node % n;    // k-major node order
        load_node_df(x, m, n, k, j, a, b, A, B);
        const int p0 = d0 < d1 ? merge_split(A, B, m, n, d0) : m;
        int c = merge_walk(A, B, a, b, m, n, p0, d0 - p0, d1 - d0, nullptr, nullptr, nullptr, 0, j, k);
        if (count_only) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
            if (lane == 0) counts[node] = c;
            const DF At = df_ld(A[m]), Bt = df_ld(B[n]);
            for (int t = lane; t < m; t += 32) {
                DF ra = df_sub(Bt, df_ld(A[t]));
                if (!df_pos(ra)) ra = DF{0.f, 0.f};
                const DF ga = df_min(DF{a[t], 0.f}, ra);
                if (df_pos(ga)) atomicAdd(&marg1[(size_t)t * n + j], df_val(ga));
            }
            for (int t = lane; t < n; t += 32) {
                DF rb = df_sub(At, df_ld(B[t]));
                if (!df_pos(rb)) rb = DF{0.f, 0.f};
                const DF gb = df_min(DF{b[t], 0.f}, rb);
                if (df_pos(gb)) atomicAdd(&marg2[(size_t)k * n + t], df_val(gb));
            }
        } else {
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (c > 0)
                merge_walk(A, B, a, b, m, n, p0, d0 - p0, d1 - d0, src, dst, mass, (size_t)(offs[node] + incl - c), j,
                           k);
        }
        __syncwarp();
    }
}

// exclusive scan of `n` ints into long long offsets (single block, chunked)
__global__ void k_scan(const int* __restrict__ counts, long long* __restrict__ offs, int n,
                       unsigned long long* __restrict__ total) {
    __shared__ long long s_tot[1024];
    __shared__ long long s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        const int t = base + threadIdx.x;
        const long long v = t < n ? counts[t] : 0;
        s_tot[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            long long y = threadIdx.x >= (unsigned)o ? s_tot[threadIdx.x - o] : 0;
            __syncthreads();
            s_tot[threadIdx.x] += y;
            __syncthreads();
        }
        if (t < n) offs[t] = s_carry + s_tot[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry += s_tot[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = (unsigned long long)s_carry;
}

__global__ void k_marg_l1(const double* __restrict__ marg, const double* __restrict__ mu, int M,
                          double* __restrict__ out) {
    __shared__ double s[1024];
    double acc = 0.0;
    for (int t = threadIdx.x; t < M; t += blockDim.x) acc += fabs(marg[t] - mu[t]);
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < (unsigned)o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

// x-bar from the slab layout into the paper's vec order (eq. 4-6):
// f1_{i,k,j} at i + m k + m^2 j (same as slab j, row k, col i);
// f2_{k,j,l} at n m^2 + k + m j + m n l (slab n + k, row j, col l); the
// slab rows sit at their padded pitch.
template <typename T>
__global__ void k_export(const T* __restrict__ x, int m, int n, double* __restrict__ out) {
    const size_t half = (size_t)m * m * n;
    const size_t V = half + (size_t)m * n * n;
    const size_t mp = row_pitch(m), np = row_pitch(n);
    // one thread per entry of the paper's order (coalesced writes)
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < V; q += (size_t)gridDim.x * blockDim.x) {
        if (q < half) {                           // f1_{i,k,j} at i + m k + m^2 j: slab j, row k, column i
            const size_t i = q % m, k = (q / m) % m, j = q / ((size_t)m * m);
            out[q] = (double)x[(j * m + k) * mp + i];
        } else {                                  // f2_{k,j,l} at k + m j + m n l: slab n + k, row j, column l
            const size_t p = q - half;
            const size_t k = p % m, j = (p / m) % n, l = p / ((size_t)m * n);
            out[q] = (double)x[(size_t)n * m * mp + (k * n + j) * np + l];
        }
    }
}

int export_flows(Inst* I, double* x, int space, cudaStream_t st) {
    const int m = I->m, n = I->n;
    const size_t V = (size_t)m * n * (m + n);
    double* dst = x;
    double* tmp = nullptr;
    if (space == HOT_SPACE_HOST) {
        HOT_CK(cudaMallocAsync(&tmp, V * 8, st));
        dst = tmp;
    }
    const int grid = 1024;
    if (I->fp64) k_export<double><<<grid, 256, 0, st>>>((const double*)I->desc.xr, m, n, dst);
    else k_export<float><<<grid, 256, 0, st>>>((const float*)I->desc.xr, m, n, dst);
    HOT_CK(cudaGetLastError());
    if (tmp) {
        HOT_CK(cudaMemcpyAsync(x, tmp, V * 8, cudaMemcpyDeviceToHost, st));
        cudaFreeAsync(tmp, st);
    }
    HOT_CK(cudaStreamSynchronize(st));
    return HOT_OK;
}

int recover_plan(Ctx* ctx, Inst* I, int32_t* src, int32_t* dst, double* mass, int space, size_t cap, size_t* nnz,
                 double* marg_l1, cudaStream_t st) {
    (void)ctx;
    const int m = I->m, n = I->n;
    const int nodes = m * n;
    int* counts = nullptr;
    long long* offs = nullptr;
    unsigned long long* dtot = nullptr;
    double* marg = nullptr;
    double* l1 = nullptr;
    HOT_CK(cudaMallocAsync(&counts, sizeof(int) * nodes, st));
    HOT_CK(cudaMallocAsync(&offs, sizeof(long long) * nodes, st));
    HOT_CK(cudaMallocAsync(&dtot, sizeof(unsigned long long), st));
    HOT_CK(cudaMallocAsync(&marg, sizeof(double) * 2 * nodes, st));
    HOT_CK(cudaMallocAsync(&l1, sizeof(double) * 2, st));
    HOT_CK(cudaMemsetAsync(marg, 0, sizeof(double) * 2 * nodes, st));
    // warps per CTA: each holds a, b and their prefix sums (2(m + n) + 2
    // doubles; FP32 mode: m + n floats and m + n + 2 float pairs)
    const size_t per_warp =
        I->fp64 ? recover_words(m, n) * sizeof(double) : recover_df_words(m, n) * sizeof(float);
    const int nw = std::max(1, std::min(kRecWarps, (int)((200 * 1024) / per_warp)));
    const size_t shm = (size_t)nw * per_warp;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_recover_df, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_recover<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    const int grid = std::max(1, std::min((nodes + nw - 1) / nw, sms * 8));
    if (I->fp64)
        k_recover<double><<<grid, nw * 32, shm, st>>>((const double*)I->desc.xr, m, n, 1, counts, nullptr,
                                                              nullptr, nullptr, nullptr, marg, marg + nodes);
    else
        k_recover_df<<<grid, nw * 32, shm, st>>>((const float*)I->desc.xr, m, n, 1, counts, nullptr, nullptr, nullptr,
                                                 nullptr, marg, marg + nodes);
    HOT_CK(cudaGetLastError());
    k_scan<<<1, 1024, 0, st>>>(counts, offs, nodes, dtot);
    unsigned long long tot = 0;
    HOT_CK(cudaMemcpyAsync(&tot, dtot, sizeof(tot), cudaMemcpyDeviceToHost, st));
    HOT_CK(cudaStreamSynchronize(st));
    *nnz = (size_t)tot;
    int rc = HOT_OK;
    if (marg_l1) {
        // marginals against mu1 (row-major (i, j)) and mu2 (row-major (k, l))
        k_marg_l1<<<1, 1024, 0, st>>>(marg, I->desc.mu1, nodes, l1);
        k_marg_l1<<<1, 1024, 0, st>>>(marg + nodes, I->desc.mu2, nodes, l1 + 1);
        HOT_CK(cudaMemcpyAsync(marg_l1, l1, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
    }
    if (cap > 0 || src || dst || mass) {
        if (cap < tot) {
            rc = HOT_EINVAL;
            set_error("output capacity " + std::to_string(cap) + " < plan size " + std::to_string(tot));
        } else if (tot > 0) {
            int32_t *ds = src, *dd = dst;
            double* dm = mass;
            if (space == HOT_SPACE_HOST) {
                HOT_CK(cudaMallocAsync(&ds, sizeof(int32_t) * tot, st));
                HOT_CK(cudaMallocAsync(&dd, sizeof(int32_t) * tot, st));
                HOT_CK(cudaMallocAsync(&dm, sizeof(double) * tot, st));
            }
            if (I->fp64)
                k_recover<double><<<grid, nw * 32, shm, st>>>((const double*)I->desc.xr, m, n, 0, counts, offs,
                                                                      ds, dd, dm, nullptr, nullptr);
            else
                k_recover_df<<<grid, nw * 32, shm, st>>>((const float*)I->desc.xr, m, n, 0, counts, offs, ds, dd, dm,
                                                         nullptr, nullptr);
            HOT_CK(cudaGetLastError());
            if (space == HOT_SPACE_HOST) {
                HOT_CK(cudaMemcpyAsync(src, ds, sizeof(int32_t) * tot, cudaMemcpyDeviceToHost, st));
                HOT_CK(cudaMemcpyAsync(dst, dd, sizeof(int32_t) * tot, cudaMemcpyDeviceToHost, st));
                HOT_CK(cudaMemcpyAsync(mass, dm, sizeof(double) * tot, cudaMemcpyDeviceToHost, st));
                cudaFreeAsync(ds, st);
                cudaFreeAsync(dd, st);
                cudaFreeAsync(dm, st);
            }
        }
    }
    cudaFreeAsync(counts, st);
    cudaFreeAsync(offs, st);
    cudaFreeAsync(dtot, st);
    cudaFreeAsync(marg, st);
    cudaFreeAsync(l1, st);
    HOT_CK(cudaStreamSynchronize(st));
    return rc;
}

}  // namespace hot
