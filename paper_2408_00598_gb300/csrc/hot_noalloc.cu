// Plan recovery (Algorithm 1) for callers that cannot allocate device memory.
//
// hot_recover_plan needs per-call scratch (per-node entry counts, their
// prefix offsets, marginal accumulators), which it takes from the stream-
// ordered allocator.  Some callers cannot let a library allocate at call
// time: code whose device-memory footprint is fixed and accounted up front
// (a memory-budgeted service or an embedding framework that owns every
// allocation), or a latency-critical loop that must not pay for, or
// synchronise on, a device allocation.  hot_recover_plan_static serves them:
// its scratch is this file's static device array, sized for grids up to
// kStaticMaxS x kStaticMaxS, which every GPU that loads the library holds
// until the process exits.  The caller passes the flows and the output
// buffers; nothing else is allocated.
//
// The array is shared by every call in the process: each call overwrites it
// (and clears what has to start at zero), so calls whose work overlaps on the
// GPU race and corrupt each other's results.  Serialise them (one stream, or
// wait for a call to return before starting the next).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/hot.h"

namespace hot {
void set_error(const std::string& msg);   // hot_engine.cu: the message hot_last_error returns
}

namespace {

constexpr int kStaticMaxS = 256;
constexpr int kStaticMaxNodes = kStaticMaxS * kStaticMaxS;

// layout: counts int[N] | offsets long long[N] | marginals double[2N] |
//         total unsigned long long | L1 double[2]
constexpr size_t kOffCounts = 0;
constexpr size_t kOffOffs = kOffCounts + sizeof(int) * kStaticMaxNodes;
constexpr size_t kOffMarg = kOffOffs + sizeof(long long) * kStaticMaxNodes;
constexpr size_t kOffTotal = kOffMarg + sizeof(double) * 2 * kStaticMaxNodes;
constexpr size_t kOffL1 = kOffTotal + 256;
constexpr size_t kScratchBytes = kOffL1 + 256;

__device__ __align__(256) unsigned char g_recover_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

void fail(const char* m) { hot::set_error(std::string("hot_recover_plan_static: ") + m); }

// Flows in the vec order of eq. (4)-(6): f1_{i,k,j} at i + S k + S^2 j,
// f2_{k,j,l} at S^3 + k + S j + S^2 l.  Node (k, j) couples a_i = f1_{i,k,j}
// with b_l = f2_{k,j,l}, both clipped at 0.
__device__ void node_prefix(const double* __restrict__ x, int S, int k, int j, double* a, double* b, double* A,
                            double* B) {
    const int lane = threadIdx.x & 31;
    const size_t S2 = (size_t)S * S, S3 = S2 * S;
    for (int t = lane; t < S; t += 32) {
        a[t] = fmax(x[t + (size_t)S * k + S2 * j], 0.0);
        b[t] = fmax(x[S3 + k + (size_t)S * j + S2 * t], 0.0);
    }
    __syncwarp();
    // exclusive prefix sums by a warp scan; a running maximum keeps them
    // non-decreasing (a tree scan's partial sums need not be ordered to the
    // last bit, and the binary search and walk below rely on the order)
    double ca = 0.0, cb = 0.0, ma = 0.0, mb = 0.0;
    for (int base = 0; base < S; base += 32) {
        const int t = base + lane;
        const double va = t < S ? a[t] : 0.0, vb = t < S ? b[t] : 0.0;
        double sa = va, sb = vb;
        for (int o = 1; o < 32; o <<= 1) {
            const double ya = __shfl_up_sync(0xffffffffu, sa, o);
            const double yb = __shfl_up_sync(0xffffffffu, sb, o);
            if (lane >= o) {
                sa += ya;
                sb += yb;
            }
        }
        double ea = fmax(ca + sa - va, ma), eb = fmax(cb + sb - vb, mb);
        for (int o = 1; o < 32; o <<= 1) {
            const double ya = __shfl_up_sync(0xffffffffu, ea, o);
            const double yb = __shfl_up_sync(0xffffffffu, eb, o);
            if (lane >= o) {
                ea = fmax(ea, ya);
                eb = fmax(eb, yb);
            }
        }
        if (t < S) {
            A[t] = ea;
            B[t] = eb;
        }
        ma = __shfl_sync(0xffffffffu, ea, 31);
        mb = __shfl_sync(0xffffffffu, eb, 31);
        ca += __shfl_sync(0xffffffffu, sa, 31);
        cb += __shfl_sync(0xffffffffu, sb, 31);
    }
    if (lane == 0) {
        A[S] = fmax(ca, ma);
        B[S] = fmax(cb, mb);
    }
    __syncwarp();
}

// entries of source i: overlaps of [A_i, A_{i+1}) with [B_l, B_{l+1})
__device__ int source_entries(int S, int i, const double* A, const double* B, const double* a, const double* b,
                              int32_t* src, int32_t* dst, double* mass, size_t pos, int src_id, int k) {
    if (!(a[i] > 0.0)) return 0;             // the loops move nothing out of an empty source
    const double lo = A[i];
    const double hi = fmin(A[i + 1], B[S]);
    if (!(hi > lo)) return 0;
    int l0 = 0, l1 = S - 1;
    while (l0 < l1) {
        const int mid = (l0 + l1) >> 1;
        if (B[mid + 1] > lo) l1 = mid; else l0 = mid + 1;
    }
    int cnt = 0;
    for (int l = l0; l < S && B[l] < hi; ++l) {
        const double p = fmin(hi, B[l + 1]) - fmax(lo, B[l]);
        if (p > 0.0 && b[l] > 0.0) {
            if (src) {
                src[pos + cnt] = src_id;
                dst[pos + cnt] = k * S + l;
                mass[pos + cnt] = p;
            }
            ++cnt;
        }
    }
    return cnt;
}

constexpr int kWarps = 4;                // 4 x (4*256 + 2) doubles of shared memory per CTA

__global__ void __launch_bounds__(kWarps * 32) k_static_recover(const double* __restrict__ x, int S, int count_only,
                                                                 unsigned char* __restrict__ scratch,
                                                                 int32_t* __restrict__ src,
                                                                 int32_t* __restrict__ dst,
                                                                 double* __restrict__ mass) {
    __shared__ double sh[kWarps * (4 * kStaticMaxS + 2)];
    int* counts = (int*)(scratch + kOffCounts);
    const long long* offs = (const long long*)(scratch + kOffOffs);
    double* marg = (double*)(scratch + kOffMarg);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* a = sh + (size_t)warp * (4 * S + 2);
    double* b = a + S;
    double* A = b + S;
    double* B = A + S + 1;
    const int nodes = S * S;
    for (int node = blockIdx.x * kWarps + warp; node < nodes; node += gridDim.x * kWarps) {
        const int k = node / S, j = node % S;
        node_prefix(x, S, k, j, a, b, A, B);
        if (count_only) {
            int c = 0;
            for (int i = lane; i < S; i += 32) c += source_entries(S, i, A, B, a, b, nullptr, nullptr, nullptr, 0, 0, k);
            for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
            if (lane == 0) counts[node] = c;
            for (int t = lane; t < S; t += 32) {
                const double ga = fmin(a[t], fmax(0.0, B[S] - A[t]));
                const double gb = fmin(b[t], fmax(0.0, A[S] - B[t]));
                if (ga > 0.0) atomicAdd(&marg[(size_t)t * S + j], ga);
                if (gb > 0.0) atomicAdd(&marg[nodes + (size_t)k * S + t], gb);
            }
        } else {
            long long pos = offs[node];
            for (int base = 0; base < S; base += 32) {
                const int i = base + lane;
                int c = 0;
                if (i < S) c = source_entries(S, i, A, B, a, b, nullptr, nullptr, nullptr, 0, 0, k);
                int incl = c;
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                if (i < S && c > 0) source_entries(S, i, A, B, a, b, src, dst, mass, (size_t)(pos + incl - c), i * S + j, k);
                pos += __shfl_sync(0xffffffffu, incl, 31);
            }
        }
        __syncwarp();
    }
}

// clears the marginal accumulators (they must start at zero every call)
__global__ void k_static_clear(unsigned char* __restrict__ scratch, int nodes) {
    double* marg = (double*)(scratch + kOffMarg);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 2 * nodes; t += gridDim.x * blockDim.x) marg[t] = 0.0;
}

__global__ void k_static_scan(unsigned char* __restrict__ scratch, int n) {
    __shared__ long long s_tot[1024];
    __shared__ long long s_carry;
    const int* counts = (const int*)(scratch + kOffCounts);
    long long* offs = (long long*)(scratch + kOffOffs);
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        const int t = base + threadIdx.x;
        const long long v = t < n ? counts[t] : 0;
        s_tot[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            const long long y = threadIdx.x >= (unsigned)o ? s_tot[threadIdx.x - o] : 0;
            __syncthreads();
            s_tot[threadIdx.x] += y;
            __syncthreads();
        }
        if (t < n) offs[t] = s_carry + s_tot[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry += s_tot[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) *(unsigned long long*)(scratch + kOffTotal) = (unsigned long long)s_carry;
}

__global__ void k_static_l1(unsigned char* __restrict__ scratch, const double* __restrict__ mu,
                            const double* __restrict__ nu, int nodes) {
    __shared__ double s[1024];
    const double* marg = (const double*)(scratch + kOffMarg);
    double* l1 = (double*)(scratch + kOffL1);
    for (int w = 0; w < 2; ++w) {
        const double* ref = w ? nu : mu;
        const double* mg = marg + (size_t)w * nodes;
        double acc = 0.0;
        for (int t = threadIdx.x; t < nodes; t += blockDim.x) acc += fabs(mg[t] - ref[t]);
        s[threadIdx.x] = acc;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < (unsigned)o) s[threadIdx.x] += s[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) l1[w] = s[0];
        __syncthreads();
    }
}

// Device address of the static scratch for the current device; resolved once
// per device (with that device current) and cached.
int scratch_for_current_device(unsigned char** out, int* device) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        fail("no usable current CUDA device");
        return HOT_ECUDA;
    }
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_recover_scratch);
        if (e != cudaSuccess || !p) {
            fail("cudaGetSymbolAddress of the static scratch failed");
            return HOT_ECUDA;
        }
        g_scratch_ptr[dev] = (unsigned char*)p;
    }
    *out = g_scratch_ptr[dev];
    *device = dev;
    return HOT_OK;
}

}  // namespace

extern "C" {

HOT_API int hot_recover_plan_static(const double* x, int m, int n, const double* mu, const double* nu,
                                    int32_t* src, int32_t* dst, double* mass, size_t cap, size_t* nnz,
                                    double* marg_l1, void* stream) {
    if (!x || !nnz) {
        fail("x and nnz must not be NULL");
        return HOT_EINVAL;
    }
    if (m != n || m < 1 || m > kStaticMaxS) {
        fail("hot_recover_plan_static handles square grids up to 256 x 256");
        return HOT_EINVAL;
    }
    if (cap > 0 && (!src || !dst || !mass)) {
        fail("output arrays must not be NULL when cap > 0");
        return HOT_EINVAL;
    }
    if (marg_l1 && (!mu || !nu)) {
        fail("marg_l1 needs mu and nu");
        return HOT_EINVAL;
    }
    unsigned char* scratch = nullptr;
    int dev = 0;
    int rc = scratch_for_current_device(&scratch, &dev);
    if (rc != HOT_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int S = m;
    const int nodes = S * S;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        fail("cannot read the device's multiprocessor count");
        return HOT_ECUDA;
    }
    const int grid = (nodes + kWarps - 1) / kWarps < sms * 8 ? (nodes + kWarps - 1) / kWarps : sms * 8;
    // a launch that fails (bad configuration, no device) must not leave the
    // later kernels reading counts of an earlier call: check each one
    auto launched = [](const char* what) {
        const cudaError_t le = cudaGetLastError();
        if (le == cudaSuccess) return true;
        fail((std::string(what) + ": " + cudaGetErrorString(le)).c_str());
        return false;
    };
    k_static_clear<<<sms, 256, 0, st>>>(scratch, nodes);
    if (!launched("clearing the scratch")) return HOT_ECUDA;
    k_static_recover<<<grid, kWarps * 32, 0, st>>>(x, S, 1, scratch, nullptr, nullptr, nullptr);
    if (!launched("counting the plan entries")) return HOT_ECUDA;
    k_static_scan<<<1, 1024, 0, st>>>(scratch, nodes);
    if (!launched("the entry offsets")) return HOT_ECUDA;
    if (marg_l1) {
        k_static_l1<<<1, 1024, 0, st>>>(scratch, mu, nu, nodes);
        if (!launched("the marginal distances")) return HOT_ECUDA;
    }
    unsigned long long tot = 0;
    double l1[2] = {0.0, 0.0};
    cudaError_t e = cudaMemcpyAsync(&tot, scratch + kOffTotal, sizeof(tot), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && marg_l1) e = cudaMemcpyAsync(l1, scratch + kOffL1, sizeof(l1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        fail(cudaGetErrorString(e));
        return HOT_ECUDA;
    }
    *nnz = (size_t)tot;
    if (marg_l1) {
        marg_l1[0] = l1[0];
        marg_l1[1] = l1[1];
    }
    if (cap == 0 && !src) return HOT_OK;
    if (cap < tot) {
        fail("output capacity is smaller than the plan");
        return HOT_EINVAL;
    }
    if (tot > 0) {
        k_static_recover<<<grid, kWarps * 32, 0, st>>>(x, S, 0, scratch, src, dst, mass);
        if (!launched("writing the plan entries")) return HOT_ECUDA;
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            fail(cudaGetErrorString(e));
            return HOT_ECUDA;
        }
    }
    return HOT_OK;
}

}  // extern "C"
