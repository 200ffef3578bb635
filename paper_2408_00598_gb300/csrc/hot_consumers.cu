// Consumers of a recovered transport plan: the barycentric projection used
// by colour transfer (Sec. IV-B and App. G of arXiv 2408.00598).
//
// A plan is a list of entries (s, t, pi) in device memory (Algorithm 1's
// output from hot_recover_plan).  Source bin s is sent to
//     T(s) = sum_t pi(s, t) y_t / sum_t pi(s, t),
// y_t a D-vector per target bin.  One streaming pass accumulates numerator
// and weight per source with FP64 atomic adds in L2 (the entries of one
// source are spread over the m nodes (k, j) it ships through, so a segmented
// sum would need an m-fold partial array); a second pass divides.  The order
// of the atomic adds is not fixed, so results are reproducible to rounding
// (about 1e-16 relative per entry), not bit for bit.
#include "hot_internal.h"
#include "hot_engine.h"

#include <string>

namespace hot {

namespace {

constexpr int kBaryMaxD = 8;

__global__ void __launch_bounds__(256) k_bary_acc(const int* __restrict__ src, const int* __restrict__ dst,
                                                  const double* __restrict__ mass, size_t nnz,
                                                  const double* __restrict__ y, int ndst, int D,
                                                  double* __restrict__ num, double* __restrict__ w, int nsrc,
                                                  int* __restrict__ bad) {
    int nbad = 0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nnz; e += (size_t)gridDim.x * blockDim.x) {
        const int s = src[e], t = dst[e];
        const double p = mass[e];
        if (s < 0 || s >= nsrc || t < 0 || t >= ndst) {   // reported, never dereferenced
            ++nbad;
            continue;
        }
        atomicAdd(&w[s], p);
        for (int d = 0; d < D; ++d) atomicAdd(&num[(size_t)s * D + d], p * y[(size_t)t * D + d]);
    }
    if (nbad) atomicAdd(bad, nbad);
}

__global__ void __launch_bounds__(256) k_bary_div(double* __restrict__ num, const double* __restrict__ w, int nsrc,
                                                  int D) {
    const size_t n = (size_t)nsrc * D;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const double ws = w[q / D];
        num[q] = ws > 0.0 ? num[q] / ws : 0.0;
    }
}

}  // namespace

int barycentric_map(const int* src, const int* dst, const double* mass, size_t nnz, const double* y, int ndst,
                    int D, double* out, double* weight, int nsrc, cudaStream_t st) {
    if (D < 1 || D > kBaryMaxD || nsrc < 0 || ndst < 0) {
        set_error("barycentric map: D must be in [1, 8] and the bin counts non-negative");
        return HOT_EINVAL;
    }
    if ((nnz > 0 && (!src || !dst || !mass || !y)) || (nsrc > 0 && (!out || !weight))) {
        set_error("barycentric map: null pointer");
        return HOT_EINVAL;
    }
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    int* d_bad = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&d_bad, sizeof(int), st);
    if (e != cudaSuccess) {
        set_error(std::string("barycentric map: ") + cudaGetErrorString(e));
        return HOT_ENOMEM;
    }
    int h_bad = 0;
    e = cudaMemsetAsync(d_bad, 0, sizeof(int), st);
    if (e == cudaSuccess && nsrc > 0) e = cudaMemsetAsync(out, 0, (size_t)nsrc * D * sizeof(double), st);
    if (e == cudaSuccess && nsrc > 0) e = cudaMemsetAsync(weight, 0, (size_t)nsrc * sizeof(double), st);
    if (e == cudaSuccess && nnz > 0) {
        k_bary_acc<<<sms * 8, 256, 0, st>>>(src, dst, mass, nnz, y, ndst, D, out, weight, nsrc, d_bad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && nsrc > 0) {
        k_bary_div<<<sms * 4, 256, 0, st>>>(out, weight, nsrc, D);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(d_bad, st);
    if (e != cudaSuccess) {
        set_error(std::string("barycentric map failed on the device: ") + cudaGetErrorString(e));
        return HOT_ECUDA;
    }
    if (h_bad) {
        set_error("barycentric map: " + std::to_string(h_bad) + " entries with a bin index out of range (skipped)");
        return HOT_EINVAL;
    }
    return HOT_OK;
}

}  // namespace hot
