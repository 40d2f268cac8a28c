// Diagnostics of a state: total mass sum(h*psi) in FP64, min psi, max psi.
//
// Determinism: the cell range is cut into kReduceBlocks fixed contiguous
// chunks; each block sums its chunk in a fixed per-thread order and a fixed
// shared-memory tree, and a single block then folds the partials in a fixed
// tree.  No atomics touch the values, so the result is bit-identical from
// run to run (and independent of the launch order of the blocks).
#include <float.h>

#include <mutex>

#include "mpdata_internal.cuh"

namespace mpdata {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void tree3(double *s, double *mn, double *mx) {
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s[threadIdx.x] += s[threadIdx.x + w];
            mn[threadIdx.x] = fmin(mn[threadIdx.x], mn[threadIdx.x + w]);
            mx[threadIdx.x] = fmax(mx[threadIdx.x], mx[threadIdx.x + w]);
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void k_mass_partial(long long n, const T *__restrict__ h, const T *__restrict__ psi,
                               double *__restrict__ part) {
    __shared__ double s[kThreads], mn[kThreads], mx[kThreads];
    long long chunk = (n + gridDim.x - 1) / gridDim.x;
    long long lo = (long long)blockIdx.x * chunk;
    long long hi = lo + chunk < n ? lo + chunk : n;
    double acc = 0.0, lo_v = DBL_MAX, hi_v = -DBL_MAX;
    for (long long q = lo + threadIdx.x; q < hi; q += kThreads) {
        double p = (double)psi[q];
        acc += (double)h[q] * p;
        lo_v = fmin(lo_v, p);
        hi_v = fmax(hi_v, p);
    }
    s[threadIdx.x] = acc;
    mn[threadIdx.x] = lo_v;
    mx[threadIdx.x] = hi_v;
    __syncthreads();
    tree3(s, mn, mx);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 0] = s[0];
        part[3 * blockIdx.x + 1] = mn[0];
        part[3 * blockIdx.x + 2] = mx[0];
    }
}

__global__ void k_mass_final(int nparts, const double *__restrict__ part, double *__restrict__ out3) {
    __shared__ double s[kThreads], mn[kThreads], mx[kThreads];
    double acc = 0.0, lo_v = DBL_MAX, hi_v = -DBL_MAX;
    for (int b = threadIdx.x; b < nparts; b += kThreads) {
        acc += part[3 * b + 0];
        lo_v = fmin(lo_v, part[3 * b + 1]);
        hi_v = fmax(hi_v, part[3 * b + 2]);
    }
    s[threadIdx.x] = acc;
    mn[threadIdx.x] = lo_v;
    mx[threadIdx.x] = hi_v;
    __syncthreads();
    tree3(s, mn, mx);
    if (threadIdx.x == 0) {
        out3[0] = s[0];
        out3[1] = mn[0];
        out3[2] = mx[0];
    }
}

// Scratch of mpdata_mass_noalloc: the per-block partials live in this
// file-scope device array instead of a cudaMalloc'd buffer.  Every GPU that
// loads the library holds it (24 KiB) until the process exits.  In host code
// the name is only a stand-in; its device address comes from
// cudaGetSymbolAddress, looked up once per device.
static __device__ __align__(256) double g_noalloc_partials[3 * kReduceBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[kMaxDevices];

}  // namespace

cudaError_t noalloc_partials(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);  // this device is current
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = (double *)p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

cudaError_t launch_mass(int dtype, long long n, const void *h, const void *psi, double *partials,
                        double *out3, cudaStream_t s) {
    if (dtype == MPDATA_F64)
        k_mass_partial<double><<<kReduceBlocks, kThreads, 0, s>>>(n, (const double *)h,
                                                                   (const double *)psi, partials);
    else
        k_mass_partial<float><<<kReduceBlocks, kThreads, 0, s>>>(n, (const float *)h,
                                                                  (const float *)psi, partials);
    k_mass_final<<<1, kThreads, 0, s>>>(kReduceBlocks, partials, out3);
    return cudaGetLastError();
}

}  // namespace mpdata
