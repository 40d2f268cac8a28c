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

// Outflow Courant number of each cell, sum_d ([U_d(upper face)]+ -
// [U_d(lower face)]-) / h: the fraction of the cell's content the donor pass
// moves out in one step (it keeps psi >= 0 while this is <= 1).  Lid faces
// carry no velocity.  Maximum per block, then over blocks in a fixed tree.
template <typename T>
__global__ void k_courant_partial(Grid g, const T *__restrict__ h, const T *__restrict__ u1,
                                  const T *__restrict__ u2, const T *__restrict__ u3,
                                  double *__restrict__ part) {
    __shared__ double s[kThreads], mn[kThreads], mx[kThreads];
    const long long n = (long long)g.nx * g.ny * g.nz;
    const long long nxy = (long long)g.nx * g.ny;
    long long chunk = (n + gridDim.x - 1) / gridDim.x;
    long long lo = (long long)blockIdx.x * chunk;
    long long hi = lo + chunk < n ? lo + chunk : n;
    double best = 0.0;
    for (long long q = lo + threadIdx.x; q < hi; q += kThreads) {
        const int i = (int)(q % g.nx), j = (int)((q / g.nx) % g.ny), k = (int)(q / nxy);
        const T *u[3] = {u1, u2, u3};
        const int idx[3] = {i, j, k}, dim[3] = {g.nx, g.ny, g.nz};
        const long long stride[3] = {1, g.nx, nxy};
        double out = 0.0;
        for (int d = 0; d < 3; ++d) {
            const bool lid = !g.per[d];
            const double lower = (lid && idx[d] == 0) ? 0.0 : (double)u[d][q];
            double upper = 0.0;
            if (idx[d] + 1 < dim[d]) upper = (double)u[d][q + stride[d]];
            else if (!lid) upper = (double)u[d][q - (long long)(dim[d] - 1) * stride[d]];
            out += fmax(upper, 0.0) - fmin(lower, 0.0);
        }
        best = fmax(best, out / (double)h[q]);
    }
    s[threadIdx.x] = 0.0;
    mn[threadIdx.x] = best;
    mx[threadIdx.x] = best;
    __syncthreads();
    tree3(s, mn, mx);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 0] = 0.0;
        part[3 * blockIdx.x + 1] = mx[0];
        part[3 * blockIdx.x + 2] = mx[0];
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

cudaError_t launch_courant_max(int dtype, const Grid &g, const void *h, const void *u1,
                               const void *u2, const void *u3, double *partials, double *out3,
                               cudaStream_t s) {
    if (dtype == MPDATA_F64)
        k_courant_partial<double><<<kReduceBlocks, kThreads, 0, s>>>(
            g, (const double *)h, (const double *)u1, (const double *)u2, (const double *)u3, partials);
    else
        k_courant_partial<float><<<kReduceBlocks, kThreads, 0, s>>>(
            g, (const float *)h, (const float *)u1, (const float *)u2, (const float *)u3, partials);
    k_mass_final<<<1, kThreads, 0, s>>>(kReduceBlocks, partials, out3);
    return cudaGetLastError();
}

}  // namespace mpdata
