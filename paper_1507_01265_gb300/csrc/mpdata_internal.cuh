// Internal declarations shared by the CUDA translation units of libmpdata.
// (Nothing here is part of the public ABI; see include/mpdata.h.)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mpdata.h"

namespace mpdata {

// Grid description passed by value to every kernel.
struct Grid {
    int nx, ny, nz;
    int per[3];  // 1 periodic, 0 rigid lid
};

// Map a cell index that is at most one grid length outside [0, n) into
// range: wrap on a periodic axis, clamp (zero-gradient ghost) on a lid axis.
__device__ __forceinline__ int cell_index(int a, int n, int per) {
    if (a >= 0 && a < n) return a;
    if (per) return a < 0 ? a + n : a - n;
    return a < 0 ? 0 : n - 1;
}

// Upstream flux through a face with velocity U between left value L and
// right value R: [U]+ L + [U]- R (a select; identical to the max/min form
// for finite values).
template <typename T>
__device__ __forceinline__ T upstream_flux(T U, T L, T R) {
    return U > T(0) ? U * L : U * R;
}

// Arguments of one grid for a fused tile body (FP32).
struct TileArgs {
    Grid g;
    int ntx;  // tiles per row of this grid
    int y0;   // grid row of tile row 0 (a band of rows; 0 for the whole grid)
    float eps;
    const float *h, *psi, *u1, *u2, *u3;
    float *out;
};

// One grid of a batched launch: both buffers of its psi ping-pong pair; the
// launch's parity picks which one is read.
struct BatchGrid {
    Grid g;
    int ntx;
    float eps;
    const float *h, *u1, *u2, *u3;
    float *buf[2];
};

__host__ __device__ inline TileArgs batch_args(const BatchGrid &b, int parity) {
    TileArgs a;
    a.g = b.g;
    a.ntx = b.ntx;
    a.y0 = 0;
    a.eps = b.eps;
    a.h = b.h; a.u1 = b.u1; a.u2 = b.u2; a.u3 = b.u3;
    a.psi = b.buf[parity];
    a.out = b.buf[parity ^ 1];
    return a;
}

// A batched launch with one CTA per work item, its grid table passed in the
// kernel parameters (constant bank) instead of global memory: the items form
// runs of consecutive tiles of one grid, CTA c belongs to the run r with
// start[r] <= c < start[r+1] and runs tile tile0[r] + c - start[r] of grid
// g[r].  A CTA's arguments are then uniform across its threads, as in a
// single-grid launch.  At most kDirectMaxRuns runs (about 28 KB of
// parameters, within the 32 KB limit).
constexpr int kDirectMaxRuns = 320;
struct DirectBatch {
    int nruns;
    int start[kDirectMaxRuns + 1];
    int tile0[kDirectMaxRuns];
    BatchGrid g[kDirectMaxRuns];
};
// kernel parameters are limited to 32764 bytes (with the parity int after it)
static_assert(sizeof(DirectBatch) + 8 <= 32764, "DirectBatch exceeds the kernel parameter limit");

// Launchers of the stage-per-kernel path (mpdata_stages.cu).
// Intermediates of the stage path; psi2 and w1..w3 (the second corrective
// pass's pseudo-velocities) only with three passes.
struct StageBuffers {
    void *psi1, *v1, *v2, *v3, *bup, *bdn;
    void *psi2, *w1, *w2, *w3;
};
cudaError_t launch_donor(int dtype, const Grid &g, const void *h, const void *psi, const void *w1,
                         const void *w2, const void *w3, void *out, cudaStream_t s);
cudaError_t launch_stage_step(int dtype, const Grid &g, int iterations, int nonosc, int extrema,
                              int precision, double eps, const void *h, const void *psi,
                              const void *u1, const void *u2, const void *u3, void *out,
                              const StageBuffers &b, cudaStream_t s);

// Fused step.  FP32 grids with a pair tile (32x16, 32x24, 32x28) run the
// two-columns-per-thread kernel (mpdata_fused2.cu); everything else runs the
// one-column kernel (mpdata_fused.cu).  Returns
// cudaErrorInvalidValue for a tile shape with no compiled instance.
cudaError_t launch_fused_step(int dtype, const Grid &g, int nonosc, double eps, int tile_x,
                              int tile_y, const void *h, const void *psi, const void *u1,
                              const void *u2, const void *u3, void *out, cudaStream_t s);
bool fused_tile_supported(int dtype, const Grid &g, int tile_x, int tile_y);
// nsm: SMs of the device (small grids with nx % 4 != 0 get one-column tiles).
void fused_default_tile(int dtype, const Grid &g, int nsm, int *tile_x, int *tile_y);
bool fused_pairs_supported(const Grid &g, int tile_x, int tile_y);
// Persistent batched launches (ncta CTAs; CTA c runs items [begin[c], begin[c+1])).
// ld: every grid of the launch has nx % 4 == 0 and the tile (24 or 28 rows)
// takes the two loader warps; tile_y 16 runs without them.
cudaError_t launch_fused_pairs_batch(int tile_x, int tile_y, int ld, int nonosc, int lid,
                                     const BatchGrid *grids, const int2 *items, const int *begin,
                                     int ncta, int parity, cudaStream_t s);
// One CTA per item, grid table in the parameters (d.start[d.nruns] CTAs).
cudaError_t launch_fused_pairs_direct(int tile_y, int ld, int nonosc, int lid, const DirectBatch &d,
                                      int parity, cudaStream_t s);
cudaError_t launch_fused_pairs(const Grid &g, int nonosc, double eps, int tile_x, int tile_y,
                               const void *h, const void *psi, const void *u1, const void *u2,
                               const void *u3, void *out, cudaStream_t s);
// Row bands of an FP32 grid with nx % 4 == 0: rows [0, 28 n28)
// in 32x28 tiles and [28 n28, ny) in 32x24 tiles (the last band may end past
// ny), launched concurrently on s and s2 (fork and join through the events)
// so that the hardware mixes the two tile sizes over the SMs.
struct BandPlan {
    int n28, n24;
};
// True when the default-tile model predicts the bands faster than the best
// single pair tile (waves x per-plane time) by at least 1 %.
bool fused_band_plan(const Grid &g, int nsm, BandPlan *plan);
cudaError_t launch_fused_bands(const Grid &g, int nonosc, double eps, const BandPlan &plan, const void *h,
                               const void *psi, const void *u1, const void *u2, const void *u3,
                               void *out, cudaStream_t s, cudaStream_t s2, cudaEvent_t ev_fork,
                               cudaEvent_t ev_join);

// Record the calling thread's last error message (mpdata_api.cu); returns code.
int set_error(int code, const char *message);

// Deterministic FP64 diagnostics (mpdata_reduce.cu).
constexpr int kReduceBlocks = 1024;  // fixed, so the summation tree never changes
cudaError_t launch_mass(int dtype, long long n, const void *h, const void *psi, double *partials,
                        double *out3, cudaStream_t s);
// Device address of the static partials array of mpdata_mass_noalloc on the
// current device (looked up on the first call per device).
cudaError_t noalloc_partials(double **out);
// out3[2] (and out3[1]) = max over cells of the outflow Courant number.
cudaError_t launch_courant_max(int dtype, const Grid &g, const void *h, const void *u1,
                               const void *u2, const void *u3, double *partials, double *out3,
                               cudaStream_t s);

}  // namespace mpdata
