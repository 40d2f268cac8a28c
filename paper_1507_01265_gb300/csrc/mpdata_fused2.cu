// Fused MPDATA step, FP32, two adjacent x-columns per thread: the launches
// (single grid, row bands, batches) over the per-height entry points of
// mpdata_fused2_t<TY>.cu; the kernels are in mpdata_fused2.cuh.
#include "mpdata_fused2.cuh"

namespace mpdata {

bool fused_pairs_supported(const Grid &g, int tx, int ty) {
    (void)g;  // any nx: 16-byte loads when nx % 4 == 0, 4-byte loads otherwise
    // 16 rows: 360 threads at up to 128 registers; 24 and 28 rows with
    // nx % 4 == 0: 16 / 18 compute warps and two loader warps at 96
    return tx == 32 && (ty == 12 || ty == 16 || ty == 24 || ty == 28);
}

cudaError_t launch_fused_pairs(const Grid &g, int nonosc, double eps, int tx, int ty, const void *h,
                               const void *psi, const void *u1, const void *u2, const void *u3,
                               void *out, cudaStream_t s) {
    if (tx != 32 || !fused_pairs_supported(g, tx, ty)) return cudaErrorInvalidValue;
    const PairsRows r{g, nonosc, eps, 0, (g.ny + ty - 1) / ty, h, psi, u1, u2, u3, out, s};
    if (ty == 12) return pairs_rows_t12(r);
    if (ty == 16) return pairs_rows_t16(r);
    if (ty == 24) return pairs_rows_t24(r);
    return pairs_rows_t28(r);
}

cudaError_t launch_fused_bands(const Grid &g, int nonosc, double eps, const BandPlan &plan, const void *h,
                               const void *psi, const void *u1, const void *u2, const void *u3,
                               void *out, cudaStream_t s, cudaStream_t s2, cudaEvent_t ev_fork,
                               cudaEvent_t ev_join) {
    // nx % 4 == 0: both heights run with their loader warps
    if (g.nx % 4 != 0 || plan.n28 < 1 || plan.n24 < 1) return cudaErrorInvalidValue;
    cudaError_t e = cudaEventRecord(ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s2, ev_fork, 0);
    if (e != cudaSuccess) return e;
    if ((e = pairs_rows_t28(PairsRows{g, nonosc, eps, 0, plan.n28, h, psi, u1, u2, u3, out, s})) != cudaSuccess)
        return e;
    if ((e = pairs_rows_t24(PairsRows{g, nonosc, eps, 28 * plan.n28, plan.n24, h, psi, u1, u2, u3, out, s2})) !=
        cudaSuccess)
        return e;
    e = cudaEventRecord(ev_join, s2);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_join, 0);
    return e;
}

cudaError_t launch_fused_pairs_batch(int tx, int ty, int ld, int nonosc, int lid, const BatchGrid *grids,
                                     const int2 *items, const int *begin, int ncta, int parity,
                                     cudaStream_t s) {
    if (tx != 32) return cudaErrorInvalidValue;
    if (ty == 16 && !ld) return pairs_batch_t16(ld, nonosc, lid, grids, items, begin, ncta, parity, s);
    if (ty == 24) return pairs_batch_t24(ld, nonosc, lid, grids, items, begin, ncta, parity, s);
    if (ty == 28) return pairs_batch_t28(ld, nonosc, lid, grids, items, begin, ncta, parity, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_fused_pairs_direct(int ty, int ld, int nonosc, int lid, const DirectBatch &d, int parity,
                                      cudaStream_t s) {
    if (d.nruns < 1 || d.nruns > kDirectMaxRuns || d.start[d.nruns] < 1) return cudaErrorInvalidValue;
    if (ty == 16 && !ld) return pairs_direct_t16(ld, nonosc, lid, d, parity, s);
    if (ty == 24) return pairs_direct_t24(ld, nonosc, lid, d, parity, s);
    if (ty == 28) return pairs_direct_t28(ld, nonosc, lid, d, parity, s);
    return cudaErrorInvalidValue;
}

}  // namespace mpdata
