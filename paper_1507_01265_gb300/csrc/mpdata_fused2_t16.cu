// Two-column kernel instances for 16-row tiles (kernels in mpdata_fused2.cuh).
#include "mpdata_fused2.cuh"

namespace mpdata {

cudaError_t pairs_rows_t16(const PairsRows &r) { return launch_rows<32, 16>(r); }

cudaError_t pairs_batch_t16(int ld, int nonosc, int lid, const BatchGrid *grids, const int2 *items,
                            const int *begin, int ncta, int parity, cudaStream_t s) {
    if (ld) return cudaErrorInvalidValue;  // no loader warps at 16 rows
    return launch_pairs_batch<32, 16, false>(nonosc, lid, grids, items, begin, ncta, parity, s);
}

cudaError_t pairs_direct_t16(int ld, int nonosc, int lid, const DirectBatch &d, int parity, cudaStream_t s) {
    if (ld) return cudaErrorInvalidValue;
    return launch_pairs_direct<32, 16, false>(nonosc, lid, d, parity, s);
}

}  // namespace mpdata
