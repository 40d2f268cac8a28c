// Two-column kernel instances for 24-row tiles (kernels in mpdata_fused2.cuh).
#include "mpdata_fused2.cuh"

namespace mpdata {

cudaError_t pairs_rows_t24(const PairsRows &r) { return launch_rows<32, 24>(r); }

cudaError_t pairs_batch_t24(int ld, int nonosc, int lid, const BatchGrid *grids, const int2 *items,
                            const int *begin, int ncta, int parity, cudaStream_t s) {
    return ld ? launch_pairs_batch<32, 24, true>(nonosc, lid, grids, items, begin, ncta, parity, s)
              : launch_pairs_batch<32, 24, false>(nonosc, lid, grids, items, begin, ncta, parity, s);
}

cudaError_t pairs_direct_t24(int ld, int nonosc, int lid, const DirectBatch &d, int parity, cudaStream_t s) {
    return ld ? launch_pairs_direct<32, 24, true>(nonosc, lid, d, parity, s)
              : launch_pairs_direct<32, 24, false>(nonosc, lid, d, parity, s);
}

}  // namespace mpdata
