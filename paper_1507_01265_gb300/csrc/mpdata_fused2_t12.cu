// Two-column kernel instances for 12-row tiles (kernels in mpdata_fused2.cuh).
#include "mpdata_fused2.cuh"

namespace mpdata {

cudaError_t pairs_rows_t12(const PairsRows &r) { return launch_rows<32, 12>(r); }

}  // namespace mpdata
