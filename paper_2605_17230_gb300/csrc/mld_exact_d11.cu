// Compile-time specialised untruncated sweep for d = 11 (own translation
// unit so that the build compiles the distances in parallel).
#include "mld_exact_impl.cuh"

namespace mld {

int exact_fpw_11() { return exact::LayoutOf<11>::lay.floats_per_warp; }

bool launch_exact_11(const ExactArgs& a, cudaStream_t s, int warps_per_block, int precision) {
    return exact::launch_d<11>(a, s, warps_per_block, precision);
}

}  // namespace mld
