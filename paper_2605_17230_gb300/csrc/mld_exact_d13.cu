// Compile-time specialised untruncated sweep for d = 13 (own translation
// unit so that the build compiles the distances in parallel).
#include "mld_exact_impl.cuh"

namespace mld {

int exact_fpw_13() { return exact::LayoutOf<13>::lay.floats_per_warp; }

bool launch_exact_13(const ExactArgs& a, cudaStream_t s, int warps_per_block, int precision) {
    return exact::launch_d<13>(a, s, warps_per_block, precision);
}

}  // namespace mld
