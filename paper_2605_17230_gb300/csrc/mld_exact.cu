// Launchers of the compile-time specialised untruncated sweep, d = 3..9
// (d = 11 and 13 are compiled in their own translation units).
#include "mld_exact_impl.cuh"

namespace mld {

bool launch_exact_11(const ExactArgs& a, cudaStream_t s, int warps_per_block, int precision);
bool launch_exact_13(const ExactArgs& a, cudaStream_t s, int warps_per_block, int precision);
int exact_fpw_11();
int exact_fpw_13();

int exact_floats_per_warp(int d) {
    switch (d) {
        case 3: return exact::LayoutOf<3>::lay.floats_per_warp;
        case 5: return exact::LayoutOf<5>::lay.floats_per_warp;
        case 7: return exact::LayoutOf<7>::lay.floats_per_warp;
        case 9: return exact::LayoutOf<9>::lay.floats_per_warp;
        case 11: return exact_fpw_11();
        case 13: return exact_fpw_13();
    }
    return 0;
}

bool launch_exact(int d, const ExactArgs& a, cudaStream_t s, int warps_per_block, int precision) {
    switch (d) {
        case 3: return exact::launch_d<3>(a, s, warps_per_block, precision);
        case 5: return exact::launch_d<5>(a, s, warps_per_block, precision);
        case 7: return exact::launch_d<7>(a, s, warps_per_block, precision);
        case 9: return exact::launch_d<9>(a, s, warps_per_block, precision);
        case 11: return launch_exact_11(a, s, warps_per_block, precision);
        case 13: return launch_exact_13(a, s, warps_per_block, precision);
    }
    return false;
}

}  // namespace mld
