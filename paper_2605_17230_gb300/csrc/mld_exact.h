// Launcher of the compile-time specialised kernel for untruncated chi.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mld {

struct ExactArgs {
    const uint64_t* dmask;     // [n][2][words]
    const float* noise;
    const uint64_t* syn;
    double* logP;
    int* status;
    int64_t B;
    int noise_mode;
    float* gws = nullptr;      // global workspace of gws_warps slices (nullptr: shared memory)
    int64_t gws_warps = 0;
};

// Distances with a specialised kernel (0 if none), its shared memory per warp
// (floats), and the launch (precision MLD_FP32 or MLD_MIXED_TF32); false if d
// has no specialised kernel or the launch failed.
int exact_floats_per_warp(int d);
bool launch_exact(int d, const ExactArgs& a, cudaStream_t s, int warps_per_block, int precision);

}  // namespace mld
