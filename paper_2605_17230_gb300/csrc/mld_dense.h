// Launcher of the untruncated sweep with a dense boundary state (d = 11, 13).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mld_internal.h"

namespace mld {

struct DenseArgs {
    const uint64_t* dmask;     // [n][2][words]
    const float* noise;        // [n][4] (I, X, Y, Z) or [B] depolarizing p
    const uint64_t* syn;       // [B][words]
    double* logP;              // [B][4]
    int* status;               // status word (bits 1 << mld_status)
    int64_t B;
    int words, noise_mode;
};

// Distances with a dense-state kernel, its counted flops per syndrome (four
// classes), and the launch (one block per (syndrome, l_Z) unit, persistent
// over the units; asynchronous on s).
bool dense_exact_supported(int d);
double dense_exact_flops_per_syndrome(int d);
bool launch_dense_exact(int d, const DenseArgs& a, cudaStream_t s);

}  // namespace mld
