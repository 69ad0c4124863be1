// Launcher of the dense adjoint for untruncated sweeps, d = 3..13.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mld {

struct GradDenseArgs {
    const uint64_t* dmask;     // [n][2][words]
    const float* noise;        // [n][4] (I, X, Y, Z)
    const uint64_t* syn;       // [B][words]
    const double* dlogP;       // [B][4] or nullptr
    double* logP;              // [B][4] or nullptr
    double* dnoise;            // [n][4], accumulated
    float* lws;                // per block: the stored left states, then 4n double partial sums
                               // (grad_dense_workspace_floats each)
    int64_t B;
    int words;
};

// Distances with a dense adjoint kernel.
bool grad_dense_supported(int d);
// Resident blocks the launch uses on a device with `sms` SMs, and the floats
// of global workspace each needs (the left states of one unit and the
// block's partial gradient sums).
int64_t grad_dense_blocks(int d, int sms, int64_t B);
int64_t grad_dense_workspace_floats(int d);
bool launch_grad_dense(int d, const GradDenseArgs& a, int64_t blocks, cudaStream_t s);

}  // namespace mld
