// Device-side validation of decode inputs, and host-side trace ranges.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

namespace mld {

// A Pauli channel's probabilities are non-negative and sum to one (Sec. 2.2).
// Checks `count` rows of a noise table (MLD_NOISE_TABLE: float[count][4], finite,
// non-negative, each row summing to 1 within 1e-6) or `count` depolarizing
// strengths (MLD_NOISE_DEPOL: 0 <= p <= 1) on the stream, and sets bit
// MLD_ERR_INVALID_ARG of the status word for any violation. False if the
// launch failed.
bool launch_noise_check(const float* noise, int noise_mode, int64_t count, int* status, cudaStream_t s);

// Named range on the calling thread's NVTX timeline around a C-ABI call
// (profilers show the enqueue of each decode; with no tool attached the
// push and pop cost a few nanoseconds).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace mld
