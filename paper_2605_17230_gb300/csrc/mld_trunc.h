// Launcher of the rank-adaptive truncated sweep (one warp per unit).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mld {

// Capacities of one unit's shapes and global slice (floats). The first pass
// over all units runs on every resident warp with the smallest that hold
// chi (bond 48, 64 or 128: 2.25, 4.5 or 17.8 MB per warp); units that exceed
// them are decoded by a second pass with the large ones on few warps.
struct TruncCaps {
    int max_bond;        // kept bond per cut
    int max_rows;        // carry rows
    int64_t mps;         // one boundary MPS, compact
    int64_t q;           // one column's reflectors and taus, compact
    int64_t spill;       // a site's work buffers when they do not fit on chip
    __host__ __device__ int64_t slice() const { return 2 * mps + q + spill; }
};
constexpr TruncCaps kTruncSmall{48, 192, 128 * 1024, 256 * 1024, 64 * 1024};
constexpr TruncCaps kTruncMid{64, 256, 256 * 1024, 512 * 1024, 128 * 1024};
constexpr TruncCaps kTruncLarge{128, 512, 1024 * 1024, 2048 * 1024, 384 * 1024};

struct TruncArgs {
    const uint64_t* dmask;           // [n][2][words]
    const float* noise;              // [n][4] or [B]
    const uint64_t* syn;             // [B][words]
    double* logP;                    // [B][4]
    int* status;                     // status word (bits 1 << mld_status)
    int64_t B;
    int d, n, words, noise_mode;
    int chi;                         // cap on every new bond
    float cutoff;                    // keep sigma_k > cutoff * sigma_1 (relative)
    int arena;                       // on-chip work arena per unit (floats)
    TruncCaps caps;                  // shape and slice capacities of this pass
    float* ws;                       // per-unit global slices of caps.slice() floats
    unsigned long long* next_unit;   // work queue head (zeroed before the launch)
    const int64_t* in_list;          // units to decode (nullptr: all 2B units)
    const int* in_count;             // number of entries of in_list
    int64_t* ovf_list;               // units whose shapes exceed the capacities
    int* ovf_count;                  // (zeroed before the launch)
    double* flops;                   // executed flop counter (added to)
    unsigned long long* bond_hist;   // [65]: kept bonds k of every truncating cut (k >= 64 in the last bin)
};

// Units (warps) per block, dynamic shared memory per block for an arena of
// `arena` floats per unit, resident blocks per SM (0 on error), and the launch.
int trunc_units_per_block();
size_t trunc_smem_bytes(int arena);
int trunc_blocks_per_sm(int arena);
bool launch_trunc(const TruncArgs& a, int blocks, cudaStream_t s);

}  // namespace mld
