// Internal structures shared by the host runtime and the CUDA kernels.
#pragma once

#include <stdint.h>

#include <utility>
#include <vector>

#include "../../include/mld.h"
#include "mld_plan.h"

struct mld_code {
    int d, n, m, words;
    std::vector<int32_t> stab_type;      // [m]
    std::vector<int32_t> stab_qubits;    // [m][4]
    std::vector<uint8_t> lx, lz;         // [n]
    std::vector<uint64_t> dmask;         // [n][2][words]: bit k set if T_k has x (z) at q
    // device copies
    uint64_t* d_dmask = nullptr;
    int* d_status = nullptr;
    struct PlanDev {
        int chi;
        mld::Plan plan;
        mld::SiteStep* d_steps;
    };
    std::vector<PlanDev> plans;
    // host-API staging
    void* h_stage_dev = nullptr;
    size_t h_stage_bytes = 0;
    // global workspace for states larger than a block's shared memory
    float* d_gws = nullptr;
    size_t gws_bytes = 0;
    // autotuned warps per CTA (resident warps per SM when the per-warp state
    // is in the global workspace), keyed by chi * 4 + precision
    std::vector<std::pair<int, int>> tuned;
    int force_warps = 0;                 // set only while mld_autotune times a candidate
    // workspace of the adjoint kernel
    float* d_gradws = nullptr;
    size_t gradws_bytes = 0;
    // rank-adaptive truncated sweep: per-block slices, the unit queue and
    // overflow list, the executed-flop counter, and the relative cutoff on
    // singular values (sigma_k <= svd_cutoff * sigma_1 is discarded)
    float* d_tws = nullptr;
    size_t tws_bytes = 0;
    void* d_tctl = nullptr;              // [0] u64 queue head, [8] int overflow count, [16] f64 flops
    int64_t* d_ovf = nullptr;
    int64_t ovf_cap = 0;
    float svd_cutoff = 1e-7f;
    // which kernel runs a truncating chi: 0 chosen per chi (autotuned, else by
    // the plan's size), 1 the rank-adaptive sweep, 2 the fixed-shape sweep;
    // trunc_tuned holds mld_autotune's choice per chi
    int trunc_kernel = 0;
    std::vector<std::pair<int, int>> trunc_tuned;
    // largest bond capacity of the rank-adaptive sweep's first pass (0: the
    // smallest that holds chi, up to 128; else 48, 64 or 128)
    int trunc_first_bond = 0;
    // which kernel runs an untruncated chi: 0 mld_autotune's choice for that
    // chi if it timed one (exact_tuned), else by d (the dense-state kernel at
    // d = 11, 13, the boundary-MPS kernel elsewhere); 1 the boundary-MPS
    // kernel; 2 the dense-state kernel (d = 9, 11, 13)
    int exact_kernel = 0;
    std::vector<std::pair<int, int>> exact_tuned;
    // Kac-Ward solver (mld_decode_xz): one device block holding the ordered
    // matrix of the spin graph (CSR row starts, columns, weight sources, each
    // band row's last column, the quarter-turn qubit map; then the phases as
    // double pairs at kw_ph_off; an executed-flop counter at kw_cnt_off),
    // built on first use, and its sizes
    void* d_kw = nullptr;
    int kw_N = 0, kw_Nb = 0, kw_bl = 0, kw_bu = 0, kw_nplaq = 0, kw_nnz = 0;
    size_t kw_ph_off = 0;
    size_t kw_cnt_off = 0;               // executed-flop counter (double) in the same block
};

namespace mld {
bool state_in_global_workspace(const mld_code* C, int chi);
bool uses_dense_exact(const mld_code* C, const Plan& P);
}
