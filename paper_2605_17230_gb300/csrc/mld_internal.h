// Internal structures shared by the host runtime and the CUDA kernels.
#pragma once

#include <stdint.h>

#include <vector>

#include "../../include/mld.h"

namespace mld {

constexpr int kMaxD = 25;
constexpr int kMaxN = kMaxD * kMaxD;
constexpr int kMaxSynWords = (kMaxN - 1 + 63) / 64;

// Right-sweep factorisation of the bond matrix T (rows x cols) of one site.
enum RMode : int16_t {
    R_IDENT = 0,   // cols <= rows, cols <= chi: site = identity, carry = T
    R_DENSE = 1,   // rows < cols, rows <= chi: site = T, carry = identity
    R_SVD = 2      // chi < min(rows, cols): truncated SVD keeps chi values
};

// One site i (plaquette row i, 0..d) of one column transfer c.
//
// Left sweep (apply the column MPO and bring the result to left-canonical
// form): the carry C[kappa][a*Dl + r] (K rows; a = alpha_{i-1}; r = old bond
// left of site i) is contracted with the old site A[r][a'*Dr + r'] and the
// qubit factor of qubit (i-1, c), w(alpha_{i-1}, alpha_i, beta_{i-1}, beta_i),
// giving for each beta_i = b' one block M^{b'}[kappa][a'*Dr + r'] (K x ncol).
// A tall block (K > ncol) is QR-factored; otherwise Q = I and R = M.
// The new carry stacks the R^{b'} blocks: row kappa' = b'*kq + j.
//
// Gauge. A column with no truncating bond (every right-sweep factorisation
// keeps min(rows, cols)) needs no canonical form: its tall blocks are kept
// as they are (site = M, carry = identity), so every tensor of the column
// stays entrywise non-negative and FP32 keeps relative accuracy in every
// coset. Only columns that truncate (canon = 1) are QR-canonicalised, since
// the SVD truncation is optimal only against a left-isometric left part.
struct SiteStep {
    int16_t pam, pa, pb;    // dims of alpha_{i-1} (1 at i = 0), alpha_i, beta_i
    int16_t Dl, Dr;         // old MPS bonds left and right of site i
    int16_t K;              // rows of the M blocks (= rows of the incoming carry)
    int16_t ncol;           // columns of an M block: pa*Dr, or 1 at i = d (alpha_d summed)
    int16_t kq;             // min(K, ncol)
    int16_t kq_prev;        // kq of site i-1 (beta_{i-1} = kappa / kq_prev); 1 at i = 0
    int16_t tall;           // K > ncol
    int16_t parity;         // (i-1 + c) & 1: orientation of the qubit factor
    int16_t qubit;          // (i-1)*d + c, or -1 at i = 0
    int16_t rmode;          // right-sweep factorisation (RMode)
    int16_t S;              // new bond right of site i
    int16_t Sl;             // new bond left of site i
    int32_t offA;           // old site A in the MPS buffer (floats)
    int32_t offQ;           // tall: blocks at offQ + b*K*ncol, tau at offQ + pb*K*ncol + b*ncol
    int32_t offN;           // new site (Sl x pb x S) in the MPS buffer
    int16_t canon;          // column is QR-canonicalised (it has an R_SVD site)
    int16_t cid;            // incoming carry is an identity (skip the GEMM)
};

struct Plan {
    int d = 0, chi = 0;
    int steps_per_col = 0;            // d + 1
    std::vector<SiteStep> steps;      // d * (d+1), column-major
    // per-warp shared-memory layout (floats, 4-aligned)
    int off_w = 0, off_mps = 0, off_buf0 = 0, off_buf1 = 0, off_q = 0, off_svd = 0;
    int floats_per_warp = 0;
    int max_buf = 0, max_mps = 0, max_q = 0, max_svd = 0;
    int svd_sites = 0;                // number of sites that truncate
    double flops_per_coset = 0.0;     // counted flops of this schedule (see plan.cpp)
    int init_sizes[kMaxD + 1];        // initial product-state site sizes
};

Plan make_plan(int d, int chi);

}  // namespace mld

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
};
