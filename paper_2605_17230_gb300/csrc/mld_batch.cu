// Mixed batches (jobs of different d, noise and chi), their capture into one
// CUDA graph, and the autotuner of the CTA shape.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "mld_checks.h"
#include "mld_dense.h"
#include "mld_internal.h"

namespace {

constexpr int kForks = 8;
constexpr int kMaxDevices = 64;

// Library-owned streams that a batch forks onto, per device.
struct ForkPool {
    bool ready = false;
    cudaStream_t s[kForks];
    cudaEvent_t done[kForks];
    cudaEvent_t start;
};

std::mutex g_pool_mutex;
ForkPool g_pools[kMaxDevices];

mld_status pool_for_current_device(ForkPool** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MLD_ERR_CUDA;
    ForkPool& p = g_pools[dev];
    if (!p.ready) {
        for (int i = 0; i < kForks; ++i) {
            if (cudaStreamCreateWithFlags(&p.s[i], cudaStreamNonBlocking) != cudaSuccess) return MLD_ERR_CUDA;
            if (cudaEventCreateWithFlags(&p.done[i], cudaEventDisableTiming) != cudaSuccess) return MLD_ERR_CUDA;
        }
        if (cudaEventCreateWithFlags(&p.start, cudaEventDisableTiming) != cudaSuccess) return MLD_ERR_CUDA;
        p.ready = true;
    }
    *out = &p;
    return MLD_OK;
}

}  // namespace

struct mld_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

mld_status mld_decode_batch(const mld_job* jobs, int n_jobs, void* stream) {
    mld::NvtxRange trace("mld_decode_batch");
    if (n_jobs < 0 || (n_jobs > 0 && !jobs)) return MLD_ERR_INVALID_ARG;
    for (int i = 0; i < n_jobs; ++i)
        if (!jobs[i].code) return MLD_ERR_INVALID_ARG;
    if (n_jobs == 0) return MLD_OK;
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    ForkPool* P = nullptr;
    mld_status st = pool_for_current_device(&P);
    if (st != MLD_OK) return st;
    // jobs of one code object share its workspace: same fork, in order
    std::vector<const mld_code*> owner;
    std::vector<int> fork(n_jobs);
    for (int i = 0; i < n_jobs; ++i) {
        int f = -1;
        for (size_t k = 0; k < owner.size(); ++k)
            if (owner[k] == jobs[i].code) f = (int)k % kForks;
        if (f < 0) {
            owner.push_back(jobs[i].code);
            f = (int)(owner.size() - 1) % kForks;
        }
        fork[i] = f;
    }
    const int used = owner.size() < (size_t)kForks ? (int)owner.size() : kForks;
    cudaStream_t origin = reinterpret_cast<cudaStream_t>(stream);
    if (cudaEventRecord(P->start, origin) != cudaSuccess) return MLD_ERR_CUDA;
    for (int f = 0; f < used; ++f)
        if (cudaStreamWaitEvent(P->s[f], P->start, 0) != cudaSuccess) return MLD_ERR_CUDA;
    for (int i = 0; i < n_jobs; ++i) {
        const mld_job& j = jobs[i];
        st = mld_decode(j.code, j.noise, j.noise_mode, j.syndromes, j.B, j.chi, j.precision, j.logP, j.argmax,
                        P->s[fork[i]]);
        if (st != MLD_OK) return st;
    }
    for (int f = 0; f < used; ++f) {
        if (cudaEventRecord(P->done[f], P->s[f]) != cudaSuccess) return MLD_ERR_CUDA;
        if (cudaStreamWaitEvent(origin, P->done[f], 0) != cudaSuccess) return MLD_ERR_CUDA;
    }
    return MLD_OK;
}

mld_status mld_graph_create(const mld_job* jobs, int n_jobs, mld_graph** out) {
    if (!out) return MLD_ERR_INVALID_ARG;
    *out = nullptr;
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return MLD_ERR_CUDA;
    // one uncaptured run allocates every plan and workspace first
    mld_status st = mld_decode_batch(jobs, n_jobs, cs);
    if (st == MLD_OK && cudaStreamSynchronize(cs) != cudaSuccess) st = MLD_ERR_CUDA;
    if (st != MLD_OK) {
        cudaStreamDestroy(cs);
        return st;
    }
    mld_graph* g = new mld_graph();
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = MLD_ERR_CUDA;
    if (st == MLD_OK) {
        const mld_status run = mld_decode_batch(jobs, n_jobs, cs);
        const cudaError_t e = cudaStreamEndCapture(cs, &g->graph);
        st = run != MLD_OK ? run : (e != cudaSuccess ? MLD_ERR_CUDA : MLD_OK);
    }
    if (st == MLD_OK && cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) st = MLD_ERR_CUDA;
    cudaStreamDestroy(cs);
    if (st != MLD_OK) {
        mld_graph_destroy(g);
        return st;
    }
    *out = g;
    return MLD_OK;
}

mld_status mld_graph_launch(mld_graph* g, void* stream) {
    mld::NvtxRange trace("mld_graph_launch");
    if (!g || !g->exec) return MLD_ERR_INVALID_ARG;
    return cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? MLD_OK : MLD_ERR_CUDA;
}

void mld_graph_destroy(mld_graph* g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

mld_status mld_autotune(const mld_code* Cc, int chi, int precision, int64_t sample_B, int* chosen) {
    mld_code* C = const_cast<mld_code*>(Cc);
    if (!C || chi < 1 || sample_B < 1) return MLD_ERR_INVALID_ARG;
    const int n = C->n, W = C->words;
    // synthetic sample: depolarizing p = 0.1, random syndromes (a fixed LCG)
    std::vector<float> noise(static_cast<size_t>(n) * 4);
    for (int q = 0; q < n; ++q) {
        noise[4 * q] = 0.9f;
        noise[4 * q + 1] = noise[4 * q + 2] = noise[4 * q + 3] = 0.1f / 3.f;
    }
    std::vector<uint64_t> syn(static_cast<size_t>(sample_B) * W);
    uint64_t x = 0x2545F4914F6CDD1DULL;
    for (auto& v : syn) {
        x = x * 6364136223846793005ULL + 1442695040888963407ULL;
        v = x;
    }
    const int m = C->m;
    for (int64_t b = 0; b < sample_B; ++b)         // clear the bits above n_stabs
        for (int w = 0; w < W; ++w) {
            const int lo = 64 * w;
            if (lo + 64 > m) syn[b * W + w] &= (m - lo) >= 64 ? ~0ULL : ((1ULL << (m - lo)) - 1);
        }
    float* dn = nullptr;
    uint64_t* ds = nullptr;
    double* dl = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    mld_status st = MLD_OK;
    if (cudaMalloc(&dn, noise.size() * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&ds, syn.size() * sizeof(uint64_t)) != cudaSuccess ||
        cudaMalloc(&dl, static_cast<size_t>(sample_B) * 4 * sizeof(double)) != cudaSuccess)
        st = MLD_ERR_NOMEM;
    if (st == MLD_OK &&
        (cudaMemcpy(dn, noise.data(), noise.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(ds, syn.data(), syn.size() * sizeof(uint64_t), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
         cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        st = MLD_ERR_CUDA;
    // candidates: warps per CTA of the fixed-shape or untruncated kernel
    // (global-workspace states: resident warps per SM 2, 4, 8, 16); for a
    // truncating chi the rank-adaptive sweep (kernel 1) as well; for an
    // untruncated chi at d = 9, 11, 13 the dense-state kernel as well
    const bool truncating = mld::make_plan(C->d, chi).svd_sites != 0;
    const bool dense_cand = !truncating && mld::dense_exact_supported(C->d) && C->exact_kernel == 0;
    const int saved_kernel = C->trunc_kernel, saved_exact = C->exact_kernel;
    if (dense_cand) C->exact_kernel = 1;          // the boundary-MPS kernel's shapes
    const int wscale = mld::state_in_global_workspace(C, chi) ? 2 : 1;
    int best_cand = 0, best_w = 0, best_k = 0;
    bool have = false;
    float best_ms = 0.f;
    for (int cand = truncating ? 0 : (dense_cand ? -1 : 1); st == MLD_OK && cand <= 4; ++cand) {
        const int kern = cand == 0 ? 1 : 2, w = cand < 0 ? 0 : (cand == 0 ? 4 : wscale << (cand - 1));
        C->trunc_kernel = truncating ? kern : saved_kernel;
        C->exact_kernel = dense_cand ? (cand < 0 ? 2 : 1) : saved_exact;
        C->force_warps = cand <= 0 ? 0 : w;
        mld_status r = mld_decode(C, dn, MLD_NOISE_TABLE, ds, sample_B, chi, precision, dl, nullptr, s);
        if (r != MLD_OK) { st = r; break; }
        cudaEventRecord(e0, s);
        for (int rep = 0; rep < 3; ++rep)
            mld_decode(C, dn, MLD_NOISE_TABLE, ds, sample_B, chi, precision, dl, nullptr, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) { st = MLD_ERR_CUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (!have || ms < best_ms) { have = true; best_cand = cand; best_w = w; best_k = kern; best_ms = ms; }
    }
    C->force_warps = 0;
    C->trunc_kernel = saved_kernel;
    C->exact_kernel = saved_exact;
    if (st == MLD_OK && have) {
        bool found = false;
        if (best_w > 0) {
            const int key = chi * 4 + precision;
            for (auto& kv : C->tuned)
                if (kv.first == key) { kv.second = best_w; found = true; }
            if (!found) C->tuned.emplace_back(key, best_w);
        }
        if (truncating) {
            found = false;
            for (auto& kv : C->trunc_tuned)
                if (kv.first == chi) { kv.second = best_k; found = true; }
            if (!found) C->trunc_tuned.emplace_back(chi, best_k);
        }
        if (dense_cand) {
            const int which = best_cand < 0 ? 2 : 1;
            found = false;
            for (auto& kv : C->exact_tuned)
                if (kv.first == chi) { kv.second = which; found = true; }
            if (!found) C->exact_tuned.emplace_back(chi, which);
        }
        if (chosen) *chosen = best_w;
        if (mld_decode_status(C) != MLD_OK) st = MLD_ERR_NUMERIC;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(dn);
    cudaFree(ds);
    cudaFree(dl);
    return st;
}

}  // extern "C"
