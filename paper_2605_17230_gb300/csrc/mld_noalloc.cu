// Decoding entry point that allocates no device memory.
//
// Some callers cannot allocate device memory: a real-time decoding loop that
// must not stall on the implicit device-wide synchronisation of cudaMalloc,
// or a process whose device memory is already fully reserved by another
// framework's caching allocator. mld_decode allocates its code tables and
// status word on first use; this variant instead keeps that scratch in one
// file-scope __device__ array of fixed size, which every GPU that loads the
// library holds until the process exits. The caller still passes inputs and
// outputs in its own device memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "mld_checks.h"
#include "mld_exact.h"
#include "mld_internal.h"

namespace {

// Scratch layout: [0, 256) status word, [256, ...) per-qubit destabiliser
// masks of the code, n * 2 * syn_words uint64 (enough for d <= 11).
constexpr size_t kNoAllocBytes = 16384;
constexpr size_t kStatusSlot = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};
// FNV-1a hash of the destabiliser tables last written to each device's
// scratch array (0: none yet), so that consecutive calls for one code skip
// the upload; calls are serialised by the caller, as the array is shared
uint64_t g_tables_written[kMaxDevices] = {};

uint64_t table_hash(const std::vector<uint64_t>& t) {
    uint64_t h = 1469598103934665603ULL;
    for (uint64_t w : t)
        for (int k = 0; k < 8; ++k) {
            h ^= (w >> (8 * k)) & 0xffu;
            h *= 1099511628211ULL;
        }
    return h | 1ULL;                 // never 0
}

__global__ void noalloc_argmax(const double* __restrict__ logP, uint8_t* __restrict__ am, int64_t B) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const double* l = logP + 4 * b;
    int best = 0;
    for (int k = 1; k < 4; ++k)
        if (l[k] > l[best]) best = k;
    am[b] = (uint8_t)best;
}

// Device address of the scratch array for the current device. In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
mld_status scratch_address(unsigned char** out, int* device) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MLD_ERR_CUDA;
    *device = dev;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MLD_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    return MLD_OK;
}

}  // namespace

extern "C" mld_status mld_decode_noalloc(const mld_code* C, const float* noise, int noise_mode,
                                         const uint64_t* syndromes, int64_t B, int chi, int precision,
                                         double* logP, uint8_t* argmax, void* stream, int check_status) {
    mld::NvtxRange trace("mld_decode_noalloc");
    if (!C || B < 0 || chi < 1) return MLD_ERR_INVALID_ARG;
    if (noise_mode != MLD_NOISE_TABLE && noise_mode != MLD_NOISE_DEPOL) return MLD_ERR_INVALID_ARG;
    if (precision != MLD_FP32 && precision != MLD_MIXED_BF16 && precision != MLD_MIXED_TF32)
        return MLD_ERR_INVALID_ARG;
    if (B == 0) return MLD_OK;
    if (!noise || !syndromes || !logP) return MLD_ERR_INVALID_ARG;
    if (noise_mode == MLD_NOISE_TABLE && (reinterpret_cast<uintptr_t>(noise) & 15)) return MLD_ERR_INVALID_ARG;
    // only the untruncated FP32 sweep of the distances with a specialised
    // kernel, and only codes whose tables fit in the scratch array
    const size_t table_bytes = C->dmask.size() * sizeof(uint64_t);
    if (precision != MLD_FP32 || C->d > 11 || mld::exact_floats_per_warp(C->d) == 0 ||
        mld::make_plan(C->d, chi).svd_sites != 0 || kStatusSlot + table_bytes > kNoAllocBytes)
        return MLD_ERR_UNSUPPORTED;
    unsigned char* scratch = nullptr;
    int device = 0;
    mld_status st = scratch_address(&scratch, &device);
    if (st != MLD_OK) return st;
    int dev = 0, max_optin = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
        return MLD_ERR_CUDA;
    const size_t pw = (size_t)mld::exact_floats_per_warp(C->d) * sizeof(float);
    if (pw > (size_t)max_optin) return MLD_ERR_UNSUPPORTED;
    int W = 1, best = 0;
    for (int w = 1; w <= 8; ++w) {
        if (pw * w > (size_t)max_optin) break;
        int ctas = (int)((size_t)per_sm / (pw * w + 1024));
        ctas = ctas < 32 ? ctas : 32;
        const int warps = ctas * w < 64 ? ctas * w : 64;
        if (warps > best) { best = warps; W = w; }
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the status word starts at zero in every call; the tables are uploaded
    // only when the array holds another code's (the previous call's code is
    // remembered per device)
    if (cudaMemsetAsync(scratch, 0, sizeof(int), s) != cudaSuccess) return MLD_ERR_CUDA;
    const uint64_t tables = table_hash(C->dmask);
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (g_tables_written[device] != tables) {
            if (cudaMemcpyAsync(scratch + kStatusSlot, C->dmask.data(), table_bytes, cudaMemcpyHostToDevice, s) !=
                cudaSuccess)
                return MLD_ERR_CUDA;
            g_tables_written[device] = tables;
        }
    }
    if (!mld::launch_noise_check(noise, noise_mode, noise_mode == MLD_NOISE_TABLE ? C->n : B,
                                 reinterpret_cast<int*>(scratch), s))
        return MLD_ERR_CUDA;
    mld::ExactArgs ea;
    ea.dmask = reinterpret_cast<const uint64_t*>(scratch + kStatusSlot);
    ea.noise = noise;
    ea.syn = syndromes;
    ea.logP = logP;
    ea.status = reinterpret_cast<int*>(scratch);
    ea.B = B;
    ea.noise_mode = noise_mode;
    if (!mld::launch_exact(C->d, ea, s, W, MLD_FP32)) return MLD_ERR_CUDA;
    if (argmax) {
        noalloc_argmax<<<(unsigned)((B + 255) / 256), 256, 0, s>>>(logP, argmax, B);
        if (cudaGetLastError() != cudaSuccess) return MLD_ERR_CUDA;
    }
    if (!check_status) return MLD_OK;
    int h = 0;
    if (cudaMemcpyAsync(&h, scratch, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return MLD_ERR_CUDA;
    if (h & (1 << MLD_ERR_INVALID_ARG)) return MLD_ERR_INVALID_ARG;
    if (h & (1 << MLD_ERR_NUMERIC)) return MLD_ERR_NUMERIC;
    if (h & (1 << MLD_ERR_TIMEOUT)) return MLD_ERR_TIMEOUT;
    return MLD_OK;
}
