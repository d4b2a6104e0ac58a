// gcp_loss_est_noalloc: the fixed-sample loss estimate without any memory
// allocation by the library.
//
// The ordinary gcp_loss_est keeps its per-block partial sums in scratch that
// gcp_create allocated with cudaMalloc.  This variant keeps them in a
// file-scope device array instead, so it needs no handle and allocates
// nothing.  It serves callers that must not call cudaMalloc when they run
// the estimate: hosts whose device memory is owned by another allocator (a
// framework's caching allocator that has reserved the GPU's memory), and
// loops that forbid allocation after start-up (real-time or latency-bound
// services), where a cudaMalloc would stall or fail.
//
// The array (kNoAllocBlocks partial sums plus a completion ticket, about
// 8 KB) lives in every GPU that loads this library until the process exits,
// and all calls share it: two calls whose kernels overlap on the GPU (on
// different streams, or on different host threads) race on it and give
// wrong results.
#include <cstddef>
#include <mutex>

#include "../../include/gcp.h"
#include "gcp_kernels.cuh"

namespace {

constexpr int kNoAllocBlocks = 1024;
constexpr int kNoAllocThreads = 256;

struct NoAllocScratch {
    double partials[kNoAllocBlocks];
    unsigned int ticket;
};

__device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Device address of g_noalloc_scratch, looked up once per device with that
// device current.  In host code the symbol's name is only a host-side stand-in.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
NoAllocScratch* g_scratch_addr[kMaxDevices] = {};

gcp_status scratch_for_current_device(NoAllocScratch** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GCP_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        // the array's device address on this device; the array itself starts
        // zeroed (module load) and every call clears the ticket it uses
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return GCP_ERR_CUDA;
        g_scratch_addr[dev] = static_cast<NoAllocScratch*>(p);
    }
    *out = g_scratch_addr[dev];
    return GCP_OK;
}

bool aligned_to(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

extern "C" gcp_status gcp_loss_est_noalloc(int32_t d, const gcp_factors* F, gcp_loss loss, const gcp_samples* list,
                                           double* out_dev, gcp_stream_t stream)
{
    using namespace gcpk;
    if (d < 2 || d > GCP_MAX_MODES || !F || !list || !out_dev || !aligned_to(out_dev, 8)) return GCP_ERR_INVALID_ARG;
    if (loss < GCP_LOSS_GAUSSIAN || loss > GCP_LOSS_BETA_HALF) return GCP_ERR_INVALID_ARG;
    if (F->rank < 1 || F->rank > 256 || F->ld < F->rank || F->ld % 4 != 0) return GCP_ERR_INVALID_ARG;
    for (int k = 0; k < d; ++k) {
        const void* a = F->bf16 ? static_cast<const void*>(F->A_bf16[k]) : static_cast<const void*>(F->A[k]);
        if (!a || !aligned_to(a, F->bf16 ? 8 : 16)) return GCP_ERR_INVALID_ARG;
    }
    if (list->n < 0 || list->n > static_cast<int64_t>(kNoAllocBlocks) * kNoAllocThreads) return GCP_ERR_INVALID_ARG;
    if (list->n > 0) {
        for (int k = 0; k < d; ++k)
            if (!list->idx[k]) return GCP_ERR_INVALID_ARG;
        if (!list->x || !list->w || !list->cls) return GCP_ERR_INVALID_ARG;
    }
    NoAllocScratch* scratch = nullptr;
    gcp_status st = scratch_for_current_device(&scratch);
    if (st != GCP_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    LossArgs a{};
    a.dr.d = d;
    a.dr.src = kSrcList;
    a.dr.n_total = list->n;
    for (int k = 0; k < d; ++k) a.dr.lidx[k] = list->idx[k];
    a.dr.lx = list->x;
    a.dr.lw = list->w;
    a.dr.lcls = list->cls;
    a.ld = F->ld;
    a.rank = F->rank;
    a.loss = loss;
    for (int k = 0; k < d; ++k)
        a.A[k] = F->bf16 ? static_cast<const void*>(F->A_bf16[k]) : static_cast<const void*>(F->A[k]);
    a.partials = scratch->partials;
    a.ticket = &scratch->ticket;
    a.out = out_dev;
    // one entry per thread: ceil(n / 256) blocks, at most kNoAllocBlocks partial sums
    const int grid = static_cast<int>(list->n > 0 ? (list->n + kNoAllocThreads - 1) / kNoAllocThreads : 1);
    // the completion ticket starts every call at zero (stream-ordered)
    if (cudaMemsetAsync(&scratch->ticket, 0, sizeof(unsigned int), s) != cudaSuccess) return GCP_ERR_CUDA;
    if (launch_loss(a, F->bf16 != 0, grid, kNoAllocThreads, s) != cudaSuccess) return GCP_ERR_CUDA;
    return GCP_OK;
}
