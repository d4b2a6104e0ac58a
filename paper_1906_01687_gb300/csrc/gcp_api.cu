// The C ABI of include/gcp.h: argument validation, library-owned memory,
// launch-shape choice and kernel dispatch.  No arithmetic of the method
// happens here except the FP64 sampling weights, computed once per call.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "../../include/gcp.h"
#include "gcp_device.cuh"
#include "gcp_kernels.cuh"

using namespace gcpk;

static_assert(sizeof(gcp_tensor) == 160, "gcp_tensor layout");
static_assert(sizeof(gcp_factors) == 144, "gcp_factors layout");
static_assert(sizeof(gcp_sampling) == 56, "gcp_sampling layout");
static_assert(sizeof(gcp_samples) == 96, "gcp_samples layout");
static_assert(sizeof(gcp_adam_params) == 24, "gcp_adam_params layout");
static_assert(sizeof(gcp_epoch_params) == 16, "gcp_epoch_params layout");
static_assert(sizeof(gcp_adam_state) == 64, "gcp_adam_state layout");
static_assert(sizeof(gcp_tuning) == 56, "gcp_tuning layout");
static_assert(sizeof(gcp_launch_info) == 80, "gcp_launch_info layout");

struct gcp_handle {
    gcp_tensor X{};
    uint64_t strides[GCP_MAX_MODES]{};
    bool omega_fits_u64 = false;
    double omega = 0.0;
    int rec_int4 = 0;
    int4* recs = nullptr;
    int32_t* d_status = nullptr;     // 32 bytes: the status word, the predicted stream (int64) at 8, the fold
                                     // tail's two block counters (uint32) at 16 and 20
    cudaStream_t last_stream = nullptr;
    int device = 0;
    int num_sms = 0;
    // set by gcp_refresh: the next gradient launch must not draw before its
    // dependency wait, since the kernel just before it rewrote the records
    bool fresh_data = false;
    // nonzero-key hash (stratified)
    unsigned long long* table = nullptr;
    float* table_vals = nullptr;
    uint64_t table_mask = 0;
    // entries of nonzero weight (observed-entry sampling), counted on first use
    int64_t n_observed = -1;
    // stratified zero list and its pass scratch
    int64_t zq_cap = 0;
    int32_t* zidx_base = nullptr;
    int64_t* zcount = nullptr;
    int64_t ztiles_cap = 0;
    unsigned long long* tile_status = nullptr;  // zero between calls (the zero pass clears it)
    unsigned int* zero_ctrs = nullptr;          // the zero pass's tile and completion counters
    // loss-estimate partial sums
    double* partials = nullptr;
    unsigned int* ticket = nullptr;
    int partials_cap = 0;
    gcp_tuning tune{0, 0, 0, 0, -1, -1, -1, 0, 0, 0, 0, 0, 0, 0};
    // replica slabs of the gradient accumulation (kept zero between calls)
    float* rep_ws = nullptr;
    int64_t rep_ws_cap = 0;  // floats
    // optional CUDA-event timing of the fused-gradient kernel (set 0) and of
    // gcp_iteration's Adam kernel (set 1)
    cudaEvent_t* prof_ev = nullptr;
    int32_t prof_cap = 0;
    int32_t prof_used = 0;
    cudaEvent_t* prof_ev2 = nullptr;
    int32_t prof_used2 = 0;
};

namespace {

constexpr int kLossMaxBlocks = 2048;

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// the CUDA error behind this thread's most recent CUDA-caused status
thread_local cudaError_t g_last_cuda_error = cudaSuccess;

gcp_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return GCP_OK;
    g_last_cuda_error = e;
    // clear the runtime's per-thread error state (a failed launch's error is
    // not sticky), so that the caller's next CUDA call does not report it again
    (void)cudaGetLastError();
    if (e == cudaErrorMemoryAllocation) return GCP_ERR_NO_MEMORY;
    return GCP_ERR_CUDA;
}

#define GCP_CUDA_TRY(expr)                                 \
    do {                                                   \
        cudaError_t e_ = (expr);                           \
        if (e_ != cudaSuccess) return cuda_status(e_);     \
    } while (0)

// prod(dims) exactly, or flag overflow of 64 bits
bool omega_u64(const gcp_tensor& X, uint64_t* out)
{
    unsigned __int128 w = 1;
    for (int k = 0; k < X.d; ++k) {
        w *= static_cast<unsigned __int128>(X.dims[k]);
        if (w >> 64) return false;
    }
    *out = static_cast<uint64_t>(w);
    return true;
}

gcp_status check_factors(const gcp_handle* h, const gcp_factors* F)
{
    if (!F) return GCP_ERR_INVALID_ARG;
    if (F->rank < 1 || F->rank > 256 || F->ld < F->rank || F->ld % 4 != 0) return GCP_ERR_INVALID_ARG;
    for (int k = 0; k < h->X.d; ++k) {
        if (!F->A[k] || !aligned(F->A[k], 16)) return GCP_ERR_INVALID_ARG;
        if (F->bf16 && (!F->A_bf16[k] || !aligned(F->A_bf16[k], 8))) return GCP_ERR_INVALID_ARG;
    }
    return GCP_OK;
}

gcp_status check_list(const gcp_handle* h, const gcp_samples* L)
{
    if (!L || L->n < 0) return GCP_ERR_INVALID_ARG;
    if (L->n == 0) return GCP_OK;
    for (int k = 0; k < h->X.d; ++k)
        if (!L->idx[k]) return GCP_ERR_INVALID_ARG;
    if (!L->x || !L->w || !L->cls) return GCP_ERR_INVALID_ARG;
    return GCP_OK;
}

gcp_status check_spec(const gcp_handle* h, const gcp_sampling* S)
{
    if (!S || S->p < 0 || S->q < 0) return GCP_ERR_INVALID_ARG;
    if (S->p > (int64_t(1) << 40) || S->q > (int64_t(1) << 40)) return GCP_ERR_INVALID_ARG;
    switch (S->kind) {
    case GCP_SAMPLER_UNIFORM:
        // over a sparse tensor each draw's value is looked up by its linear key
        if (h->X.sparse && !h->omega_fits_u64) return GCP_ERR_UNSUPPORTED;
        return GCP_OK;
    case GCP_SAMPLER_STRATIFIED:
        if (!h->X.sparse) return GCP_ERR_INVALID_ARG;
        if (!h->omega_fits_u64) return GCP_ERR_UNSUPPORTED;
        if (S->q > 0 && h->omega - static_cast<double>(h->X.nnz) <= 0.0) return GCP_ERR_INVALID_ARG;
        return GCP_OK;
    case GCP_SAMPLER_SEMI_STRATIFIED:
        if (!h->X.sparse) return GCP_ERR_INVALID_ARG;
        return GCP_OK;
    case GCP_SAMPLER_OBSERVED:
        // dense tensors with entry weights: the observed set is {i : v_i != 0}
        if (h->X.sparse || !h->X.weights || S->p != 0) return GCP_ERR_INVALID_ARG;
        return GCP_OK;
    default:
        return GCP_ERR_INVALID_ARG;
    }
}

// Draw descriptor shared by every kernel that generates or reads draws.
DrawArgs make_draw_args(const gcp_handle* h, const gcp_sampling* S, const gcp_samples* L,
                        const int64_t* stream_dev)
{
    DrawArgs a{};
    a.d = h->X.d;
    for (int k = 0; k < h->X.d; ++k) {
        a.dims[k] = static_cast<uint32_t>(h->X.dims[k]);
        a.strides[k] = h->strides[k];
    }
    a.X = h->X.sparse ? nullptr : h->X.vals;
    a.W = h->X.sparse ? nullptr : h->X.weights;
    a.table = h->table;
    a.table_vals = h->table_vals;
    a.table_mask = h->table_mask;
    a.nz_rec = h->recs;
    a.rec_int4 = h->rec_int4;
    a.nnz = h->X.nnz;
    a.stream_dev = stream_dev;
    if (L) {
        a.src = kSrcList;
        a.n_total = L->n;
        for (int k = 0; k < h->X.d; ++k) a.lidx[k] = L->idx[k];
        a.lx = L->x;
        a.lw = L->w;
        a.lcls = L->cls;
        return a;
    }
    a.seed = S->seed;
    a.problem = S->problem;
    a.stream = S->stream;
    const double omega = h->omega, eta = static_cast<double>(h->X.nnz);
    if (S->kind == GCP_SAMPLER_OBSERVED) {  // reads the list of the observed-entry pass
        a.src = kSrcObserved;
        a.p = 0;
        a.n_total = S->q;
        a.w_first = S->q > 0 ? static_cast<float>(static_cast<double>(h->n_observed) / static_cast<double>(S->q)) : 0.0f;
        return a;
    }
    if (S->kind == GCP_SAMPLER_UNIFORM) {
        a.src = h->X.sparse ? kSrcUniformSparse : kSrcUniformDense;
        a.p = 0;
        a.n_total = S->q;
        a.w_first = S->q > 0 ? static_cast<float>(omega / static_cast<double>(S->q)) : 0.0f;
        return a;
    }
    a.src = kSrcSparse;
    a.semi = S->kind == GCP_SAMPLER_SEMI_STRATIFIED;
    a.p = S->p;
    a.n_total = S->p + S->q;
    a.w_first = S->p > 0 ? static_cast<float>(eta / static_cast<double>(S->p)) : 0.0f;
    if (S->q > 0)
        a.w_second = static_cast<float>((a.semi ? omega : omega - eta) / static_cast<double>(S->q));
    return a;
}

gcp_status ensure_hash(gcp_handle* h, cudaStream_t s)
{
    if (h->table) return GCP_OK;
    uint64_t cap = 1024;
    while (cap < 2 * static_cast<uint64_t>(h->X.nnz)) cap <<= 1;
    GCP_CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&h->table), cap * sizeof(unsigned long long)));
    GCP_CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&h->table_vals), cap * sizeof(float)));
    h->table_mask = cap - 1;
    GCP_CUDA_TRY(cudaMemsetAsync(h->table, 0xFF, cap * sizeof(unsigned long long), s));
    GCP_CUDA_TRY(launch_hash_build(h->recs, h->rec_int4, h->X.d, h->strides, h->X.nnz, h->table, h->table_vals,
                                   h->table_mask, h->d_status, s));
    return GCP_OK;
}

gcp_status ensure_zero_list(gcp_handle* h, int64_t q)
{
    if (q <= h->zq_cap) return GCP_OK;
    cudaFree(h->zidx_base);
    h->zidx_base = nullptr;
    h->zq_cap = 0;
    GCP_CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&h->zidx_base), static_cast<size_t>(q) * h->X.d * sizeof(int32_t)));
    h->zq_cap = q;
    return GCP_OK;
}

gcp_status ensure_zero_scratch(gcp_handle* h, int64_t tiles, cudaStream_t s)
{
    if (tiles <= h->ztiles_cap) return GCP_OK;
    cudaFree(h->tile_status);
    cudaFree(h->zero_ctrs);
    h->tile_status = nullptr;
    h->zero_ctrs = nullptr;
    h->ztiles_cap = 0;
    GCP_CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&h->tile_status), static_cast<size_t>(tiles) * sizeof(unsigned long long)));
    GCP_CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&h->zero_ctrs), 2 * sizeof(unsigned int)));
    GCP_CUDA_TRY(cudaMemsetAsync(h->tile_status, 0, static_cast<size_t>(tiles) * sizeof(unsigned long long), s));
    GCP_CUDA_TRY(cudaMemsetAsync(h->zero_ctrs, 0, 2 * sizeof(unsigned int), s));
    h->ztiles_cap = tiles;
    return GCP_OK;
}

// Candidate batch of Section 4.2: ceil(rho * q * omega / zeta).
int64_t zero_batch(const gcp_handle* h, const gcp_sampling* S)
{
    const double rho = S->oversample > 0.0 ? S->oversample : 1.1;
    const double accept = S->kind == GCP_SAMPLER_OBSERVED ? static_cast<double>(h->n_observed)
                                                          : h->omega - static_cast<double>(h->X.nnz);
    return static_cast<int64_t>(std::ceil(rho * static_cast<double>(S->q) * h->omega / accept));
}

// Counts the entries of nonzero weight once (a host read: call gcp_reserve
// before capturing a graph).  Errors: no entry of nonzero weight.
gcp_status ensure_observed(gcp_handle* h, cudaStream_t s)
{
    if (h->n_observed >= 0) return h->n_observed > 0 ? GCP_OK : GCP_ERR_INVALID_ARG;
    const int64_t n = static_cast<int64_t>(h->omega);
    GCP_CUDA_TRY(launch_count_nonzero(h->X.weights, n, h->zcount, s));
    int64_t c = 0;
    GCP_CUDA_TRY(cudaMemcpyAsync(&c, h->zcount, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GCP_CUDA_TRY(cudaStreamSynchronize(s));
    h->n_observed = c;
    return c > 0 ? GCP_OK : GCP_ERR_INVALID_ARG;
}

// Runs the ordered rejection pass; the accepted zeros go to the given destination.
gcp_status run_zero_pass(gcp_handle* h, const gcp_sampling* S, const int64_t* stream_dev,
                         int32_t* const out_idx[GCP_MAX_MODES], float* out_x, float* out_w, int8_t* out_cls,
                         float w_zero, cudaStream_t s)
{
    const bool observed = S->kind == GCP_SAMPLER_OBSERVED;
    gcp_status st = observed ? ensure_observed(h, s) : ensure_hash(h, s);
    if (st != GCP_OK) return st;
    const int64_t batch = zero_batch(h, S);
    const int64_t tiles = (batch + 1023) / 1024;
    st = ensure_zero_scratch(h, tiles, s);
    if (st != GCP_OK) return st;
    ZeroArgs z{};
    z.d = h->X.d;
    for (int k = 0; k < h->X.d; ++k) {
        z.dims[k] = static_cast<uint32_t>(h->X.dims[k]);
        z.strides[k] = h->strides[k];
        z.out_idx[k] = out_idx[k];
    }
    z.seed = S->seed;
    z.problem = S->problem;
    z.stream = S->stream;
    z.stream_dev = stream_dev;
    z.q = S->q;
    z.first_tiles = tiles;
    z.cap = 64 * batch;
    z.table = h->table;
    z.table_mask = h->table_mask;
    z.tag = static_cast<uint32_t>(observed ? kTagObserved : kTagZeroCandidate);
    if (observed) {
        z.obs_w = h->X.weights;
        z.obs_x = h->X.vals;
        z.w_obs = static_cast<double>(h->n_observed) / static_cast<double>(S->q);
    }
    z.tile_status = h->tile_status;
    z.tile_ctr = h->zero_ctrs;
    z.done_ctr = h->zero_ctrs + 1;
    z.count_out = h->zcount;
    z.status = h->d_status;
    z.out_x = out_x;
    z.out_w = out_w;
    z.out_cls = out_cls;
    z.w_zero = w_zero;
    GCP_CUDA_TRY(launch_zero_sampling(z, s));
    return GCP_OK;
}

}  // namespace

namespace {

struct Shape {
    int D = 3, L = 1, NC = 1, block = 256, grid = 1;
    size_t smem = 0;
    uint32_t mask = 0;
    uint32_t comb = 0;  // modes whose updates are combined within a warp step
    uint32_t off[GCP_MAX_MODES] = {};
    uint32_t reps[GCP_MAX_MODES] = {};
    int64_t rep_floats = 0;  // replica workspace the shape needs
    int group = 0;           // group_draws layout
    int pf = 0;              // 1: prefetch layout, 2: staged walk
    int early = 0;           // early descriptors (where the draw source allows)
    int layout() const { return pf; }
};

int next_pow2(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

struct OccKey {
    int D, L, NC, bf16, layout, block;
    size_t smem;
    int device;
};
struct OccEntry {
    OccKey key;
    int bps;
};
std::mutex g_occ_mutex;
OccEntry g_occ[256];
int g_occ_n = 0;

int occupancy(int D, int L, int NC, bool bf16, int layout, int block, size_t smem, int device)
{
    std::lock_guard<std::mutex> lock(g_occ_mutex);
    for (int i = 0; i < g_occ_n; ++i) {
        const OccKey& k = g_occ[i].key;
        if (k.D == D && k.L == L && k.NC == NC && k.bf16 == int(bf16) && k.layout == layout && k.block == block &&
            k.smem == smem && k.device == device)
            return g_occ[i].bps;
    }
    int bps = 0;
    if (grad_occupancy(D, L, NC, bf16, layout, block, smem, &bps) != cudaSuccess || bps < 1) bps = 1;
    if (g_occ_n < 256) g_occ[g_occ_n++] = OccEntry{OccKey{D, L, NC, int(bf16), layout, block, smem, device}, bps};
    return bps;
}

gcp_status choose_shape(const gcp_handle* h, const gcp_factors* F, int64_t n_total, Shape* sh)
{
    const int d = h->X.d;
    sh->D = d == 3 ? 3 : (d == 4 ? 4 : 8);
    const int chunks = (F->rank + 3) / 4;
    const gcp_tuning& t = h->tune;
    if (t.lanes > 0) {
        sh->L = t.lanes;
        sh->NC = t.chunks > 0 ? t.chunks : 1;
        if (!grad_has_config(sh->D, sh->L, sh->NC, 0) || sh->L * sh->NC < chunks) return GCP_ERR_INVALID_ARG;
    } else if (chunks <= 32) {  // one float4 chunk per lane: measured fastest across ranks
        sh->L = next_pow2(chunks);
        sh->NC = 1;
    } else {
        sh->L = 32;
        sh->NC = 2;
    }
    if (!grad_has_config(sh->D, sh->L, sh->NC, 0)) {  // automatic choices must be compiled pairs
        sh->L = 32;
        sh->NC = chunks <= 32 ? 1 : 2;
        if (chunks <= 4) {
            sh->L = 1;
            sh->NC = chunks;
        }
    }
    sh->block = t.block > 0 ? t.block : 256;
    if (sh->block % 32 != 0 || sh->block > 256) return GCP_ERR_INVALID_ARG;  // kernels are built for <= 256
    sh->group = (t.group_draws == 1 && sh->L > 1) ? 1 : 0;
    sh->early = t.early_draws == 1 ? 1 : 0;
    sh->pf = 0;
    if (t.prefetch == 2 && !sh->group && grad_has_config(sh->D, sh->L, sh->NC, 2) && h->X.d == sh->D)
        sh->pf = 2;  // the staged walk
    else if (t.prefetch == 1 && !sh->group && grad_has_config(sh->D, sh->L, sh->NC, 1) && h->X.d == sh->D)
        sh->pf = 1;  // the prefetch layout
    const int64_t per_warp = sh->group ? 32 / sh->L : 32;
    const int64_t warps = (n_total + per_warp - 1) / per_warp;
    const int64_t blocks_needed = std::max<int64_t>(1, (warps + sh->block / 32 - 1) / (sh->block / 32));

    // shared-memory accumulation of small, often-hit G_k (off unless tuned on:
    // shared-memory float atomics are slower than L2 vector reductions here)
    // (the staged walk's shared memory holds the row stage instead)
    const int64_t budget = (t.smem_bytes > 0 && sh->pf != 2) ? t.smem_bytes : 0;
    const double min_hits = t.smem_min_hits >= 0 ? t.smem_min_hits / 10.0 : 2.0;
    const int64_t grid0 = std::min<int64_t>(blocks_needed, static_cast<int64_t>(h->num_sms) * 4);
    const double draws_per_cta = static_cast<double>(n_total) / static_cast<double>(std::max<int64_t>(grid0, 1));
    int64_t used = 0;
    sh->mask = 0;
    for (int k = 0; k < d; ++k) {
        const int64_t bytes = h->X.dims[k] * F->ld * 4;
        if (used + bytes <= budget && draws_per_cta / static_cast<double>(h->X.dims[k]) >= min_hits) {
            sh->mask |= 1u << k;
            sh->off[k] = static_cast<uint32_t>(used / 4);
            used += bytes;
        }
    }
    sh->smem = static_cast<size_t>(used);
    // warp-level pre-reduction (the group walk's variant, 3 or 4 modes)
    sh->comb = 0;
    if (t.warp_combine > 0 && sh->pf == 0 && grad_has_config(sh->D, sh->L, sh->NC, 4) && h->X.d == sh->D)
        for (int k = 0; k < d; ++k)
            if (!((sh->mask >> k) & 1u) && h->X.dims[k] <= t.warp_combine &&
                h->X.dims[k] * (F->ld / 4) < (int64_t(1) << 31))
                sh->comb |= 1u << k;
    if (sh->pf == 1 && sh->smem > 0) sh->pf = 0;  // the prefetch layout accumulates through L2 only
    if (sh->pf == 2)  // the staged walk: each warp stages L draws x d rows x 32 lanes of 16 (BF16: 8) bytes
        sh->smem = static_cast<size_t>(sh->block / 32) * sh->L * sh->D * 32 * (F->bf16 ? 8 : 16);
    const int bps = occupancy(sh->D, sh->L, sh->NC, F->bf16 != 0, sh->layout(), sh->block, sh->smem, h->device);
    const int64_t resident = static_cast<int64_t>(h->num_sms) * bps;
    // one resident wave; the kernel deals batches across all of its blocks
    // evenly, so a launch that fills at least half the wave takes all of it
    const int64_t auto_grid = blocks_needed * 2 >= resident ? resident : blocks_needed;
    sh->grid = static_cast<int>(t.grid_blocks > 0 ? t.grid_blocks : auto_grid);

    // replica slabs for modes whose rows each receive many updates per launch
    const int64_t max_reps = t.max_replicas >= 0 ? t.max_replicas : 32;
    const double target = t.replica_target > 0 ? t.replica_target : 64.0;
    sh->rep_floats = 0;
    for (int k = 0; k < d; ++k) {
        int64_t r = 1;
        if (!((sh->mask >> k) & 1u)) {
            const double hits = static_cast<double>(n_total) / static_cast<double>(h->X.dims[k]);
            r = static_cast<int64_t>(std::ceil(hits / target));
            r = std::max<int64_t>(1, std::min<int64_t>({r, max_reps, static_cast<int64_t>(sh->grid)}));
        }
        sh->reps[k] = static_cast<uint32_t>(r);
        if (r > 1) sh->rep_floats += r * h->X.dims[k] * F->ld;
    }
    return GCP_OK;
}

// Whether a stratified or observed-entry launch of this shape makes its zeros
// inside the gradient kernel (layout 3: the group walk of 3 or 4 modes).
bool zero_tiles_apply(const gcp_handle* h, const Shape& sh)
{
    return h->tune.zero_pass == 0 && sh.layout() == 0 && h->X.d == sh.D &&
           grad_has_config(sh.D, sh.L, sh.NC, sh.comb ? 5 : 3);
}

ModeTable mode_table(const gcp_factors* F, int32_t d, const int64_t* dims)
{
    ModeTable mt{};
    mt.d = d;
    mt.ld = F->ld;
    mt.rank = F->rank;
    mt.off4[0] = 0;
    for (int k = 0; k < d; ++k) {
        mt.off4[k + 1] = mt.off4[k] + dims[k] * F->ld / 4;
        mt.A[k] = F->A[k];
        mt.Abf[k] = F->A_bf16[k];
    }
    return mt;
}

gcp_status check_modes(const gcp_factors* F, int32_t d, const int64_t* dims)
{
    if (!F || !dims || d < 1 || d > GCP_MAX_MODES) return GCP_ERR_INVALID_ARG;
    if (F->rank < 1 || F->rank > 256 || F->ld < F->rank || F->ld % 4 != 0) return GCP_ERR_INVALID_ARG;
    for (int k = 0; k < d; ++k) {
        if (dims[k] < 1 || dims[k] >= (int64_t(1) << 31)) return GCP_ERR_INVALID_ARG;
        if (!F->A[k] || !aligned(F->A[k], 16)) return GCP_ERR_INVALID_ARG;
        if (F->A_bf16[k] && !aligned(F->A_bf16[k], 8)) return GCP_ERR_INVALID_ARG;
    }
    return GCP_OK;
}

bool modes_ok(float* const P[GCP_MAX_MODES], int32_t d)
{
    if (!P) return false;
    for (int k = 0; k < d; ++k)
        if (!P[k] || !aligned(P[k], 16)) return false;
    return true;
}

int elementwise_grid(const ModeTable& mt)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t total4 = mt.off4[mt.d];
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((total4 + 255) / 256, int64_t(sms) * 8)));
}

}  // namespace

extern "C" {

const char* gcp_version(void) { return "gcp_gb300 0.1 (sm_103a)"; }

int32_t gcp_last_cuda_error(void) { return static_cast<int32_t>(g_last_cuda_error); }

const char* gcp_last_cuda_error_name(void) { return cudaGetErrorName(g_last_cuda_error); }

const char* gcp_status_string(gcp_status s)
{
    switch (s) {
    case GCP_OK: return "ok";
    case GCP_ERR_INVALID_ARG: return "invalid argument";
    case GCP_ERR_CUDA: return "CUDA error";
    case GCP_ERR_NO_MEMORY: return "out of device memory";
    case GCP_ERR_SAMPLE_SHORTFALL: return "stratified sampling found fewer zeros than requested";
    case GCP_ERR_TIMEOUT: return "device wait timed out";
    case GCP_ERR_NONFINITE: return "non-finite loss estimate";
    case GCP_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

int64_t gcp_sample_count(const gcp_sampling* S)
{
    if (!S || S->p < 0 || S->q < 0) return -1;
    if (S->kind == GCP_SAMPLER_UNIFORM || S->kind == GCP_SAMPLER_OBSERVED) return S->q;
    if (S->kind == GCP_SAMPLER_STRATIFIED || S->kind == GCP_SAMPLER_SEMI_STRATIFIED) return S->p + S->q;
    return -1;
}

gcp_status gcp_create(gcp_handle** out, const gcp_tensor* X, gcp_stream_t stream)
{
    if (!out || !X) return GCP_ERR_INVALID_ARG;
    *out = nullptr;
    if (X->d < 2 || X->d > GCP_MAX_MODES) return GCP_ERR_INVALID_ARG;
    for (int k = 0; k < X->d; ++k)
        if (X->dims[k] < 1 || X->dims[k] >= (int64_t(1) << 31)) return GCP_ERR_INVALID_ARG;
    if (X->sparse) {
        if (X->nnz < 1) return GCP_ERR_INVALID_ARG;
        for (int k = 0; k < X->d; ++k)
            if (!X->idx[k]) return GCP_ERR_INVALID_ARG;
    } else if (!X->vals) {
        return GCP_ERR_INVALID_ARG;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    gcp_handle* h = new (std::nothrow) gcp_handle();
    if (!h) return GCP_ERR_NO_MEMORY;
    h->X = *X;
    for (int k = X->d; k < GCP_MAX_MODES; ++k) {
        h->X.dims[k] = 0;
        h->X.idx[k] = nullptr;
    }
    if (!X->sparse) h->X.nnz = 0;
    if (X->sparse) h->X.weights = nullptr;
    uint64_t om = 0;
    h->omega_fits_u64 = omega_u64(h->X, &om);
    h->omega = 1.0;
    for (int k = 0; k < X->d; ++k) h->omega *= static_cast<double>(X->dims[k]);
    if (!X->sparse && !h->omega_fits_u64) {
        delete h;
        return GCP_ERR_INVALID_ARG;
    }
    // row-major strides (wrap modulo 2^64 only when the tensor has >= 2^64 entries,
    // in which case no linear key is ever formed)
    uint64_t stride = 1;
    for (int k = X->d - 1; k >= 0; --k) {
        h->strides[k] = stride;
        stride *= static_cast<uint64_t>(X->dims[k]);
    }
    auto fail = [&](gcp_status st) {
        gcp_destroy(h);
        return st;
    };
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) return fail(cuda_status(e));
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (h->num_sms < 1) h->num_sms = 1;
    if ((e = cudaMalloc(reinterpret_cast<void**>(&h->d_status), 32)) != cudaSuccess) return fail(cuda_status(e));
    if ((e = cudaMalloc(reinterpret_cast<void**>(&h->zcount), sizeof(int64_t))) != cudaSuccess) return fail(cuda_status(e));
    if ((e = cudaMalloc(reinterpret_cast<void**>(&h->partials), kLossMaxBlocks * sizeof(double))) != cudaSuccess)
        return fail(cuda_status(e));
    if ((e = cudaMalloc(reinterpret_cast<void**>(&h->ticket), sizeof(unsigned int))) != cudaSuccess) return fail(cuda_status(e));
    h->partials_cap = kLossMaxBlocks;
    if ((e = cudaMemsetAsync(h->d_status, 0, 32, s)) != cudaSuccess) return fail(cuda_status(e));
    if ((e = cudaMemsetAsync(h->zcount, 0, sizeof(int64_t), s)) != cudaSuccess) return fail(cuda_status(e));
    if ((e = cudaMemsetAsync(h->ticket, 0, sizeof(unsigned int), s)) != cudaSuccess) return fail(cuda_status(e));
    if (X->sparse) {
        h->rec_int4 = (X->d + 1 + 3) / 4;
        const size_t bytes = static_cast<size_t>(X->nnz) * h->rec_int4 * sizeof(int4);
        if ((e = cudaMalloc(reinterpret_cast<void**>(&h->recs), bytes)) != cudaSuccess) return fail(cuda_status(e));
        if ((e = launch_pack_records(h->X, h->recs, h->rec_int4, s)) != cudaSuccess) return fail(cuda_status(e));
    }
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(cuda_status(e));
    h->last_stream = s;
    *out = h;
    return GCP_OK;
}

static void profile_free(gcp_handle* h)
{
    if (!h->prof_ev) return;
    for (int i = 0; i < 2 * h->prof_cap; ++i) {
        cudaEventDestroy(h->prof_ev[i]);
        cudaEventDestroy(h->prof_ev2[i]);
    }
    delete[] h->prof_ev;
    delete[] h->prof_ev2;
    h->prof_ev = h->prof_ev2 = nullptr;
    h->prof_cap = h->prof_used = h->prof_used2 = 0;
}

gcp_status gcp_profile(gcp_handle* h, int32_t enable, int32_t capacity)
{
    if (!h || (enable && (capacity < 1 || capacity > 65536))) return GCP_ERR_INVALID_ARG;
    GCP_CUDA_TRY(cudaDeviceSynchronize());
    profile_free(h);
    if (!enable) return GCP_OK;
    h->prof_ev = new (std::nothrow) cudaEvent_t[2 * static_cast<size_t>(capacity)]();
    h->prof_ev2 = new (std::nothrow) cudaEvent_t[2 * static_cast<size_t>(capacity)]();
    if (!h->prof_ev || !h->prof_ev2) {
        delete[] h->prof_ev;
        delete[] h->prof_ev2;
        h->prof_ev = h->prof_ev2 = nullptr;
        return GCP_ERR_NO_MEMORY;
    }
    h->prof_cap = capacity;
    for (int i = 0; i < 2 * capacity; ++i) {
        if (cudaEventCreate(&h->prof_ev[i]) != cudaSuccess || cudaEventCreate(&h->prof_ev2[i]) != cudaSuccess) {
            profile_free(h);
            return GCP_ERR_CUDA;
        }
    }
    h->prof_used = h->prof_used2 = 0;
    return GCP_OK;
}

gcp_status gcp_profile_read(gcp_handle* h, int32_t which, double* total_ms, int64_t* launches)
{
    if (!h || !total_ms || !launches || which < 0 || which > 1) return GCP_ERR_INVALID_ARG;
    cudaEvent_t* ev = which == 0 ? h->prof_ev : h->prof_ev2;
    int32_t* used = which == 0 ? &h->prof_used : &h->prof_used2;
    double sum = 0.0;
    for (int i = 0; i < *used; ++i) {
        GCP_CUDA_TRY(cudaEventSynchronize(ev[2 * i + 1]));
        float ms = 0.f;
        GCP_CUDA_TRY(cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]));
        sum += ms;
    }
    *total_ms = sum;
    *launches = *used;
    *used = 0;
    return GCP_OK;
}

gcp_status gcp_destroy(gcp_handle* h)
{
    if (!h) return GCP_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    profile_free(h);
    cudaFree(h->recs);
    cudaFree(h->d_status);
    cudaFree(h->table);
    cudaFree(h->table_vals);
    cudaFree(h->zidx_base);
    cudaFree(h->zcount);
    cudaFree(h->tile_status);
    cudaFree(h->zero_ctrs);
    cudaFree(h->partials);
    cudaFree(h->ticket);
    cudaFree(h->rep_ws);
    delete h;
    return GCP_OK;
}

gcp_status gcp_get_device_status(gcp_handle* h, int32_t* host_out)
{
    if (!h || !host_out) return GCP_ERR_INVALID_ARG;
    GCP_CUDA_TRY(cudaDeviceSynchronize());
    int32_t v = 0;
    GCP_CUDA_TRY(cudaMemcpy(&v, h->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost));
    GCP_CUDA_TRY(cudaMemset(h->d_status, 0, sizeof(int32_t)));
    *host_out = v;
    return GCP_OK;
}

gcp_status gcp_set_tuning(gcp_handle* h, const gcp_tuning* t)
{
    if (!h) return GCP_ERR_INVALID_ARG;
    if (!t) {
        h->tune = gcp_tuning{0, 0, 0, 0, -1, -1, -1, 0, 0, 0, 0, 0, 0, 0};
        return GCP_OK;
    }
    if (t->lanes > 0 && !grad_has_config(3, t->lanes, t->chunks > 0 ? t->chunks : 1, 0)) return GCP_ERR_INVALID_ARG;
    if (t->prefetch < 0 || t->prefetch > 2) return GCP_ERR_INVALID_ARG;
    if (t->block != 0 && (t->block < 32 || t->block > 256 || t->block % 32 != 0)) return GCP_ERR_INVALID_ARG;
    if (t->grid_blocks < 0 || t->smem_bytes > 200 * 1024 || t->max_replicas > 1024 || t->replica_target < 0 ||
        t->group_draws < 0 || t->group_draws > 1 || t->early_draws < 0 || t->early_draws > 1 || t->zero_pass < 0 ||
        t->zero_pass > 1 || t->warp_combine < 0 || t->tail_work < 0 || t->tail_work > 1)
        return GCP_ERR_INVALID_ARG;
    h->tune = *t;
    return GCP_OK;
}

gcp_status gcp_get_launch(gcp_handle* h, const gcp_factors* F, int64_t n_draws, gcp_launch_info* out)
{
    if (!h || !out || n_draws < 0) return GCP_ERR_INVALID_ARG;
    gcp_status st = check_factors(h, F);
    if (st != GCP_OK) return st;
    Shape sh;
    st = choose_shape(h, F, n_draws, &sh);
    if (st != GCP_OK) return st;
    *out = gcp_launch_info{};
    out->lanes = sh.L;
    out->chunks = sh.NC;
    out->block = sh.block;
    out->grid_blocks = sh.grid;
    out->smem_bytes = static_cast<int32_t>(sh.smem);
    out->smem_mode_mask = sh.mask;
    out->group_draws = sh.group;
    out->prefetch = sh.pf;
    out->early_draws = sh.early;
    out->zero_tiles = zero_tiles_apply(h, sh) ? 1 : 0;
    out->combine_mode_mask = sh.comb;
    {
        int64_t total4 = 0;
        for (int k = 0; k < h->X.d; ++k) total4 += h->X.dims[k] * (F->ld / 4);
        const int64_t blocks = std::max<int64_t>(1, (total4 * 4 + sh.block - 1) / sh.block);
        out->adam_tail_blocks = (h->tune.tail_work == 1 && blocks <= 64 && blocks <= sh.grid && n_draws > 0)
                                    ? static_cast<int32_t>(blocks) : 0;
    }
    for (int k = 0; k < h->X.d; ++k) out->replicas[k] = static_cast<int32_t>(sh.reps[k]);
    return GCP_OK;
}

gcp_status gcp_sample(gcp_handle* h, const gcp_sampling* S, const gcp_samples* out, gcp_stream_t stream)
{
    if (!h) return GCP_ERR_INVALID_ARG;
    gcp_status st = check_spec(h, S);
    if (st != GCP_OK) return st;
    st = check_list(h, out);
    if (st != GCP_OK) return st;
    if (out->n != gcp_sample_count(S)) return GCP_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    h->last_stream = s;
    if (out->n == 0) return GCP_OK;
    if (S->kind == GCP_SAMPLER_UNIFORM && h->X.sparse) {
        st = ensure_hash(h, s);
        if (st != GCP_OK) return st;
    }
    if (S->kind == GCP_SAMPLER_OBSERVED) {  // the whole list comes from the observed-entry pass
        if ((st = ensure_observed(h, s)) != GCP_OK) return st;
        int32_t* odst[GCP_MAX_MODES] = {};
        for (int k = 0; k < h->X.d; ++k) odst[k] = out->idx[k];
        return run_zero_pass(h, S, nullptr, odst, out->x, out->w, out->cls, 0.0f, s);
    }
    DrawArgs dr = make_draw_args(h, S, nullptr, nullptr);
    if (S->kind != GCP_SAMPLER_STRATIFIED) {
        GCP_CUDA_TRY(launch_materialise(dr, out->idx, out->x, out->w, out->cls, 0, dr.n_total, h->d_status, s));
        return GCP_OK;
    }
    GCP_CUDA_TRY(launch_materialise(dr, out->idx, out->x, out->w, out->cls, 0, S->p, h->d_status, s));
    if (S->q == 0) return GCP_OK;
    int32_t* zdst[GCP_MAX_MODES] = {};
    for (int k = 0; k < h->X.d; ++k) zdst[k] = out->idx[k] + S->p;
    return run_zero_pass(h, S, nullptr, zdst, out->x + S->p, out->w + S->p, out->cls + S->p, dr.w_second, s);
}

gcp_status gcp_reserve(gcp_handle* h, const gcp_sampling* S, gcp_stream_t stream)
{
    if (!h) return GCP_ERR_INVALID_ARG;
    gcp_status st = check_spec(h, S);
    if (st != GCP_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    h->last_stream = s;
    if (S->kind == GCP_SAMPLER_UNIFORM && h->X.sparse) {
        if ((st = ensure_hash(h, s)) != GCP_OK) return st;
    }
    if ((S->kind == GCP_SAMPLER_STRATIFIED || S->kind == GCP_SAMPLER_OBSERVED) && S->q > 0) {
        st = S->kind == GCP_SAMPLER_OBSERVED ? ensure_observed(h, s) : ensure_hash(h, s);
        if (st != GCP_OK) return st;
        // tile words for tiles of 1024 candidates (the separate pass) or of one
        // block (zeros made in the gradient launch: blocks of at least 32 threads)
        if ((st = ensure_zero_scratch(h, (zero_batch(h, S) + 31) / 32, s)) != GCP_OK) return st;
        if ((st = ensure_zero_list(h, S->q)) != GCP_OK) return st;
    }
    GCP_CUDA_TRY(cudaStreamSynchronize(s));
    return GCP_OK;
}

// advance_t (gcp_iteration): the gradient kernel advances advance_t->t for the
// Adam step that follows; *launched reports whether a gradient kernel ran.
// first / count (count >= 0): only the draws j in [first, first + count) of the spec.
// adam (gcp_iteration, with deferred_fold and advance_t): the step that follows;
// where the factor set is small the gradient kernel's last blocks take it
// (*adam_fused = true) and no Adam launch is needed.
static gcp_status grad_impl(gcp_handle* h, const gcp_factors* F, gcp_loss loss, const gcp_sampling* S,
                            const gcp_samples* list, const int64_t* stream_dev, float* const G[GCP_MAX_MODES],
                            cudaStream_t s, FoldArgs* deferred_fold, gcp_adam_state* advance_t = nullptr,
                            bool* launched = nullptr, int64_t first = 0, int64_t count = -1,
                            const AdamArgs* adam = nullptr, bool* adam_fused = nullptr)
{
    if (adam_fused) *adam_fused = false;
    if (launched) *launched = false;
    if (!h || (S == nullptr) == (list == nullptr)) return GCP_ERR_INVALID_ARG;
    if (loss < GCP_LOSS_GAUSSIAN || loss > GCP_LOSS_BETA_HALF) return GCP_ERR_INVALID_ARG;
    gcp_status st = check_factors(h, F);
    if (st != GCP_OK) return st;
    if (!modes_ok(G, h->X.d)) return GCP_ERR_INVALID_ARG;
    st = S ? check_spec(h, S) : check_list(h, list);
    if (st != GCP_OK) return st;
    h->last_stream = s;
    const bool table_ready = h->table != nullptr;
    if (S && S->kind == GCP_SAMPLER_UNIFORM && h->X.sparse) {
        st = ensure_hash(h, s);
        if (st != GCP_OK) return st;
    }
    if (S && S->kind == GCP_SAMPLER_OBSERVED && S->q > 0) {
        st = ensure_observed(h, s);
        if (st != GCP_OK) return st;
    }
    GradArgs a{};
    a.dr = make_draw_args(h, S, list, stream_dev);
    if (count >= 0) {  // a draw range of the spec
        if (first < 0 || first > a.dr.n_total || count > a.dr.n_total - first) return GCP_ERR_INVALID_ARG;
        a.dr.j_begin = first;
        a.dr.n_total = first + count;
    }
    const int64_t n_draws = a.dr.n_total - a.dr.j_begin;
    // early descriptors only for draws that read nothing but the data tensor and
    // tables built before this call (not a list; with stratified sampling the
    // kernel keeps them to warps whose first batch holds nonzero draws only),
    // and not right after gcp_refresh rewrote the records
    const bool early_ok = (a.dr.src == kSrcUniformDense || (a.dr.src == kSrcUniformSparse && table_ready) ||
                           a.dr.src == kSrcSparse) && !h->fresh_data;
    if (n_draws == 0) return GCP_OK;
    Shape sh;
    st = choose_shape(h, F, n_draws, &sh);
    if (st != GCP_OK) return st;
    int layout = (sh.layout() == 0 && sh.comb) ? 4 : sh.layout();
    int grid = sh.grid;
    if (S && (S->kind == GCP_SAMPLER_STRATIFIED || S->kind == GCP_SAMPLER_OBSERVED) && S->q > 0) {
        // the zero draws of this launch: ranks [z_begin, z_end) of the kept candidates
        const int64_t z_begin = std::max<int64_t>(a.dr.j_begin - a.dr.p, 0);
        const int64_t z_end = std::max<int64_t>(a.dr.n_total - a.dr.p, 0);
        if (zero_tiles_apply(h, sh) && z_end > z_begin) {
            // made inside the gradient launch (layout 3): the first `tiles` blocks
            if (S->kind == GCP_SAMPLER_STRATIFIED && (st = ensure_hash(h, s)) != GCP_OK) return st;
            const int64_t batch = zero_batch(h, S);
            const int64_t tiles = (batch + sh.block - 1) / sh.block;
            if ((st = ensure_zero_scratch(h, tiles, s)) != GCP_OK) return st;
            ZeroTileArgs& z = a.zt;
            z.tiles = tiles;
            z.cap = 64 * batch;
            z.q = S->q;
            z.z_begin = z_begin;
            z.z_end = z_end;
            z.observed = S->kind == GCP_SAMPLER_OBSERVED ? 1 : 0;
            z.tag = static_cast<uint32_t>(z.observed ? kTagObserved : kTagZeroCandidate);
            z.tile_status = h->tile_status;
            z.tile_ctr = h->zero_ctrs;
            z.done_ctr = h->zero_ctrs + 1;
            z.count_out = h->zcount;
            z.status = h->d_status;
            a.dr.table = h->table;
            a.dr.table_mask = h->table_mask;
            // the other blocks walk the nonzero draws [j_begin, min(end, p))
            a.dr.n_total = std::min(a.dr.n_total, a.dr.p);
            const int64_t nz = std::max<int64_t>(a.dr.n_total - a.dr.j_begin, 0);
            const int64_t per_warp = sh.group ? 32 / sh.L : 32;
            const int64_t blocks_nz = (((nz + per_warp - 1) / per_warp) + sh.block / 32 - 1) / (sh.block / 32);
            grid = static_cast<int>(tiles + std::min<int64_t>(sh.grid, blocks_nz));
            layout = sh.comb ? 5 : 3;
        } else if (z_end > z_begin) {  // (a range of nonzero draws only needs no zeros)
            st = ensure_zero_list(h, S->q);
            if (st != GCP_OK) return st;
            int32_t* zdst[GCP_MAX_MODES] = {};
            for (int k = 0; k < h->X.d; ++k) zdst[k] = h->zidx_base + static_cast<size_t>(k) * h->zq_cap;
            st = run_zero_pass(h, S, stream_dev, zdst, nullptr, nullptr, nullptr, 0.0f, s);
            if (st != GCP_OK) return st;
            for (int k = 0; k < h->X.d; ++k) a.dr.zidx[k] = zdst[k];
            a.dr.zcount = h->zcount;
        }
    }
    if (sh.rep_floats > h->rep_ws_cap) {
        cudaFree(h->rep_ws);
        h->rep_ws = nullptr;
        h->rep_ws_cap = 0;
        GCP_CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&h->rep_ws), static_cast<size_t>(sh.rep_floats) * sizeof(float)));
        GCP_CUDA_TRY(cudaMemsetAsync(h->rep_ws, 0, static_cast<size_t>(sh.rep_floats) * sizeof(float), s));
        h->rep_ws_cap = sh.rep_floats;
    }
    a.ld = F->ld;
    a.rank = F->rank;
    a.loss = loss;
    a.smem_floats = sh.pf == 2 ? 0 : static_cast<int32_t>(sh.smem / 4);  // accumulators to zero (not the stage)
    a.smem_mask = sh.mask;
    a.comb_mask = sh.comb;
    a.group_draws = sh.group;
    a.early = (sh.early && early_ok) ? 1 : 0;
    a.stream_pred = reinterpret_cast<int64_t*>(reinterpret_cast<char*>(h->d_status) + 8);
    a.st_advance = advance_t;
    FoldArgs fold{};
    int64_t ws_off = 0;
    for (int k = 0; k < GCP_MAX_MODES; ++k) a.reps[k] = 1;
    for (int k = 0; k < h->X.d; ++k) {
        a.A[k] = F->bf16 ? static_cast<const void*>(F->A_bf16[k]) : static_cast<const void*>(F->A[k]);
        a.smem_off[k] = sh.off[k];
        a.reps[k] = sh.reps[k];
        const int64_t slab = h->X.dims[k] * F->ld;
        if (deferred_fold) {
            deferred_fold->reps[k] = 1;
            deferred_fold->R[k] = nullptr;
        }
        if (sh.reps[k] > 1) {
            a.G[k] = h->rep_ws + ws_off;
            a.rep_stride[k] = static_cast<uint64_t>(slab);
            if (deferred_fold) {  // per mode, indexed by k
                deferred_fold->reps[k] = sh.reps[k];
                deferred_fold->R[k] = h->rep_ws + ws_off;
                deferred_fold->rep_stride4[k] = static_cast<uint64_t>(slab / 4);
            } else {  // compacted over the replicated modes
                const int m = fold.nmodes++;
                fold.R[m] = h->rep_ws + ws_off;
                fold.G[m] = G[k];
                fold.reps[m] = sh.reps[k];
                fold.rep_stride4[m] = static_cast<uint64_t>(slab / 4);
                fold.off4[m + 1] = fold.off4[m] + slab / 4;
            }
            ws_off += slab * sh.reps[k];
        } else {
            a.G[k] = G[k];
            a.rep_stride[k] = 0;
        }
    }
    // the fold is done by the gradient kernel's last blocks to finish instead of
    // a launch of its own: enough blocks that each lane loads about eight
    // replica chunks (one round trip), at most 64
    if (!deferred_fold && fold.nmodes > 0 && h->tune.tail_work == 1) {
        int64_t loads = 0;
        for (int m = 0; m < fold.nmodes; ++m) loads += (fold.off4[m + 1] - fold.off4[m]) * fold.reps[m];
        const int64_t blocks = std::max<int64_t>(1, (loads + 8 * sh.block - 1) / (8 * sh.block));
        if (blocks <= 64 && blocks <= grid) {
            a.tail.fold = fold;
            a.tail.done = reinterpret_cast<unsigned int*>(reinterpret_cast<char*>(h->d_status) + 16);
            a.tail.blocks = static_cast<int32_t>(blocks);
            a.tail.status = h->d_status;
        }
    }
    // the Adam step of gcp_iteration by the gradient kernel's last blocks (four
    // lanes per float4 element, at most 64 blocks) for small factor sets
    if (adam && deferred_fold && advance_t && h->tune.tail_work == 1) {
        AdamArgs ad = *adam;
        for (int k = 0; k < h->X.d; ++k) {
            ad.reps[k] = deferred_fold->reps[k] > 1 ? deferred_fold->reps[k] : 1;
            ad.R[k] = deferred_fold->R[k];
            ad.rep_stride4[k] = deferred_fold->rep_stride4[k];
        }
        ad.t_advanced = 1;
        const int64_t blocks = std::max<int64_t>(1, (ad.mt.off4[h->X.d] * 4 + sh.block - 1) / sh.block);
        if (blocks <= 64 && blocks <= grid) {
            a.tail.adam = ad;
            a.tail.adam_on = 1;
            a.tail.blocks = static_cast<int32_t>(std::max<int64_t>(1, blocks));
            a.tail.done = reinterpret_cast<unsigned int*>(reinterpret_cast<char*>(h->d_status) + 16);
            a.tail.status = h->d_status;
            if (adam_fused) *adam_fused = true;
        }
    }
    const bool timed = h->prof_ev && h->prof_used < h->prof_cap;
    if (timed) GCP_CUDA_TRY(cudaEventRecord(h->prof_ev[2 * h->prof_used], s));
    GCP_CUDA_TRY(launch_grad(a, sh.D, sh.L, sh.NC, F->bf16 != 0, layout, grid, sh.block, sh.smem, s));
    h->fresh_data = false;
    if (launched) *launched = true;
    if (timed) {
        GCP_CUDA_TRY(cudaEventRecord(h->prof_ev[2 * h->prof_used + 1], s));
        h->prof_used++;
    }
    if (!deferred_fold && fold.nmodes > 0 && a.tail.blocks == 0) {
        const int64_t total4 = fold.off4[fold.nmodes];
        const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((total4 + 255) / 256, int64_t(h->num_sms) * 8)));
        GCP_CUDA_TRY(launch_fold(fold, grid, s));
    }
    return GCP_OK;
}

// The gradient kernel over an arbitrary prepared draw source (no sampling spec).
static gcp_status grad_from_args(gcp_handle* h, const gcp_factors* F, gcp_loss loss, GradArgs a,
                                 float* const G[GCP_MAX_MODES], cudaStream_t s)
{
    Shape sh;
    gcp_status st = choose_shape(h, F, a.dr.n_total, &sh);
    if (st != GCP_OK) return st;
    a.ld = F->ld;
    a.rank = F->rank;
    a.loss = loss;
    a.smem_floats = 0;
    a.smem_mask = 0;
    a.comb_mask = 0;
    a.group_draws = sh.group;
    a.early = 0;
    a.stream_pred = nullptr;
    a.st_advance = nullptr;
    for (int k = 0; k < GCP_MAX_MODES; ++k) a.reps[k] = 1;
    for (int k = 0; k < h->X.d; ++k) {
        a.A[k] = F->bf16 ? static_cast<const void*>(F->A_bf16[k]) : static_cast<const void*>(F->A[k]);
        a.G[k] = G[k];
        a.rep_stride[k] = 0;
    }
    GCP_CUDA_TRY(launch_grad(a, sh.D, sh.L, sh.NC, F->bf16 != 0, 0, sh.grid, sh.block, 0, s));
    return GCP_OK;
}

gcp_status gcp_full_grad(gcp_handle* h, const gcp_factors* F, gcp_loss loss, float* const G[GCP_MAX_MODES],
                         gcp_stream_t stream)
{
    if (!h || h->X.sparse) return GCP_ERR_INVALID_ARG;
    if (loss < GCP_LOSS_GAUSSIAN || loss > GCP_LOSS_BETA_HALF) return GCP_ERR_INVALID_ARG;
    gcp_status st = check_factors(h, F);
    if (st != GCP_OK) return st;
    if (!modes_ok(G, h->X.d)) return GCP_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    h->last_stream = s;
    GradArgs a{};
    gcp_sampling none{};
    a.dr = make_draw_args(h, &none, nullptr, nullptr);
    a.dr.src = kSrcEnumerate;
    a.dr.n_total = static_cast<int64_t>(h->omega);
    return grad_from_args(h, F, loss, a, G, s);
}

gcp_status gcp_full_loss(gcp_handle* h, const gcp_factors* F, gcp_loss loss, double* out_dev, gcp_stream_t stream)
{
    if (!h || h->X.sparse || !out_dev || !aligned(out_dev, 8)) return GCP_ERR_INVALID_ARG;
    if (loss < GCP_LOSS_GAUSSIAN || loss > GCP_LOSS_BETA_HALF) return GCP_ERR_INVALID_ARG;
    gcp_status st = check_factors(h, F);
    if (st != GCP_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    h->last_stream = s;
    LossArgs a{};
    gcp_sampling none{};
    a.dr = make_draw_args(h, &none, nullptr, nullptr);
    a.dr.src = kSrcEnumerate;
    a.dr.n_total = static_cast<int64_t>(h->omega);
    a.ld = F->ld;
    a.rank = F->rank;
    a.loss = loss;
    for (int k = 0; k < h->X.d; ++k)
        a.A[k] = F->bf16 ? static_cast<const void*>(F->A_bf16[k]) : static_cast<const void*>(F->A[k]);
    a.partials = h->partials;
    a.ticket = h->ticket;
    a.out = out_dev;
    const int64_t want = std::max<int64_t>(1, (a.dr.n_total + 255) / 256);
    const int grid = static_cast<int>(std::min<int64_t>(want, std::min<int64_t>(h->partials_cap, int64_t(h->num_sms) * 4)));
    GCP_CUDA_TRY(launch_loss(a, F->bf16 != 0, grid, 256, s));
    return GCP_OK;
}

gcp_status gcp_grad(gcp_handle* h, const gcp_factors* F, gcp_loss loss, const gcp_sampling* S,
                    const gcp_samples* list, const int64_t* stream_dev, float* const G[GCP_MAX_MODES],
                    gcp_stream_t stream)
{
    return grad_impl(h, F, loss, S, list, stream_dev, G, reinterpret_cast<cudaStream_t>(stream), nullptr);
}

gcp_status gcp_grad_range(gcp_handle* h, const gcp_factors* F, gcp_loss loss, const gcp_sampling* S, int64_t first,
                          int64_t count, const int64_t* stream_dev, float* const G[GCP_MAX_MODES],
                          gcp_stream_t stream)
{
    if (!S || count < 0) return GCP_ERR_INVALID_ARG;
    return grad_impl(h, F, loss, S, nullptr, stream_dev, G, reinterpret_cast<cudaStream_t>(stream), nullptr,
                     nullptr, nullptr, first, count);
}

gcp_status gcp_refresh(gcp_handle* h, gcp_stream_t stream)
{
    if (!h) return GCP_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    h->last_stream = s;
    if (!h->X.sparse) {
        h->n_observed = -1;  // the entries of nonzero weight are counted again on next use
        return GCP_OK;
    }
    GCP_CUDA_TRY(launch_pack_records(h->X, h->recs, h->rec_int4, s));
    if (h->table) {  // rebuilt in place: same nonzero count, same table size
        GCP_CUDA_TRY(cudaMemsetAsync(h->table, 0xFF, (h->table_mask + 1) * sizeof(unsigned long long), s));
        GCP_CUDA_TRY(launch_hash_build(h->recs, h->rec_int4, h->X.d, h->strides, h->X.nnz, h->table, h->table_vals,
                                       h->table_mask, h->d_status, s));
    }
    h->fresh_data = true;
    return GCP_OK;
}

gcp_status gcp_loss_est(gcp_handle* h, const gcp_factors* F, gcp_loss loss, const gcp_samples* list,
                        double* out_dev, gcp_stream_t stream)
{
    if (!h || !out_dev || !aligned(out_dev, 8)) return GCP_ERR_INVALID_ARG;
    if (loss < GCP_LOSS_GAUSSIAN || loss > GCP_LOSS_BETA_HALF) return GCP_ERR_INVALID_ARG;
    gcp_status st = check_factors(h, F);
    if (st != GCP_OK) return st;
    st = check_list(h, list);
    if (st != GCP_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    h->last_stream = s;
    LossArgs a{};
    a.dr = make_draw_args(h, nullptr, list, nullptr);
    a.ld = F->ld;
    a.rank = F->rank;
    a.loss = loss;
    for (int k = 0; k < h->X.d; ++k)
        a.A[k] = F->bf16 ? static_cast<const void*>(F->A_bf16[k]) : static_cast<const void*>(F->A[k]);
    a.partials = h->partials;
    a.ticket = h->ticket;
    a.out = out_dev;
    const int64_t want = std::max<int64_t>(1, (list->n + 255) / 256);
    const int grid = static_cast<int>(std::min<int64_t>(want, std::min<int64_t>(h->partials_cap, int64_t(h->num_sms) * 4)));
    GCP_CUDA_TRY(launch_loss(a, F->bf16 != 0, grid, 256, s));
    return GCP_OK;
}

gcp_status gcp_state_init(gcp_adam_state* state, float alpha, gcp_stream_t stream)
{
    if (!state || !aligned(state, 8)) return GCP_ERR_INVALID_ARG;
    GCP_CUDA_TRY(launch_state_init(state, alpha, reinterpret_cast<cudaStream_t>(stream)));
    return GCP_OK;
}

gcp_status gcp_adam_step(const gcp_factors* F, int32_t d, const int64_t* dims, float* const G[GCP_MAX_MODES],
                         float* const B[GCP_MAX_MODES], float* const C[GCP_MAX_MODES], const gcp_adam_params* prm,
                         gcp_adam_state* state, gcp_stream_t stream)
{
    gcp_status st = check_modes(F, d, dims);
    if (st != GCP_OK) return st;
    if (!prm || !state || !aligned(state, 8) || !modes_ok(G, d) || !modes_ok(B, d) || !modes_ok(C, d))
        return GCP_ERR_INVALID_ARG;
    if (!(prm->beta1 >= 0.f && prm->beta1 < 1.f && prm->beta2 >= 0.f && prm->beta2 < 1.f && prm->eps >= 0.f))
        return GCP_ERR_INVALID_ARG;
    AdamArgs a{};
    a.mt = mode_table(F, d, dims);
    if (a.mt.off4[a.mt.d] >= (int64_t(1) << 31)) return GCP_ERR_INVALID_ARG;  // 32-bit element indices
    for (int k = 0; k < d; ++k) {
        a.mt.G[k] = G[k];
        a.mt.B[k] = B[k];
        a.mt.C[k] = C[k];
    }
    a.beta1 = prm->beta1;
    a.beta2 = prm->beta2;
    a.eps = prm->eps;
    a.lower = prm->lower;
    a.eps_inside_sqrt = prm->eps_inside_sqrt;
    a.st = state;
    for (int k = 0; k < GCP_MAX_MODES; ++k) a.reps[k] = 1;
    GCP_CUDA_TRY(launch_adam(a, elementwise_grid(a.mt), reinterpret_cast<cudaStream_t>(stream)));
    return GCP_OK;
}

gcp_status gcp_iteration(gcp_handle* h, const gcp_factors* F, gcp_loss loss, const gcp_sampling* S,
                         const int64_t* stream_dev, float* const G[GCP_MAX_MODES], float* const B[GCP_MAX_MODES],
                         float* const C[GCP_MAX_MODES], const gcp_adam_params* prm, gcp_adam_state* state,
                         gcp_stream_t stream)
{
    if (!h || !S) return GCP_ERR_INVALID_ARG;
    gcp_status st = check_modes(F, h->X.d, h->X.dims);
    if (st != GCP_OK) return st;
    if (!prm || !state || !aligned(state, 8) || !modes_ok(B, h->X.d) || !modes_ok(C, h->X.d)) return GCP_ERR_INVALID_ARG;
    if (!(prm->beta1 >= 0.f && prm->beta1 < 1.f && prm->beta2 >= 0.f && prm->beta2 < 1.f && prm->eps >= 0.f))
        return GCP_ERR_INVALID_ARG;
    if (mode_table(F, h->X.d, h->X.dims).off4[h->X.d] >= (int64_t(1) << 31))  // 32-bit element indices
        return GCP_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    AdamArgs a{};
    a.mt = mode_table(F, h->X.d, h->X.dims);
    for (int k = 0; k < h->X.d; ++k) {
        a.mt.G[k] = G[k];
        a.mt.B[k] = B[k];
        a.mt.C[k] = C[k];
    }
    a.beta1 = prm->beta1;
    a.beta2 = prm->beta2;
    a.eps = prm->eps;
    a.lower = prm->lower;
    a.eps_inside_sqrt = prm->eps_inside_sqrt;
    a.st = state;
    FoldArgs fold{};
    bool advanced = false, fused = false;
    st = grad_impl(h, F, loss, S, nullptr, stream_dev, G, s, &fold, state, &advanced, 0, -1, &a, &fused);
    if (st != GCP_OK) return st;
    if (fused) return GCP_OK;  // the gradient kernel's last blocks took the step
    for (int k = 0; k < h->X.d; ++k) {
        a.reps[k] = fold.reps[k] > 1 ? fold.reps[k] : 1;
        a.R[k] = fold.R[k];
        a.rep_stride4[k] = fold.rep_stride4[k];
    }
    a.t_advanced = advanced ? 1 : 0;
    const bool timed = h->prof_ev2 && h->prof_used2 < h->prof_cap;
    if (timed) GCP_CUDA_TRY(cudaEventRecord(h->prof_ev2[2 * h->prof_used2], s));
    if (advanced)
        GCP_CUDA_TRY(launch_adam_advanced(a, h->num_sms, s));
    else
        GCP_CUDA_TRY(launch_adam(a, elementwise_grid(a.mt), s));
    if (timed) {
        GCP_CUDA_TRY(cudaEventRecord(h->prof_ev2[2 * h->prof_used2 + 1], s));
        h->prof_used2++;
    }
    return GCP_OK;
}

static gcp_status epoch_common(const gcp_factors* F, int32_t d, const int64_t* dims, float* const B[GCP_MAX_MODES],
                               float* const C[GCP_MAX_MODES], float* const SA[GCP_MAX_MODES],
                               float* const SB[GCP_MAX_MODES], float* const SC[GCP_MAX_MODES],
                               const gcp_epoch_params* ep, int begin, gcp_adam_state* state, gcp_stream_t stream)
{
    gcp_status st = check_modes(F, d, dims);
    if (st != GCP_OK) return st;
    if (!state || !aligned(state, 8) || !modes_ok(B, d) || !modes_ok(C, d) || !modes_ok(SA, d) || !modes_ok(SB, d) ||
        !modes_ok(SC, d))
        return GCP_ERR_INVALID_ARG;
    if (!begin && (!ep || ep->tau < 0 || ep->kappa < 0)) return GCP_ERR_INVALID_ARG;
    EpochArgs a{};
    a.mt = mode_table(F, d, dims);
    for (int k = 0; k < d; ++k) {
        a.mt.B[k] = B[k];
        a.mt.C[k] = C[k];
        a.mt.SA[k] = SA[k];
        a.mt.SB[k] = SB[k];
        a.mt.SC[k] = SC[k];
    }
    if (ep) {
        a.tau = ep->tau;
        a.nu = ep->nu;
        a.kappa = ep->kappa;
    }
    a.begin = begin;
    a.st = state;
    GCP_CUDA_TRY(launch_epoch(a, elementwise_grid(a.mt), reinterpret_cast<cudaStream_t>(stream)));
    return GCP_OK;
}

gcp_status gcp_epoch_begin(const gcp_factors* F, int32_t d, const int64_t* dims, float* const B[GCP_MAX_MODES],
                           float* const C[GCP_MAX_MODES], float* const SA[GCP_MAX_MODES],
                           float* const SB[GCP_MAX_MODES], float* const SC[GCP_MAX_MODES], gcp_adam_state* state,
                           gcp_stream_t stream)
{
    return epoch_common(F, d, dims, B, C, SA, SB, SC, nullptr, 1, state, stream);
}

gcp_status gcp_epoch_end(const gcp_factors* F, int32_t d, const int64_t* dims, float* const B[GCP_MAX_MODES],
                         float* const C[GCP_MAX_MODES], float* const SA[GCP_MAX_MODES], float* const SB[GCP_MAX_MODES],
                         float* const SC[GCP_MAX_MODES], const gcp_epoch_params* ep, gcp_adam_state* state,
                         gcp_stream_t stream)
{
    return epoch_common(F, d, dims, B, C, SA, SB, SC, ep, 0, state, stream);
}

gcp_status gcp_factors_to_bf16(const gcp_factors* F, int32_t d, const int64_t* dims, gcp_stream_t stream)
{
    gcp_status st = check_modes(F, d, dims);
    if (st != GCP_OK) return st;
    for (int k = 0; k < d; ++k)
        if (!F->A_bf16[k]) return GCP_ERR_INVALID_ARG;
    ModeTable mt = mode_table(F, d, dims);
    GCP_CUDA_TRY(launch_to_bf16(mt, elementwise_grid(mt), reinterpret_cast<cudaStream_t>(stream)));
    return GCP_OK;
}

}  // extern "C"
