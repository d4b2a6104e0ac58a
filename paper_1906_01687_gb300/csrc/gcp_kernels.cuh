// Kernel argument blocks and the host-side launchers shared by the C ABI
// (gcp_api.cu) and the kernel translation units.
#pragma once

#include <cstdint>
#include <utility>
#include <cuda_runtime.h>

#include "../../include/gcp.h"

namespace gcpk {

// Where the drawn entries of a gradient come from.
enum Source : int32_t {
    kSrcUniformDense = 0,  // Alg. 1 over a dense tensor, generated in-kernel
    kSrcSparse = 1,        // Algs. 2/3: nonzeros generated in-kernel, zeros generated (semi) or listed (stratified)
    kSrcList = 2,          // a materialised list
    kSrcUniformSparse = 3, // Alg. 1 over a sparse tensor: values looked up in the nonzero hash
    kSrcEnumerate = 4,     // every index of a dense tensor once, weight 1 (or v_i): the full gradient
    kSrcObserved = 5       // Section 4.4: the listed entries of nonzero weight (from the rejection pass)
};

struct DrawArgs {
    int32_t d;
    int32_t src;
    int32_t semi;         // kSrcSparse: 1 = semi-stratified, 0 = stratified
    int32_t rec_int4;     // int4 words per packed nonzero record
    uint32_t dims[GCP_MAX_MODES];
    uint64_t strides[GCP_MAX_MODES];  // row-major strides of the linear index
    int64_t p;            // nonzero draws: j in [0, p)
    int64_t n_total;      // end of the draws this launch takes (exclusive)
    int64_t j_begin;      // first draw this launch takes (a draw range; 0 = from the start)
    uint64_t seed, problem, stream;
    const int64_t* stream_dev;
    float w_first;        // uniform: omega/s; sparse: eta/p
    float w_second;       // stratified: zeta/q; semi: omega/q
    const float* X;       // dense values
    const float* W;       // dense entry weights (Eq. (4.5)), or null
    const unsigned long long* table;  // nonzero key hash (kSrcUniformSparse)
    const float* table_vals;          // the value of each occupied slot
    uint64_t table_mask;
    const int4* nz_rec;   // packed nonzero records
    int64_t nnz;
    const int32_t* zidx[GCP_MAX_MODES];  // stratified zero list (scratch)
    const int64_t* zcount;                // accepted zeros in the list
    const int32_t* lidx[GCP_MAX_MODES];  // kSrcList
    const float* lx;
    const float* lw;
    const int8_t* lcls;
};

// Stratified zeros (Alg. 2) or observed entries (Section 4.4) made inside the
// gradient launch instead of listed by a separate pass: the grid's first
// `tiles` blocks each take a tile of blockDim.x consecutive candidates (tiles
// numbered in the order the blocks claim them), count the accepted ones,
// learn how many earlier tiles accepted by decoupled look-back, and walk the
// accepted candidates whose rank in candidate order is in [z_begin, z_end)
// as zero draws; the block of the last tile continues in candidate order
// when the tiles accepted fewer than q.
struct ZeroTileArgs {
    int64_t tiles;            // 0: off (zeros come from a separate pass's list)
    int64_t cap;              // candidates allowed in total (64 batches)
    int64_t q;                // zeros (entries) kept
    int64_t z_begin, z_end;   // ranks of the kept candidates that are this launch's draws
    uint32_t tag;             // candidate stream: zero candidates, or observed-entry candidates
    int32_t observed;         // 1: accept v_i != 0 (dr.W); x = X(i), w = dr.w_first v_i
    unsigned long long* tile_status;  // per tile: flag and count or inclusive prefix (zero between launches)
    unsigned int* tile_ctr;   // next tile to claim (zero between launches)
    unsigned int* done_ctr;   // tiles finished (zero between launches)
    int64_t* count_out;       // accepted candidates kept (<= q)
    int32_t* status;
};

// Folds replica slabs into G: G_k += sum_r R_k[r]; R_k[r] = 0 (fixed order r = 0, 1, ...).
struct FoldArgs {
    int32_t nmodes;
    int32_t pad;
    int64_t off4[GCP_MAX_MODES + 1];  // prefix of the folded modes' float4 counts
    uint32_t reps[GCP_MAX_MODES];
    uint64_t rep_stride4[GCP_MAX_MODES];
    float* R[GCP_MAX_MODES];
    float* G[GCP_MAX_MODES];
};

struct ModeTable {
    int32_t d, ld, rank, pad;
    int64_t off4[GCP_MAX_MODES + 1];  // prefix of n_k * ld / 4
    float* A[GCP_MAX_MODES];
    float* B[GCP_MAX_MODES];
    float* C[GCP_MAX_MODES];
    float* G[GCP_MAX_MODES];
    uint16_t* Abf[GCP_MAX_MODES];
    float* SA[GCP_MAX_MODES];
    float* SB[GCP_MAX_MODES];
    float* SC[GCP_MAX_MODES];
};

struct AdamArgs {
    ModeTable mt;
    float beta1, beta2, eps, lower;
    int32_t eps_inside_sqrt;
    gcp_adam_state* st;
    // replica slabs still to be folded into G (gcp_iteration): mode k's gradient
    // is G_k + sum_r R_k[r] when reps[k] > 1; the slabs are zeroed after use
    uint32_t reps[GCP_MAX_MODES];
    uint64_t rep_stride4[GCP_MAX_MODES];
    float* R[GCP_MAX_MODES];
    // 1 (gcp_iteration): the gradient kernel of the same iteration has already
    // advanced st->t, so no block of this launch has to wait for the others
    int32_t t_advanced;
};

// Work the last `blocks` blocks of a gradient launch to finish take on after
// every block's reductions (the kernel tail): fold `fold`'s replica slabs
// into G, or (adam_on) take the Adam step `adam`.
struct TailArgs {
    FoldArgs fold;
    AdamArgs adam;
    unsigned int* done;   // [0] blocks finished, [1] tail blocks finished (zero between launches)
    int32_t* status;      // status word (a wait that ran out)
    int32_t blocks;       // 0: no tail work; else 1..64
    int32_t adam_on;
};

struct GradArgs {
    DrawArgs dr;
    int32_t ld, rank, loss, smem_floats;
    const void* A[GCP_MAX_MODES];  // float or bf16 rows
    float* G[GCP_MAX_MODES];       // destination of mode k: the caller's G_k or a replica slab
    uint32_t reps[GCP_MAX_MODES];  // replicas of mode k's destination (CTA b adds into replica b % reps)
    uint64_t rep_stride[GCP_MAX_MODES];  // floats between replicas
    uint32_t smem_mask;            // bit k: mode k accumulates in shared memory first
    uint32_t comb_mask;            // bit k: same-address updates of a warp step are summed before the reduction
    uint32_t smem_off[GCP_MAX_MODES];
    int32_t group_draws;           // 1: each group of L lanes takes its own draw (32/L draws per warp step)
    int32_t early;                 // 1: each warp's first descriptors are made before the dependency wait
    int64_t* stream_pred;          // handle word: predicted stream of the next launch with dr.stream_dev
    gcp_adam_state* st_advance;    // gcp_iteration: the Adam state whose step count t this launch advances
    ZeroTileArgs zt;               // layout 3: the zeros made in this launch (dr.n_total then ends the nonzeros)
    TailArgs tail;                 // blocks > 0: work the last blocks to finish do instead of a launch
};

struct LossArgs {
    DrawArgs dr;  // always kSrcList
    int32_t ld, rank, loss, pad;
    const void* A[GCP_MAX_MODES];
    double* partials;     // one per block
    unsigned int* ticket; // zero between launches
    double* out;
};


struct EpochArgs {
    ModeTable mt;
    int64_t tau;
    float nu;
    int32_t kappa;
    int32_t begin;  // 1: epoch_begin (snapshot only), 0: epoch_end
    gcp_adam_state* st;
};

// Stratified zero sampling (Alg. 2 with the oversampling of Section 4.2).
struct ZeroArgs {
    int32_t d;
    int32_t pad;
    uint32_t dims[GCP_MAX_MODES];
    uint64_t strides[GCP_MAX_MODES];
    uint64_t seed, problem, stream;
    const int64_t* stream_dev;
    int64_t q;
    int64_t first_tiles;      // tiles of 1024 candidates examined in parallel (one block each)
    int64_t cap;              // candidates allowed in total (64 batches)
    const unsigned long long* table;  // nonzero key hash (open addressing)
    uint64_t table_mask;
    uint32_t tag;             // candidate stream: zero candidates, or observed-entry candidates
    const float* obs_w;       // observed-entry pass (Section 4.4): accept v_i != 0 (else: not a nonzero)
    const float* obs_x;       //   and list x = X(i), w = w_obs v_i
    double w_obs;             //   |Omega_obs| / q (the list weight is rounded once, from FP64)
    unsigned long long* tile_status;  // per tile: flag and count or inclusive prefix (zero between calls)
    unsigned int* tile_ctr;   // next tile to take (zero between calls)
    unsigned int* done_ctr;   // blocks finished (zero between calls)
    int64_t* count_out;       // accepted zeros kept (<= q)
    int32_t* status;
    // destination list (zero draw e goes to slot e)
    int32_t* out_idx[GCP_MAX_MODES];
    float* out_x;
    float* out_w;
    int8_t* out_cls;
    float w_zero;
};

// Launches a kernel with programmatic stream serialization (see pdl_wait).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

inline cudaError_t launch_pdl_ptr(const void* kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t s, void** args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, kernel, args);
}

// Launchers (defined in the kernel translation units).
// layout: 0 the group walk, 1 the prefetch layout, 2 the staged walk, 3 the group walk with
// the stratified zeros made in the launch (ZeroTileArgs), 4 the group walk with warp-level
// pre-reduction (comb_mask), 5 both
cudaError_t launch_grad(const GradArgs& a, int D, int L, int NC, bool bf16, int layout, int grid, int block,
                        size_t smem, cudaStream_t s);
cudaError_t grad_occupancy(int D, int L, int NC, bool bf16, int layout, int block, size_t smem, int* blocks_per_sm);
bool grad_has_config(int D, int L, int NC, int layout);

cudaError_t launch_fold(const FoldArgs& a, int grid, cudaStream_t s);
cudaError_t launch_loss(const LossArgs& a, bool bf16, int grid, int block, cudaStream_t s);
cudaError_t launch_materialise(const DrawArgs& a, int32_t* const idx[GCP_MAX_MODES], float* x, float* w,
                               int8_t* cls, int64_t first, int64_t count, int32_t* status, cudaStream_t s);
cudaError_t launch_zero_sampling(const ZeroArgs& a, cudaStream_t s);
// Number of nonzero entries of w[0..n) into *out (device), stream-ordered.
cudaError_t launch_count_nonzero(const float* w, int64_t n, int64_t* out, cudaStream_t s);
cudaError_t launch_hash_build(const int4* recs, int rec_int4, int d, const uint64_t* strides, int64_t nnz,
                              unsigned long long* table, float* table_vals, uint64_t mask, int32_t* status,
                              cudaStream_t s);
cudaError_t launch_pack_records(const gcp_tensor& X, int4* recs, int rec_int4, cudaStream_t s);
cudaError_t launch_adam(const AdamArgs& a, int grid, cudaStream_t s);
cudaError_t launch_adam_advanced(const AdamArgs& a, int num_sms, cudaStream_t s);
cudaError_t launch_epoch(const EpochArgs& a, int grid, cudaStream_t s);
cudaError_t launch_state_init(gcp_adam_state* st, float alpha, cudaStream_t s);
cudaError_t launch_to_bf16(const ModeTable& mt, int grid, cudaStream_t s);

}  // namespace gcpk
