// The fused sampled-gradient kernel: draw -> gather rows -> m_i -> y_i ->
// scatter y_i * (Hadamard product of the other modes' rows) into every G_k
// (Eq. (4.3) computed as in Algs. 1-3, with the model entry and the MTTKRP
// sharing the gathered rows).
//
// Work layout.  A warp takes 32 consecutive draws at a time.  First every
// lane computes one draw's descriptor (Philox, the nonzero record or the
// dense value gather): the random DRAM reads of 32 draws are in flight at
// once.  Then the warp splits into groups of L lanes; a group walks its L
// draws, each lane holding NC float4 column chunks of every mode's row (so
// L * NC * 4 >= rank).  With group_draws the warp instead takes 32 / L draws
// at a time, one per group, each group's lanes computing the same
// descriptor: L times more warps for the same draws, for small launches
// that are bound by latency rather than by instructions.  m_i is reduced
// across the group with shuffles; the row updates go either to shared-memory
// accumulators (modes whose whole G_k fits and is hit often: flushed once
// per CTA) or straight to global memory with 16-byte reductions
// (red.global.add.v4.f32), optionally summed first across the groups of a
// warp step that update the same 16 bytes (layouts 4 and 5).  A mode whose
// rows are hit many times per launch adds into one of several replica slabs
// (CTA b into replica b % reps), which keeps same-address contention at L2
// low; a fold kernel (or the kernel's own last blocks) then sums the
// replicas into G_k.
//
// Stratified zeros (layouts 3 and 5).  The grid's first blocks draw the
// zero candidates of Alg. 2 themselves, a tile of blockDim.x per block, and
// keep the first q accepted in candidate order by decoupled look-back
// (zero_tiles_block); the other blocks walk the nonzero draws.
//
// Early descriptors.  With a.early the first batch of each warp is drawn
// before the dependency wait (griddepcontrol.wait), while the preceding
// kernel (the previous iteration's Adam step) is still running: the draw
// reads only the data tensor, which no kernel of the sequence writes.  The
// updates, which need the preceding kernel's factors and zeroed
// accumulators, come after the wait.  When the stream word is read from
// device memory the kernel starts from a predicted stream and checks it
// after the wait.
#pragma once

#include <type_traits>

#include "gcp_adam_phase.cuh"
#include "gcp_draw.cuh"
#include "gcp_lookback.cuh"

namespace gcpk {

// One batch of the group walk.  Groups of L lanes take the batch's draws in
// turn (step b: the descriptor of lane gbase + b), or with `group` each group
// takes its own draw in one step.  m_i is reduced across the group with
// shuffles, then y_i and the d row updates follow.  verify: the batch was
// drawn from a predicted stream word, checked against `actual` before the
// first update; on a miss the batch is redrawn (jfirst: this lane's draw).
template <int D, int L, int NC, bool BF16, bool COMB>
__device__ __forceinline__ void walk_batch(const GradArgs& a, Draw<D>& my, float* (&gdst)[D], float* sG, int steps,
                                           bool group, bool& verify, uint64_t& stream, uint64_t actual,
                                           int64_t jfirst)
{
    using T = std::conditional_t<BF16, __nv_bfloat16, float>;
    constexpr unsigned kFull = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (L - 1);
    const int gbase = lane & ~(L - 1);
    const int d = D <= 4 ? D : a.dr.d;
    const int ld = a.ld, rank = a.rank;
    auto row4 = [&](int k, uint32_t i, int col) -> float4 {
        return load4(static_cast<const T*>(a.A[k]) + static_cast<size_t>(i) * ld + col);
    };
#pragma unroll 1
    for (int b = 0; b < steps; ++b) {
        const int src = group ? lane : gbase + b;
        uint32_t ix[D];
#pragma unroll
        for (int k = 0; k < D; ++k) ix[k] = __shfl_sync(kFull, my.ix[k], src);
        const float x = __shfl_sync(kFull, my.x, src);
        const float w = __shfl_sync(kFull, my.w, src);
        const int cls = __shfl_sync(kFull, my.cls, src);
        const bool valid = __shfl_sync(kFull, static_cast<int>(my.valid), src) != 0;

        // m_i = sum_j prod_k A_k(i_k, j) over this lane's chunks of the d rows.
        // With one chunk per lane the rows stay in registers for the scatter;
        // with several they are re-read there (L1 hits) to keep registers low.
        // For 3 and 4 modes with one chunk, the pairwise products of the rows
        // serve both m and the leave-one-out products of the scatter.
        constexpr bool kKeep = NC == 1;
        constexpr bool kPairs = kKeep && (D == 3 || D == 4);
        float4 r[D];
        float4 p01 = make_float4(0.f, 0.f, 0.f, 0.f), p23 = p01;
        float part = 0.0f;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int col = (gl * NC + c) * 4;
            float4 v[D];
#pragma unroll
            for (int k = 0; k < D; ++k) {
                if (k >= d) {
                    v[k] = make_float4(1.f, 1.f, 1.f, 1.f);
                } else if (valid && col < rank) {
                    v[k] = row4(k, ix[k], col);
                } else {
                    v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                if (kKeep) r[k] = v[k];
            }
            float4 prod;
            if constexpr (kPairs) {
                p01 = mul4(v[0], v[1]);
                if constexpr (D == 4) {
                    p23 = mul4(v[2], v[3]);
                    prod = mul4(p01, p23);
                } else {
                    prod = mul4(p01, v[2]);
                }
            } else {
                prod = v[0];
#pragma unroll
                for (int k = 1; k < D; ++k) prod = mul4(prod, v[k]);
            }
            part += sum4(prod);
        }
#pragma unroll
        for (int off = L / 2; off > 0; off >>= 1) part += __shfl_xor_sync(kFull, part, off);
        if (verify) {  // warp-uniform; first batch only
            verify = false;
            if (actual != stream) {  // mispredicted: redraw the batch and start it again
                stream = actual;
                make_draw<D>(a.dr, jfirst, stream, my);
                b = -1;
                continue;
            }
        }
        if (!valid) continue;  // no shuffles below this point
        const float y = entry_y(a.loss, cls, x, part, w);

#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int col = (gl * NC + c) * 4;
            if (col >= rank) continue;
            // upd[k] = y prod_{l != k} A_l(i_l, cols)
            float4 upd[D];
            if constexpr (kPairs) {
                if constexpr (D == 4) {
                    const float4 yp23 = scale4(y, p23), yp01 = scale4(y, p01);
                    upd[0] = mul4(yp23, r[1]);
                    upd[1] = mul4(yp23, r[0]);
                    upd[2] = mul4(yp01, r[3]);
                    upd[3] = mul4(yp01, r[2]);
                } else {
                    const float4 yr2 = scale4(y, r[2]);
                    upd[0] = mul4(yr2, r[1]);
                    upd[1] = mul4(yr2, r[0]);
                    upd[2] = scale4(y, p01);
                }
            } else {
                float4 rc[D];
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    if (kKeep) rc[k] = r[k];
                    else rc[k] = k < d ? row4(k, ix[k], col) : make_float4(1.f, 1.f, 1.f, 1.f);
                }
                // prefix and suffix products
                float4 pre[D], suf[D];
                pre[0] = make_float4(y, y, y, y);
#pragma unroll
                for (int k = 1; k < D; ++k) pre[k] = mul4(pre[k - 1], rc[k - 1]);
                suf[D - 1] = make_float4(1.f, 1.f, 1.f, 1.f);
#pragma unroll
                for (int k = D - 2; k >= 0; --k) suf[k] = mul4(suf[k + 1], rc[k + 1]);
#pragma unroll
                for (int k = 0; k < D; ++k) upd[k] = mul4(pre[k], suf[k]);
            }
#pragma unroll
            for (int k = 0; k < D; ++k) {
                if (k >= d) continue;
                if ((a.smem_mask >> k) & 1u) {
                    float* s = sG + a.smem_off[k] + static_cast<size_t>(ix[k]) * ld + col;
                    atomicAdd(s + 0, upd[k].x);
                    atomicAdd(s + 1, upd[k].y);
                    atomicAdd(s + 2, upd[k].z);
                    atomicAdd(s + 3, upd[k].w);
                } else if (COMB && ((a.comb_mask >> k) & 1u)) {
                    // warp-level pre-reduction: the lanes of this step that update
                    // the same 16 bytes of G_k (groups whose draws share row i_k)
                    // sum their updates and the lowest of them issues one reduction
                    const unsigned act = __activemask();
                    const unsigned key = ix[k] * static_cast<unsigned>(ld >> 2) + static_cast<unsigned>(col >> 2);
                    const unsigned same = __match_any_sync(act, key);
                    float4 sum = upd[k];
                    unsigned rest = same & ~(1u << lane);
                    const int rounds = static_cast<int>(__reduce_max_sync(act, static_cast<unsigned>(__popc(rest))));
                    for (int i = 0; i < rounds; ++i) {
                        const int src = rest ? __ffs(rest) - 1 : lane;
                        const float4 v = make_float4(__shfl_sync(act, upd[k].x, src), __shfl_sync(act, upd[k].y, src),
                                                     __shfl_sync(act, upd[k].z, src), __shfl_sync(act, upd[k].w, src));
                        if (rest) {
                            sum = add4(sum, v);
                            rest &= rest - 1u;
                        }
                    }
                    if (lane == __ffs(same) - 1) red_add4(gdst[k] + static_cast<size_t>(ix[k]) * ld + col, sum);
                } else {
                    red_add4(gdst[k] + static_cast<size_t>(ix[k]) * ld + col, upd[k]);
                }
            }
        }
    }
}

// The kernel's tail work, done by the last tail.blocks blocks to finish
// their draws instead of a launch of its own: the fold of gcp_grad's replica
// slabs into the caller's G_k, or (adam_on, gcp_iteration with a small
// factor set) the whole Adam step of Alg. 4 with the fold inside it.  After a
// block barrier one thread fences (a release that covers the block's
// reductions) and counts the block done; a
// tail block then waits (bounded: kSpinLimit polls, then GCP_ERR_TIMEOUT and
// no tail work) until every block has counted itself, and reads through L2
// (ld.cg) what other blocks wrote.  Fold: four lanes share a float4 element
// of G_k, lane s sums replicas s, s + 4, s + 8, ... in order, the four
// partial sums are added by two shuffles and lane 0 adds the total to G_k;
// the slabs are left zero.  Adam: the elements are dealt to the tail blocks'
// threads as in the split Adam kernel (four lanes per element).  At most 64
// blocks wait, fewer than the blocks one wave keeps resident, so the blocks
// still to run always find room.  The last tail block to finish clears both
// counters for the next launch (and, after an Adam step, advances the
// iteration count).
static __device__ __noinline__ void tail_work(const TailArgs& t, int rank, bool tail_ok)
{
    const unsigned K = static_cast<unsigned>(t.blocks);
    if (tail_ok && t.adam_on) {
        __threadfence();
        const AdamArgs& ad = t.adam;
        const uint32_t total4 = static_cast<uint32_t>(ad.mt.off4[ad.mt.d]);
        const uint32_t gthread = static_cast<uint32_t>(rank) * blockDim.x + threadIdx.x;
        const volatile gcp_adam_state* st = ad.st;
        const int64_t step = st->t;  // advanced by block 0 at the kernel's start
        const float alpha = st->alpha;
        const int done = st->done;
        AdamElem e;
        adam_prepare(ad, gthread / kParts, total4, gthread % kParts, e);
        adam_elements(ad, gthread, K * blockDim.x, e, step, alpha, done);
    } else if (tail_ok) {
        __threadfence();
        const FoldArgs& f = t.fold;
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        const int sub = threadIdx.x & 3;
        const unsigned quad = 0xFu << (threadIdx.x & 28);
        const int64_t first = (static_cast<int64_t>(rank) * blockDim.x + threadIdx.x) >> 2;
        const int64_t step = (static_cast<int64_t>(K) * blockDim.x) >> 2;
#pragma unroll
        for (int m = 0; m < GCP_MAX_MODES; ++m) {  // constant indices into the launch parameters
            if (m >= f.nmodes) break;
            const int64_t n4 = f.off4[m + 1] - f.off4[m];
            const uint32_t reps = f.reps[m];
            const uint64_t stride = f.rep_stride4[m];
#pragma unroll 1
            for (int64_t loc = first; loc < n4; loc += step) {  // the same trip count in all four lanes
                float4* r = reinterpret_cast<float4*>(f.R[m]) + loc;
                constexpr int kWide = 4;
                float4 acc = zero;
#pragma unroll 1
                for (uint32_t q0 = sub; q0 < reps; q0 += 4 * kWide) {
                    float4 v[kWide];
#pragma unroll
                    for (int j = 0; j < kWide; ++j) v[j] = q0 + 4 * j < reps ? __ldcg(r + (q0 + 4 * j) * stride) : zero;
#pragma unroll
                    for (int j = 0; j < kWide; ++j) {
                        acc = add4(acc, v[j]);
                        if (q0 + 4 * j < reps) r[(q0 + 4 * j) * stride] = zero;
                    }
                }
#pragma unroll
                for (int off = 1; off <= 2; off <<= 1)
                    acc = add4(acc, make_float4(__shfl_xor_sync(quad, acc.x, off), __shfl_xor_sync(quad, acc.y, off),
                                                __shfl_xor_sync(quad, acc.z, off), __shfl_xor_sync(quad, acc.w, off)));
                if (sub == 0) {
                    float4* g = reinterpret_cast<float4*>(f.G[m]) + loc;
                    *g = add4(__ldcg(g), acc);
                }
            }
        }
    } else if (threadIdx.x == 0) {
        set_status(t.status, GCP_ERR_TIMEOUT);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(t.done + 1, 1u) == K - 1) {
            if (t.adam_on) t.adam.st->iter += 1;
            t.done[0] = 0u;
            t.done[1] = 0u;
        }
    }
}

// Candidate c of the zero stream (Alg. 2), or of the observed-entry stream
// (Section 4.4), as a draw descriptor; returns whether it is accepted: c is
// below the cap and its linear key is not a nonzero's (observed: its weight
// v_i is nonzero).
template <int D>
__device__ __forceinline__ bool zt_candidate(const GradArgs& a, uint64_t stream, int64_t c, Draw<D>& o)
{
    const DrawArgs& dr = a.dr;
    draw_index<D>(dr.dims, dr.seed, dr.problem, stream, a.zt.tag, static_cast<uint64_t>(c), dr.d, o.ix);
    o.valid = false;
    o.x = 0.0f;
    o.w = dr.w_second;
    o.cls = GCP_CLS_STRAT_ZERO;
    if (c >= a.zt.cap) return false;
    uint64_t key = 0;
#pragma unroll
    for (int k = 0; k < D; ++k)
        if (k < dr.d) key += static_cast<uint64_t>(o.ix[k]) * dr.strides[k];
    if (a.zt.observed) {
        const float v = __ldg(dr.W + key);
        o.cls = GCP_CLS_UNIFORM;
        o.x = v != 0.0f ? __ldg(dr.X + key) : 0.0f;
        o.w = dr.w_first * v;
        return v != 0.0f;
    }
    return !hash_contains(dr.table, dr.table_mask, key);
}

// A block of the first a.zt.tiles (layout 3): claims the next tile of
// blockDim.x candidates, one per thread (every hash probe in flight at once),
// ranks its accepted candidates, looks back for the count accepted by the
// earlier tiles, and walks the accepted candidates whose rank in candidate
// order falls in [z_begin, z_end) as zero draws (x = 0, w = zeta / q).  The
// block of the last tile continues in candidate order up to the cap while
// fewer than q were accepted, and reports a shortfall.  The last tile to
// finish clears the tile words and counters for the next launch.
template <int D, int L, int NC, bool BF16, bool COMB>
__device__ __forceinline__ void zero_tiles_block(const GradArgs& a, float* (&gdst)[D], float* sG, uint64_t stream)
{
    __shared__ int zt_warp[32];
    __shared__ int64_t zt_tile, zt_excl;
    __shared__ int zt_ok, zt_last;
    const ZeroTileArgs& z = a.zt;
    const int64_t B = blockDim.x;
    if (threadIdx.x == 0) zt_tile = static_cast<int64_t>(atomicAdd(z.tile_ctr, 1u));
    __syncthreads();
    const int64_t tile = zt_tile;
    Draw<D> my;
    const bool acc = zt_candidate<D>(a, stream, tile * B + threadIdx.x, my);
    int total = 0;
    const int rank = block_flag_rank(acc, zt_warp, total);
    if (threadIdx.x < 32) {
        int64_t excl = 0;
        const bool ok = tile_lookback(z.tile_status, tile, total, excl);
        if (threadIdx.x == 0) {
            if (!ok) set_status(z.status, GCP_ERR_TIMEOUT);
            zt_excl = excl;
            zt_ok = ok ? 1 : 0;
        }
    }
    __syncthreads();
    const bool ok = zt_ok != 0;
    int64_t count = zt_excl;  // accepted before this thread's batch of candidates
    int ntot = total, nrank = rank;
    bool nacc = acc;
    bool verify = false;
    uint64_t st = stream;
    // the tile, then (the last tile's block only, block-uniform) continuation
    // batches of blockDim.x candidates in order while fewer than q were accepted
#pragma unroll 1
    for (int64_t c0 = z.tiles * B;; c0 += B) {
        my.valid = ok && nacc && count + nrank >= z.z_begin && count + nrank < z.z_end;
        walk_batch<D, L, NC, BF16, COMB>(a, my, gdst, sG, L, false, verify, st, stream, 0);
        if (tile != z.tiles - 1) break;
        count = ok ? count + ntot : 0;
        if (!(ok && count < z.q && c0 < z.cap)) {
            if (threadIdx.x == 0) {
                const int64_t kept = count < z.q ? count : z.q;
                if (z.count_out) *z.count_out = kept;
                if (kept < z.q) set_status(z.status, ok ? GCP_ERR_SAMPLE_SHORTFALL : GCP_ERR_TIMEOUT);
            }
            break;
        }
        nacc = zt_candidate<D>(a, stream, c0 + threadIdx.x, my);
        nrank = block_flag_rank(nacc, zt_warp, ntot);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        zt_last = atomicAdd(z.done_ctr, 1u) == static_cast<unsigned int>(z.tiles - 1);
    }
    __syncthreads();
    if (zt_last) {
        for (int64_t t = threadIdx.x; t < z.tiles; t += B) z.tile_status[t] = 0ull;
        if (threadIdx.x == 0) {
            *z.tile_ctr = 0u;
            *z.done_ctr = 0u;
        }
    }
}

// LAYOUT 0: the group walk; 1: the prefetch layout; 2: the staged walk; 3: the
// group walk with the stratified zeros made in the launch (zero_tiles_block);
// 4: the group walk with warp-level pre-reduction of same-address updates
// (GradArgs::comb_mask); 5: both 3 and 4.
// Blocks of 256 per SM the registers must allow: four (64 registers) for the
// group walk with one chunk per lane and 2 or more lanes, which fits without
// spilling; three for the other group and staged walks of at most 4 modes;
// two otherwise.
template <int D, int L, int NC>
constexpr int grad_min_blocks(int layout)
{
    return (D <= 4 && layout != 1 && layout != 2 && NC == 1 && L >= 2) ? 4 : ((D <= 4 && layout != 1) ? 3 : 2);
}

template <int D, int L, int NC, bool BF16, int LAYOUT>
__global__ void __launch_bounds__(256, grad_min_blocks<D, L, NC>(LAYOUT)) grad_kernel(const GradArgs a)
{
    constexpr bool PF = LAYOUT == 1;
    constexpr bool STAGED = LAYOUT == 2;
    constexpr bool ZT = LAYOUT == 3 || LAYOUT == 5;
    constexpr bool COMB = LAYOUT == 4 || LAYOUT == 5;
    using T = std::conditional_t<BF16, __nv_bfloat16, float>;
    extern __shared__ float4 smem4[];
    float* sG = reinterpret_cast<float*>(smem4);
    for (int i = threadIdx.x; i < a.smem_floats; i += blockDim.x) sG[i] = 0.0f;

    constexpr unsigned kFull = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (L - 1);
    const int gbase = lane & ~(L - 1);
    // layout 3: the first a.zt.tiles blocks make and walk the zeros; the
    // others walk the nonzero draws as blocks 0, 1, ... of the rest of the grid
    const bool zblock = ZT && static_cast<int64_t>(blockIdx.x) < a.zt.tiles;
    const int64_t vblock = ZT ? static_cast<int64_t>(blockIdx.x) - a.zt.tiles : static_cast<int64_t>(blockIdx.x);
    const int64_t vgrid = ZT ? static_cast<int64_t>(gridDim.x) - a.zt.tiles : static_cast<int64_t>(gridDim.x);
    const int64_t nwarps = (vgrid * blockDim.x) >> 5;
    const int d = D <= 4 ? D : a.dr.d;
    const int ld = a.ld, rank = a.rank;

    // Batches are dealt to warps interleaved across blocks (batch i of a
    // round goes to block i % gridDim.x), so that every SM of a resident
    // wave receives the same share even when the draws fill only part of it.
    // A warp takes 32 draws per batch (each lane makes one descriptor, each
    // group walks its L draws), or with group_draws 32 / L (each group makes
    // its own draw's descriptor in all its lanes and takes it at once: more
    // warps, shorter chains).
    const int per_warp = a.group_draws ? 32 / L : 32;
    const int steps = a.group_draws ? 1 : L;
    const int sub = a.group_draws ? lane / L : lane;
    // (draws j_begin .. n_total - 1: a draw range of the spec when j_begin > 0)
    const int64_t wb0 = a.dr.j_begin + (static_cast<int64_t>(threadIdx.x >> 5) * vgrid + vblock) * per_warp;
    // early descriptors for this warp: every draw of its first batch reads only
    // data written before the preceding kernel (with stratified sampling, the
    // nonzero draws j < p; the zeros come from the zero pass just before)
    // (a warp vote, so that the condition is warp-uniform by construction)
    const bool early = a.early != 0 && !zblock &&
                       __all_sync(0xFFFFFFFFu, a.dr.src != kSrcSparse || a.dr.semi || wb0 + per_warp <= a.dr.p);

    // The first batch's descriptors: before the dependency wait when early
    // (from the predicted stream word when it lives in device memory).
    uint64_t stream = 0;
    Draw<D> my;
    if (early) {
        stream = a.dr.stream_dev ? static_cast<uint64_t>(*reinterpret_cast<const volatile int64_t*>(a.stream_pred))
                                 : a.dr.stream;
        make_draw<D>(a.dr, wb0 + sub, stream, my);
    }
    pdl_wait();
    // With the Adam step in this kernel's tail the next launch (the next
    // iteration's gradient kernel) starts as soon as every block of this one
    // has triggered, long before this one ends: block 0 publishes the next
    // launch's stream prediction before it triggers (fenced, so that the next
    // launch's early reads see it).  Otherwise it is written at the end.
    if (a.tail.adam_on && a.dr.stream_dev && a.stream_pred && blockIdx.x == 0 && threadIdx.x == 0) {
        *reinterpret_cast<volatile int64_t*>(a.stream_pred) =
            *reinterpret_cast<const volatile int64_t*>(a.dr.stream_dev) + 1;
        __threadfence();
    }
    pdl_trigger();

    // gcp_iteration: this iteration's Adam step count, advanced here so that the
    // Adam kernel that follows needs no grid-wide ordering of its own
    if (a.st_advance && blockIdx.x == 0 && threadIdx.x == 0 && !a.st_advance->done) a.st_advance->t += 1;
    // The true stream word.  With early draws in the group walk, its check
    // against the prediction is deferred to just before the first update of
    // the first batch, so that the load overlaps that batch's row gathers.
    uint64_t actual = stream;
    bool verify = false;
    if (a.dr.stream_dev) {
        actual = static_cast<uint64_t>(*reinterpret_cast<const volatile int64_t*>(a.dr.stream_dev));
        if (early && !PF && !STAGED) {
            verify = true;
        } else {
            if (early && actual != stream) make_draw<D>(a.dr, wb0 + sub, actual, my);  // mispredicted: redraw
            stream = actual;
        }
    } else if (!early) {
        stream = a.dr.stream;
    }
    if (!early && !zblock) make_draw<D>(a.dr, wb0 + sub, stream, my);
    if (a.smem_floats > 0) __syncthreads();  // the shared accumulators are zero

    // this CTA's destination of each mode (its replica slab, or G_k itself)
    float* gdst[D];
#pragma unroll
    for (int k = 0; k < D; ++k)
        gdst[k] = k < d ? a.G[k] + static_cast<size_t>(blockIdx.x % a.reps[k]) * a.rep_stride[k] : nullptr;

    if constexpr (ZT) {
        if (zblock) zero_tiles_block<D, L, NC, BF16, COMB>(a, gdst, sG, stream);
    }
    // warp-uniform loop over this warp's batches (none in a zero-tile block)
    for (int64_t wb = zblock ? a.dr.n_total : wb0; wb < a.dr.n_total; wb += nwarps * per_warp) {
        if (wb != wb0) make_draw<D>(a.dr, wb + sub, stream, my);
        if constexpr (STAGED) {
            // staged walk (one chunk per lane): every lane copies its own chunk of
            // every row of its group's L draws into shared memory (cp.async), waits
            // once, and the group then walks its draws from shared memory: one
            // round trip to L2 per batch instead of one per draw, and no registers
            // held for the rows.  Layout [draw b][mode k][lane]: conflict-free.
            static_assert(NC == 1 && D <= 4, "staged walk: one chunk per lane, at most 4 modes");
            using C = std::conditional_t<BF16, uint2, float4>;
            C* stage = reinterpret_cast<C*>(smem4) + static_cast<size_t>(threadIdx.x >> 5) * (L * D * 32);
            const int col = gl * 4;
            const bool colok = col < rank;
#pragma unroll
            for (int b = 0; b < L; ++b) {
                const int src = gbase + b;
                const bool v = __shfl_sync(kFull, static_cast<int>(my.valid), src) != 0;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const uint32_t i = __shfl_sync(kFull, my.ix[k], src);
                    if (v && colok) {
                        const T* g = static_cast<const T*>(a.A[k]) + static_cast<size_t>(i) * ld + col;
                        if constexpr (BF16)
                            cp_async8(stage + (b * D + k) * 32 + lane, g);
                        else
                            cp_async16(stage + (b * D + k) * 32 + lane, g);
                    }
                }
            }
            cp_async_wait_all();
#pragma unroll 1
            for (int b = 0; b < L; ++b) {
                const int src = gbase + b;
                uint32_t ix[D];
#pragma unroll
                for (int k = 0; k < D; ++k) ix[k] = __shfl_sync(kFull, my.ix[k], src);
                const float x = __shfl_sync(kFull, my.x, src);
                const float w = __shfl_sync(kFull, my.w, src);
                const int cls = __shfl_sync(kFull, my.cls, src);
                const bool valid = __shfl_sync(kFull, static_cast<int>(my.valid), src) != 0;
                float4 r[D];
#pragma unroll
                for (int k = 0; k < D; ++k)
                    r[k] = (valid && colok) ? staged4(stage + (b * D + k) * 32 + lane) : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 p01 = mul4(r[0], r[1]);
                const float4 p23 = D == 4 ? mul4(r[2], r[3]) : r[D - 1];
                float part = sum4(mul4(p01, p23));
#pragma unroll
                for (int off = L / 2; off > 0; off >>= 1) part += __shfl_xor_sync(kFull, part, off);
                if (!valid || !colok) continue;  // no shuffles below this point in the iteration
                const float y = entry_y(a.loss, cls, x, part, w);
                float4 upd[D];
                if constexpr (D == 4) {
                    const float4 yp23 = scale4(y, p23), yp01 = scale4(y, p01);
                    upd[0] = mul4(yp23, r[1]);
                    upd[1] = mul4(yp23, r[0]);
                    upd[2] = mul4(yp01, r[3]);
                    upd[3] = mul4(yp01, r[2]);
                } else {
                    const float4 yr2 = scale4(y, r[2]);
                    upd[0] = mul4(yr2, r[1]);
                    upd[1] = mul4(yr2, r[0]);
                    upd[2] = scale4(y, p01);
                }
#pragma unroll
                for (int k = 0; k < D; ++k)
                    red_add4(gdst[k] + static_cast<size_t>(ix[k]) * ld + col, upd[k]);
            }
            continue;
        }
        if constexpr (PF) {
            // prefetch layout (one chunk per lane): the descriptors and row loads
            // of all L draws of the group are issued before any is consumed, so
            // the group waits for one round trip to L2 instead of L in turn
            static_assert(NC == 1 && D <= 4, "prefetch layout: one chunk per lane, at most 4 modes");
            const int col = gl * 4;
            uint32_t pix[L][D];
            float px[L], pw[L];
            int pcls[L];
            bool pv[L];
            float4 rows[L][D];
#pragma unroll
            for (int b = 0; b < L; ++b) {
                const int src = gbase + b;
#pragma unroll
                for (int k = 0; k < D; ++k) pix[b][k] = __shfl_sync(kFull, my.ix[k], src);
                px[b] = __shfl_sync(kFull, my.x, src);
                pw[b] = __shfl_sync(kFull, my.w, src);
                pcls[b] = __shfl_sync(kFull, my.cls, src);
                pv[b] = __shfl_sync(kFull, static_cast<int>(my.valid), src) != 0;
#pragma unroll
                for (int k = 0; k < D; ++k)
                    rows[b][k] = (pv[b] && col < rank)
                                     ? load4(static_cast<const T*>(a.A[k]) + static_cast<size_t>(pix[b][k]) * ld + col)
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int b = 0; b < L; ++b) {
                const float4 p01 = mul4(rows[b][0], rows[b][1]);
                const float4 p23 = D == 4 ? mul4(rows[b][2], rows[b][3]) : rows[b][D - 1];
                float part = sum4(mul4(p01, p23));
#pragma unroll
                for (int off = L / 2; off > 0; off >>= 1) part += __shfl_xor_sync(kFull, part, off);
                if (!pv[b] || col >= rank) continue;  // no shuffles below this point in the iteration
                const float y = entry_y(a.loss, pcls[b], px[b], part, pw[b]);
                float4 upd[D];
                if constexpr (D == 4) {
                    const float4 yp23 = scale4(y, p23), yp01 = scale4(y, p01);
                    upd[0] = mul4(yp23, rows[b][1]);
                    upd[1] = mul4(yp23, rows[b][0]);
                    upd[2] = mul4(yp01, rows[b][3]);
                    upd[3] = mul4(yp01, rows[b][2]);
                } else {
                    const float4 yr2 = scale4(y, rows[b][2]);
                    upd[0] = mul4(yr2, rows[b][1]);
                    upd[1] = mul4(yr2, rows[b][0]);
                    upd[2] = scale4(y, p01);
                }
#pragma unroll
                for (int k = 0; k < D; ++k)
                    red_add4(gdst[k] + static_cast<size_t>(pix[b][k]) * ld + col, upd[k]);
            }
            continue;
        }
        walk_batch<D, L, NC, BF16, COMB>(a, my, gdst, sG, steps, a.group_draws != 0, verify, stream, actual, wb + sub);
    }

    // the prediction for the next launch that reads its stream word from memory
    if (!a.tail.adam_on && a.dr.stream_dev && a.stream_pred && blockIdx.x == 0 && threadIdx.x == 0)
        *reinterpret_cast<volatile int64_t*>(a.stream_pred) = static_cast<int64_t>(actual + 1);
    if (a.smem_mask != 0) {
        __syncthreads();
#pragma unroll 1
        for (int k = 0; k < d; ++k) {
            if (!((a.smem_mask >> k) & 1u)) continue;
            const int n4 = static_cast<int>(a.dr.dims[k]) * ld / 4;
            const float4* s = reinterpret_cast<const float4*>(sG + a.smem_off[k]);
            float4* g =
                reinterpret_cast<float4*>(a.G[k] + static_cast<size_t>(blockIdx.x % a.reps[k]) * a.rep_stride[k]);
            for (int e = threadIdx.x; e < n4; e += blockDim.x) {
                const float4 v = s[e];
                if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f) red_add4(reinterpret_cast<float*>(g + e), v);
            }
        }
    }
    if (a.tail.blocks > 0) {
        // count this block done (after a block barrier one thread fences: a
        // release that covers the block's reductions); the last tail.blocks to
        // count wait, bounded, for every block, then do the tail work
        __shared__ int tail_rank, tail_ok;
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned grid = gridDim.x;
            __threadfence();
            const unsigned ticket = atomicAdd(a.tail.done, 1u);
            const int rank = static_cast<int>(ticket) - static_cast<int>(grid - static_cast<unsigned>(a.tail.blocks));
            int ok = 1;
            if (rank >= 0) {
                int spins = 0;
                while (*reinterpret_cast<volatile unsigned int*>(a.tail.done) < grid) {
                    if (++spins > kSpinLimit) {
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            tail_rank = rank;
            tail_ok = ok;
        }
        __syncthreads();
        if (tail_rank >= 0) {
            // the tail's arguments in shared memory: a called function reaches
            // the launch parameters only through generic loads, which are slow
            __shared__ TailArgs s_tail;
            if (threadIdx.x == 0) s_tail = a.tail;
            __syncthreads();
            tail_work(s_tail, tail_rank, tail_ok != 0);
        }
    }
}

#define GCP_GRAD_CONFIGS(X) \
    X(1, 1) X(1, 2) X(1, 3) X(1, 4) X(2, 1) X(2, 2) X(4, 1) X(4, 2) X(8, 1) X(8, 2) X(16, 1) X(32, 1) X(32, 2)

// The prefetch layout exists for one chunk per lane with 2 or 4 lanes (3 or 4 modes).
template <int D, bool BF16>
const void* grad_kernel_ptr(int L, int NC, int layout)
{
    if (layout == 2) {  // the staged walk: one chunk per lane, at most 8 lanes, at most 4 modes
        if constexpr (D <= 4) {
            if (NC == 1 && L == 1) return reinterpret_cast<const void*>(&grad_kernel<D, 1, 1, BF16, 2>);
            if (NC == 1 && L == 2) return reinterpret_cast<const void*>(&grad_kernel<D, 2, 1, BF16, 2>);
            if (NC == 1 && L == 4) return reinterpret_cast<const void*>(&grad_kernel<D, 4, 1, BF16, 2>);
            if (NC == 1 && L == 8) return reinterpret_cast<const void*>(&grad_kernel<D, 8, 1, BF16, 2>);
        }
        return nullptr;
    }
    if (layout == 1) {
        if constexpr (D <= 4) {
            if (NC == 1 && L == 2) return reinterpret_cast<const void*>(&grad_kernel<D, 2, 1, BF16, 1>);
            if (NC == 1 && L == 4) return reinterpret_cast<const void*>(&grad_kernel<D, 4, 1, BF16, 1>);
        }
        return nullptr;
    }
    if (layout != 0) return nullptr;
#define GCP_CASE(LL, CC) \
    if (L == LL && NC == CC) return reinterpret_cast<const void*>(&grad_kernel<D, LL, CC, BF16, 0>);
    GCP_GRAD_CONFIGS(GCP_CASE)
#undef GCP_CASE
    return nullptr;
}

// The group-walk variants of layouts 3, 4 and 5 (LAYOUT), at most 4 modes:
// instantiated in translation units of their own.
template <int D, bool BF16, int LAYOUT>
const void* grad_kernel_ptr_variant(int L, int NC)
{
    static_assert(D <= 4 && LAYOUT >= 3 && LAYOUT <= 5, "layouts 3-5: at most 4 modes");
#define GCP_CASE(LL, CC) \
    if (L == LL && NC == CC) return reinterpret_cast<const void*>(&grad_kernel<D, LL, CC, BF16, LAYOUT>);
    GCP_GRAD_CONFIGS(GCP_CASE)
#undef GCP_CASE
    return nullptr;
}

}  // namespace gcpk
