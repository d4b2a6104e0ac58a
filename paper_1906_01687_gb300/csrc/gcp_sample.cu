// Sampling kernels: packed nonzero records, the nonzero-key hash table,
// materialised draws (Algs. 1-3) and the ordered rejection pass that picks
// stratified zeros (Alg. 2 with the oversampling of Section 4.2).
#include <algorithm>

#include "gcp_draw.cuh"
#include "gcp_lookback.cuh"

namespace gcpk {


// ---------------------------------------------------------------------------
// Packed nonzero records: the d indices then the value's bits, padded to
// whole 16-byte words, so that a nonzero draw reads one aligned record.
// ---------------------------------------------------------------------------
struct PackArgs {
    int32_t d, rec_int4;
    int64_t nnz;
    const int32_t* idx[GCP_MAX_MODES];
    const float* vals;
    int4* recs;
};

__global__ void pack_records_kernel(const PackArgs a)
{
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= a.nnz) return;
    int words[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) words[k] = 0;
#pragma unroll
    for (int k = 0; k < GCP_MAX_MODES; ++k)
        if (k < a.d) words[k] = a.idx[k][e];
    const float v = a.vals ? a.vals[e] : 1.0f;
#pragma unroll
    for (int k = 0; k < 12; ++k)
        if (k == a.d) words[k] = __float_as_int(v);
    int4* rec = a.recs + e * a.rec_int4;
#pragma unroll
    for (int r = 0; r < 3; ++r)
        if (r < a.rec_int4) rec[r] = make_int4(words[4 * r], words[4 * r + 1], words[4 * r + 2], words[4 * r + 3]);
}

cudaError_t launch_pack_records(const gcp_tensor& X, int4* recs, int rec_int4, cudaStream_t s)
{
    PackArgs a{};
    a.d = X.d;
    a.rec_int4 = rec_int4;
    a.nnz = X.nnz;
    for (int k = 0; k < X.d; ++k) a.idx[k] = X.idx[k];
    a.vals = X.vals;
    a.recs = recs;
    const int block = 256;
    const int64_t grid = (X.nnz + block - 1) / block;
    pack_records_kernel<<<static_cast<unsigned>(grid), block, 0, s>>>(a);
    return cudaGetLastError();
}

struct HashArgs {
    const int4* recs;
    int32_t rec_int4, d;
    uint64_t strides[GCP_MAX_MODES];
    int64_t nnz;
    unsigned long long* table;
    float* table_vals;
    uint64_t mask;
    int32_t* status;
};

__global__ void hash_build_kernel(const HashArgs a)
{
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= a.nnz) return;
    const int4* rec = a.recs + e * a.rec_int4;
    int words[12];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const int4 v = r < a.rec_int4 ? rec[r] : make_int4(0, 0, 0, 0);
        words[4 * r] = v.x;
        words[4 * r + 1] = v.y;
        words[4 * r + 2] = v.z;
        words[4 * r + 3] = v.w;
    }
    uint64_t key = 0;
#pragma unroll
    for (int k = 0; k < GCP_MAX_MODES; ++k)
        if (k < a.d) key += static_cast<uint64_t>(static_cast<uint32_t>(words[k])) * a.strides[k];
    uint64_t slot = mix64(key) & a.mask;
    for (uint64_t probe = 0; probe <= a.mask; ++probe) {
        const unsigned long long prev = atomicCAS(a.table + slot, kEmptyKey, static_cast<unsigned long long>(key));
        if (prev == kEmptyKey) {
            a.table_vals[slot] = __int_as_float(words[a.d]);  // the value stored after the indices
            return;
        }
        if (prev == key) return;
        slot = (slot + 1) & a.mask;
    }
    set_status(a.status, GCP_ERR_NO_MEMORY);  // table full: cannot happen at load <= 1/2
}

cudaError_t launch_hash_build(const int4* recs, int rec_int4, int d, const uint64_t* strides, int64_t nnz,
                              unsigned long long* table, float* table_vals, uint64_t mask, int32_t* status,
                              cudaStream_t s)
{
    HashArgs a{};
    a.recs = recs;
    a.rec_int4 = rec_int4;
    a.d = d;
    for (int k = 0; k < d; ++k) a.strides[k] = strides[k];
    a.nnz = nnz;
    a.table = table;
    a.table_vals = table_vals;
    a.mask = mask;
    a.status = status;
    const int block = 256;
    hash_build_kernel<<<static_cast<unsigned>((nnz + block - 1) / block), block, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Materialised draws: entry j of the list is make_draw(j).
// ---------------------------------------------------------------------------
struct MatArgs {
    DrawArgs dr;
    int32_t* idx[GCP_MAX_MODES];
    float* x;
    float* w;
    int8_t* cls;
    int64_t first, count;
};

template <int D>
__global__ void materialise_kernel(const MatArgs a)
{
    pdl_wait();
    pdl_trigger();
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= a.count) return;
    const int64_t j = a.first + t;
    Draw<D> o;
    make_draw<D>(a.dr, j, read_stream(a.dr), o);
#pragma unroll
    for (int k = 0; k < D; ++k)
        if (k < a.dr.d) a.idx[k][j] = static_cast<int32_t>(o.ix[k]);
    a.x[j] = o.x;
    a.w[j] = o.w;
    a.cls[j] = static_cast<int8_t>(o.cls);
}

cudaError_t launch_materialise(const DrawArgs& dr, int32_t* const idx[GCP_MAX_MODES], float* x, float* w,
                               int8_t* cls, int64_t first, int64_t count, int32_t* /*status*/, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    MatArgs a{};
    a.dr = dr;
    for (int k = 0; k < GCP_MAX_MODES; ++k) a.idx[k] = idx[k];
    a.x = x;
    a.w = w;
    a.cls = cls;
    a.first = first;
    a.count = count;
    const int block = 256;
    const unsigned grid = static_cast<unsigned>((count + block - 1) / block);
    if (dr.d == 3) return launch_pdl(materialise_kernel<3>, dim3(grid), dim3(block), 0, s, a);
    if (dr.d == 4) return launch_pdl(materialise_kernel<4>, dim3(grid), dim3(block), 0, s, a);
    return launch_pdl(materialise_kernel<8>, dim3(grid), dim3(block), 0, s, a);
}

// ---------------------------------------------------------------------------
// Stratified zeros (Alg. 2): candidates c = 0, 1, 2, ... each a uniform
// multi-index from the zero-candidate stream; a candidate is accepted when
// c < cap and its linear key is not a nonzero's; the first q accepted in
// candidate order are kept.  One launch, an ordered compaction with
// decoupled look-back:
//   - tiles of 1024 candidates, one per thread (every hash probe of a tile
//     in flight at once);
//   - a block takes the next tile in launch order from a counter, so every
//     tile it waits on belongs to a block that is already running or done;
//   - the block counts its accepted candidates and publishes the count, then
//     looks back over the earlier tiles, a window of 32 per round trip
//     (adding their counts), until it meets a published prefix, and
//     publishes its own inclusive prefix;
//   - accepted candidates whose slot (prefix + rank in the tile) is below q
//     are written;
//   - the block of the last tile, once it knows the batch's total, continues
//     in candidate order (1024 at a time) up to cap if the batch fell short,
//     and records how many were kept;
//   - the last block to finish clears the tile words and counters for the
//     next call.
// Every look-back wait is bounded: after kSpinLimit polls the block records
// GCP_ERR_TIMEOUT and writes nothing (it cannot happen while the blocks it
// waits on run, which the launch-order tiles guarantee).
// ---------------------------------------------------------------------------
constexpr int kZeroTile = 1024;
constexpr int kZeroBlock = 1024;  // one candidate per thread

template <int D>
__device__ __forceinline__ bool zero_candidate(const ZeroArgs& a, uint64_t stream, int64_t c, uint32_t (&ix)[D])
{
    draw_index<D>(a.dims, a.seed, a.problem, stream, a.tag, static_cast<uint64_t>(c), a.d, ix);
    if (c >= a.cap) return false;
    uint64_t key = 0;
#pragma unroll
    for (int k = 0; k < D; ++k)
        if (k < a.d) key += static_cast<uint64_t>(ix[k]) * a.strides[k];
    if (a.obs_w) return __ldg(a.obs_w + key) != 0.0f;  // an observed entry (Section 4.4)
    return !hash_contains(a.table, a.table_mask, key);
}

// Writes accepted candidate `slot` of the destination list: a zero of Alg. 2
// (x = 0, w = zeta / q), or an observed entry (x = X(i), w = w_obs v_i).
template <int D>
__device__ __forceinline__ void write_zero(const ZeroArgs& a, int64_t slot, const uint32_t (&ix)[D])
{
    uint64_t key = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        if (k < a.d) {
            a.out_idx[k][slot] = static_cast<int32_t>(ix[k]);
            key += static_cast<uint64_t>(ix[k]) * a.strides[k];
        }
    }
    if (a.obs_w) {
        if (a.out_x) a.out_x[slot] = __ldg(a.obs_x + key);
        if (a.out_w) a.out_w[slot] = static_cast<float>(a.w_obs * static_cast<double>(__ldg(a.obs_w + key)));
        if (a.out_cls) a.out_cls[slot] = static_cast<int8_t>(GCP_CLS_UNIFORM);
        return;
    }
    if (a.out_x) a.out_x[slot] = 0.0f;
    if (a.out_w) a.out_w[slot] = a.w_zero;
    if (a.out_cls) a.out_cls[slot] = static_cast<int8_t>(GCP_CLS_STRAT_ZERO);
}

__device__ __forceinline__ uint64_t zero_stream(const ZeroArgs& a)
{
    return a.stream_dev ? static_cast<uint64_t>(*a.stream_dev) : a.stream;
}

// Block-wide exclusive scan of one int64 per thread (1024 threads); returns
// the exclusive prefix, and the block total through *total.
__device__ __forceinline__ int64_t block_exclusive_scan_1024(int64_t v, int64_t* sh_warp, int64_t* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t inc = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int64_t n = __shfl_up_sync(0xFFFFFFFFu, inc, off);
        if (lane >= off) inc += n;
    }
    if (lane == 31) sh_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int64_t w = sh_warp[lane];
        int64_t winc = w;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t n = __shfl_up_sync(0xFFFFFFFFu, winc, off);
            if (lane >= off) winc += n;
        }
        sh_warp[lane] = winc - w;  // exclusive prefix of warp totals
        if (lane == 31) sh_warp[32] = winc;
    }
    __syncthreads();
    const int64_t out = sh_warp[warp] + inc - v;
    *total = sh_warp[32];
    __syncthreads();
    return out;
}

template <int D>
__global__ void __launch_bounds__(kZeroBlock) zero_pass_kernel(const ZeroArgs a)
{
    pdl_wait();
    pdl_trigger();
    __shared__ int64_t sh_warp[33];
    __shared__ int64_t s_tile, s_excl;
    __shared__ int s_ok, s_last;
    if (threadIdx.x == 0) s_tile = static_cast<int64_t>(atomicAdd(a.tile_ctr, 1u));
    __syncthreads();
    const int64_t tile = s_tile;
    const uint64_t stream = zero_stream(a);
    uint32_t ix[D];
    const bool acc = zero_candidate<D>(a, stream, tile * kZeroTile + threadIdx.x, ix);
    int64_t total;
    const int64_t rank = block_exclusive_scan_1024(acc ? 1 : 0, sh_warp, &total);
    if (threadIdx.x < 32) {
        // warp 0 publishes this tile's count and looks back over the earlier tiles
        int64_t excl = 0;
        const bool ok = tile_lookback(a.tile_status, tile, total, excl);
        if (threadIdx.x == 0) {
            if (!ok) set_status(a.status, GCP_ERR_TIMEOUT);
            s_excl = excl;
            s_ok = ok ? 1 : 0;
        }
    }
    __syncthreads();
    const int64_t excl = s_excl;
    const bool ok = s_ok != 0;
    if (ok && acc && excl + rank < a.q) write_zero<D>(a, excl + rank, ix);

    if (tile == a.first_tiles - 1) {
        // the batch's total is known here: continue in candidate order if it fell short
        int64_t count = ok ? excl + total : 0;
#pragma unroll 1
        for (int64_t c0 = a.first_tiles * kZeroTile; ok && count < a.q && c0 < a.cap; c0 += kZeroBlock) {
            uint32_t cix[D];
            const bool cacc = zero_candidate<D>(a, stream, c0 + threadIdx.x, cix);
            int64_t ctotal;
            const int64_t crank = block_exclusive_scan_1024(cacc ? 1 : 0, sh_warp, &ctotal);
            if (cacc && count + crank < a.q) write_zero<D>(a, count + crank, cix);
            count += ctotal;
        }
        const int64_t kept = count < a.q ? count : a.q;
        if (threadIdx.x == 0) {
            *a.count_out = kept;
            if (kept < a.q) set_status(a.status, ok ? GCP_ERR_SAMPLE_SHORTFALL : GCP_ERR_TIMEOUT);
        }
        // unfilled slots of a shortfall carry weight 0
        if (a.out_w) {
            for (int64_t s = kept + threadIdx.x; s < a.q; s += blockDim.x) {
                uint32_t zix[D];
#pragma unroll
                for (int k = 0; k < D; ++k) zix[k] = 0u;
                write_zero<D>(a, s, zix);
                a.out_w[s] = 0.0f;
                if (a.out_x) a.out_x[s] = 0.0f;
            }
        }
    }

    // the last block to finish clears the tile words and counters for the next call
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(a.done_ctr, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        for (int64_t t = threadIdx.x; t < a.first_tiles; t += blockDim.x) a.tile_status[t] = 0ull;
        if (threadIdx.x == 0) {
            *a.tile_ctr = 0u;
            *a.done_ctr = 0u;
        }
    }
}

template <int D>
static cudaError_t zero_launch(const ZeroArgs& a, cudaStream_t s)
{
    return launch_pdl(zero_pass_kernel<D>, dim3(static_cast<unsigned>(a.first_tiles)), dim3(kZeroBlock), 0, s, a);
}

__global__ void __launch_bounds__(256) count_nonzero_kernel(const float* w, int64_t n, int64_t* out)
{
    int64_t local = 0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        local += w[i] != 0.0f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) local += __shfl_down_sync(0xFFFFFFFFu, local, off);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(reinterpret_cast<unsigned long long*>(out), static_cast<unsigned long long>(local));
}

cudaError_t launch_count_nonzero(const float* w, int64_t n, int64_t* out, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int64_t), s);
    if (e != cudaSuccess || n <= 0) return e;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    count_nonzero_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(w, n, out);
    return cudaGetLastError();
}

cudaError_t launch_zero_sampling(const ZeroArgs& a, cudaStream_t s)
{
    if (a.q <= 0) return cudaSuccess;
    if (a.d == 3) return zero_launch<3>(a, s);
    if (a.d == 4) return zero_launch<4>(a, s);
    return zero_launch<8>(a, s);
}

}  // namespace gcpk
