// Sampling kernels: packed nonzero records, the nonzero-key hash table,
// materialised draws (Algs. 1-3) and the ordered rejection pass that picks
// stratified zeros (Alg. 2 with the oversampling of Section 4.2).
#include <algorithm>

#include "gcp_draw.cuh"

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
// candidate order are kept.  Three launches, no inter-block waiting:
//   count   -- tiles of 1024 candidates in parallel: accept bits + counts;
//   scan    -- one block: exclusive scan of the tile counts; if the parallel
//              pass fell short, the same block continues through further
//              candidates in order (1024 at a time) up to cap;
//   scatter -- each tile writes its accepted candidates' slots below q.
// ---------------------------------------------------------------------------
constexpr int kZeroTile = 1024;
constexpr int kZeroBlock = 1024;  // one candidate per thread: every hash probe of a tile in flight at once

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

template <int D>
__global__ void __launch_bounds__(kZeroBlock) zero_count_kernel(const ZeroArgs a)
{
    pdl_wait();
    pdl_trigger();
    __shared__ int warp_counts[kZeroBlock / 32];
    const uint64_t stream = zero_stream(a);
    const int64_t tile = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int count = 0;
#pragma unroll 1
    for (int r = 0; r < kZeroTile / kZeroBlock; ++r) {
        const int64_t c = tile * kZeroTile + r * kZeroBlock + threadIdx.x;
        uint32_t ix[D];
        const bool acc = zero_candidate<D>(a, stream, c, ix);
        const unsigned bits = __ballot_sync(0xFFFFFFFFu, acc);
        if (lane == 0) {
            a.mask_words[tile * (kZeroTile / 32) + r * (kZeroBlock / 32) + warp] = bits;
            count += __popc(bits);
        }
    }
    if (lane == 0) warp_counts[warp] = count;
    __syncthreads();
    if (threadIdx.x == 0) {
        int total = 0;
        for (int w = 0; w < kZeroBlock / 32; ++w) total += warp_counts[w];
        a.tile_counts[tile] = total;
    }
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
__global__ void __launch_bounds__(1024) zero_scan_kernel(const ZeroArgs a)
{
    pdl_wait();
    pdl_trigger();
    __shared__ int64_t sh_warp[33];
    int64_t running = 0;
#pragma unroll 1
    for (int64_t base = 0; base < a.first_tiles; base += 1024) {
        const int64_t t = base + threadIdx.x;
        const int64_t v = t < a.first_tiles ? a.tile_counts[t] : 0;
        int64_t total;
        const int64_t ex = block_exclusive_scan_1024(v, sh_warp, &total);
        if (t < a.first_tiles) a.tile_offsets[t] = running + ex;
        running += total;
    }
    // continuation in candidate order when the parallel pass fell short
    const uint64_t stream = zero_stream(a);
    int64_t count = running;
#pragma unroll 1
    for (int64_t c0 = a.first_tiles * kZeroTile; count < a.q && c0 < a.cap; c0 += 1024) {
        const int64_t c = c0 + threadIdx.x;
        uint32_t ix[D];
        const bool acc = zero_candidate<D>(a, stream, c, ix);
        int64_t total;
        const int64_t rank = block_exclusive_scan_1024(acc ? 1 : 0, sh_warp, &total);
        if (acc && count + rank < a.q) write_zero<D>(a, count + rank, ix);
        count += total;
    }
    const int64_t kept = count < a.q ? count : a.q;
    if (threadIdx.x == 0) {
        *a.count_out = kept;
        if (kept < a.q) set_status(a.status, GCP_ERR_SAMPLE_SHORTFALL);
    }
    // unfilled slots of a shortfall carry weight 0
    if (a.out_w) {
        for (int64_t s = kept + threadIdx.x; s < a.q; s += blockDim.x) {
            uint32_t ix[D];
#pragma unroll
            for (int k = 0; k < D; ++k) ix[k] = 0u;
            write_zero<D>(a, s, ix);
            a.out_w[s] = 0.0f;
            if (a.out_x) a.out_x[s] = 0.0f;
        }
    }
}

template <int D>
__global__ void __launch_bounds__(kZeroBlock) zero_scatter_kernel(const ZeroArgs a)
{
    pdl_wait();
    pdl_trigger();
    __shared__ unsigned words[kZeroTile / 32];
    __shared__ int prefix[kZeroTile / 32];
    const int64_t tile = blockIdx.x;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < kZeroTile / 32) words[threadIdx.x] = a.mask_words[tile * (kZeroTile / 32) + threadIdx.x];
    __syncthreads();
    if (threadIdx.x < 32) {
        const int v = __popc(words[lane]);
        int inc = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int n = __shfl_up_sync(0xFFFFFFFFu, inc, off);
            if (lane >= off) inc += n;
        }
        prefix[lane] = inc - v;
    }
    __syncthreads();
    const int64_t base = a.tile_offsets[tile];
    if (base >= a.q) return;
    const uint64_t stream = zero_stream(a);
#pragma unroll 1
    for (int r = 0; r < kZeroTile / kZeroBlock; ++r) {
        const int widx = r * (kZeroBlock / 32) + (threadIdx.x >> 5);
        const unsigned wbits = words[widx];
        if (!((wbits >> lane) & 1u)) continue;
        const int64_t slot = base + prefix[widx] + __popc(wbits & ((1u << lane) - 1u));
        if (slot >= a.q) continue;
        const int64_t c = tile * kZeroTile + r * kZeroBlock + threadIdx.x;
        uint32_t ix[D];
        draw_index<D>(a.dims, a.seed, a.problem, stream, a.tag, static_cast<uint64_t>(c), a.d, ix);
        write_zero<D>(a, slot, ix);
    }
}

template <int D>
static cudaError_t zero_launch(const ZeroArgs& a, cudaStream_t s)
{
    const dim3 tiles(static_cast<unsigned>(a.first_tiles));
    cudaError_t e = launch_pdl(zero_count_kernel<D>, tiles, dim3(kZeroBlock), 0, s, a);
    if (e == cudaSuccess) e = launch_pdl(zero_scan_kernel<D>, dim3(1), dim3(1024), 0, s, a);
    if (e == cudaSuccess) e = launch_pdl(zero_scatter_kernel<D>, tiles, dim3(kZeroBlock), 0, s, a);
    return e;
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
