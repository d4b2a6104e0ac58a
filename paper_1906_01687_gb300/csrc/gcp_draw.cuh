// One drawn entry of Algs. 1-3: its multi-index, value x, weight w and class,
// as a pure function of the draw number j (counter-based sampling).
#pragma once

#include "gcp_device.cuh"
#include "gcp_kernels.cuh"

namespace gcpk {

// ---------------------------------------------------------------------------
// Nonzero-key hash: open addressing with linear probing over a power-of-two
// table at most half full; slot = splitmix64 finaliser of the key (Steele,
// Lea, Flood: "Fast splittable pseudorandom number generators", 2014).
// ---------------------------------------------------------------------------
constexpr unsigned long long kEmptyKey = 0xFFFFFFFFFFFFFFFFull;

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// The slot holding key, or -1 when key is not a nonzero.
__device__ __forceinline__ int64_t hash_find(const unsigned long long* __restrict__ table, uint64_t mask,
                                             uint64_t key)
{
    uint64_t slot = mix64(key) & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
        const unsigned long long v = __ldg(table + slot);
        if (v == key) return static_cast<int64_t>(slot);
        if (v == kEmptyKey) return -1;
        slot = (slot + 1) & mask;
    }
    return -1;
}

__device__ __forceinline__ bool hash_contains(const unsigned long long* __restrict__ table, uint64_t mask,
                                              uint64_t key)
{
    return hash_find(table, mask, key) >= 0;
}

template <int D>
struct Draw {
    uint32_t ix[D];
    float x;
    float w;
    int cls;
    bool valid;
};

__device__ __forceinline__ uint64_t read_stream(const DrawArgs& a)
{
    return a.stream_dev ? static_cast<uint64_t>(*a.stream_dev) : a.stream;
}

// D is the compile-time mode bound (3, 4 or 8); a.d the runtime count (a.d == D when D <= 4).
template <int D>
__device__ __forceinline__ void make_draw(const DrawArgs& a, int64_t j, uint64_t stream, Draw<D>& o)
{
    o.valid = j < a.n_total;
    o.x = 0.0f;
    o.w = 0.0f;
    o.cls = GCP_CLS_UNIFORM;
#pragma unroll
    for (int k = 0; k < D; ++k) o.ix[k] = 0u;
    if (!o.valid) return;

    if (a.src == kSrcList) {
#pragma unroll
        for (int k = 0; k < D; ++k)
            if (k < a.d) o.ix[k] = static_cast<uint32_t>(__ldg(a.lidx[k] + j));
        o.x = __ldg(a.lx + j);
        o.w = __ldg(a.lw + j);
        o.cls = __ldg(a.lcls + j);
        return;
    }

    if (a.src == kSrcObserved) {
        // Section 4.4: draw j is the j-th accepted entry of nonzero weight; its
        // value and weight (|Omega_obs| / s) v_i are read at its linear key
        uint64_t lin = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if (k < a.d) {
                o.ix[k] = static_cast<uint32_t>(__ldg(a.zidx[k] + j));
                lin += static_cast<uint64_t>(o.ix[k]) * a.strides[k];
            }
        }
        o.cls = GCP_CLS_UNIFORM;
        if (j >= *a.zcount) {  // shortfall slot: contributes nothing
            o.valid = false;
            return;
        }
        o.x = __ldg(a.X + lin);
        o.w = a.w_first * __ldg(a.W + lin);
        return;
    }

    if (a.src == kSrcEnumerate) {
        // draw j is the index with row-major linear index j (Eqs. (1.2), (4.2) over all of Omega)
        uint64_t rem = static_cast<uint64_t>(j);
#pragma unroll
        for (int k = D - 1; k >= 0; --k) {
            if (k < a.d) {
                o.ix[k] = static_cast<uint32_t>(rem % a.dims[k]);
                rem /= a.dims[k];
            }
        }
        o.x = __ldg(a.X + j);
        o.w = a.W ? __ldg(a.W + j) : 1.0f;
        o.cls = GCP_CLS_UNIFORM;
        return;
    }
    if (a.src == kSrcUniformDense || a.src == kSrcUniformSparse) {
        // Alg. 1: i_k = randi(n_k); x = X(i); weight omega / s (times v_i with entry weights)
        draw_index<D>(a.dims, a.seed, a.problem, stream, kTagUniform, static_cast<uint64_t>(j), a.d, o.ix);
        uint64_t lin = 0;
#pragma unroll
        for (int k = 0; k < D; ++k)
            if (k < a.d) lin += static_cast<uint64_t>(o.ix[k]) * a.strides[k];
        o.w = a.w_first;
        o.cls = GCP_CLS_UNIFORM;
        if (a.src == kSrcUniformDense) {
            o.x = __ldcs(a.X + lin);  // read once: evict-first
            if (a.W) o.w *= __ldg(a.W + lin);
        } else {  // a sparse tensor: the value of a nonzero, else 0
            const int64_t slot = hash_find(a.table, a.table_mask, lin);
            o.x = slot >= 0 ? __ldg(a.table_vals + slot) : 0.0f;
        }
        return;
    }

    // Algs. 2 and 3
    if (j < a.p) {
        // xi = randi(eta); the xi-th nonzero's packed record holds its indices and value
        const U64x4 b = philox4x64_10(static_cast<uint64_t>(j), stream, kTagNonzero, 0, a.seed, a.problem);
        const uint64_t xi = randi64(b.w[0], static_cast<uint64_t>(a.nnz));
        constexpr int kRecMax = (D + 1 + 3) / 4;
        int words[4 * kRecMax];
        const int4* rec = a.nz_rec + xi * static_cast<uint64_t>(a.rec_int4);
#pragma unroll
        for (int r = 0; r < kRecMax; ++r) {
            if (r < a.rec_int4) {
                const int4 v = __ldcs(rec + r);  // read once: evict-first
                words[4 * r + 0] = v.x;
                words[4 * r + 1] = v.y;
                words[4 * r + 2] = v.z;
                words[4 * r + 3] = v.w;
            } else {
                words[4 * r + 0] = words[4 * r + 1] = words[4 * r + 2] = words[4 * r + 3] = 0;
            }
        }
#pragma unroll
        for (int k = 0; k < D; ++k)
            if (k < a.d) o.ix[k] = static_cast<uint32_t>(words[k]);
        int vbits = 0;  // the value follows the d indices
        if constexpr (D <= 4) {
            vbits = words[D];
        } else {
#pragma unroll
            for (int k = 0; k < 4 * kRecMax; ++k)
                if (k == a.d) vbits = words[k];
        }
        o.x = __int_as_float(vbits);
        o.w = a.w_first;
        o.cls = a.semi ? GCP_CLS_SEMI_NZ : GCP_CLS_STRAT_NZ;
        return;
    }
    const int64_t z = j - a.p;
    o.x = 0.0f;
    o.w = a.w_second;
    if (a.semi) {
        // Alg. 3: a "zero" drawn from all of Omega, no rejection
        draw_index<D>(a.dims, a.seed, a.problem, stream, kTagSemiZero, static_cast<uint64_t>(z), a.d, o.ix);
        o.cls = GCP_CLS_SEMI_ZERO;
    } else {
        // Alg. 2: the z-th accepted zero of the rejection pass
#pragma unroll
        for (int k = 0; k < D; ++k)
            if (k < a.d) o.ix[k] = static_cast<uint32_t>(__ldg(a.zidx[k] + z));
        o.cls = GCP_CLS_STRAT_ZERO;
        if (z >= *a.zcount) {  // shortfall slot: contributes nothing
            o.w = 0.0f;
            o.valid = false;
        }
    }
}

}  // namespace gcpk
