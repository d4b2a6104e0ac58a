/*
 * FP64 CPU oracle for the sampled GCP gradient (Kolda & Hong, "Stochastic
 * Gradients for Large-Scale Tensor Decomposition", arXiv:1906.01687).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The
 * product (the CUDA library under paper_1906_01687_gb300/) never calls it and
 * shares no code, header, table or constant generator with it.
 *
 * Everything here is plain, slow and written to be checked against the paper
 * by eye: FP64 throughout, no blocking, no fusion, one loop per formula.
 *
 * Conventions shared with the CUDA path only through their written
 * definition (both sides implement them independently):
 *   - indices are 0-based; linear keys are row-major (last mode fastest);
 *   - random numbers come from Philox4x64-10 (Salmon, Moraes, Dror, Shaw,
 *     SC'11) with key = (seed, problem) and counter = (j, stream, tag, g),
 *     where j is the draw (or candidate) number, stream the iteration, tag
 *     the sampling stream and g = k / 4 the group of modes; mode k of a draw
 *     takes word k % 4 of that block;
 *   - randi(n) = floor(W * n / 2^64) for a 64-bit word W (multiply-high).
 *
 * Parity status: every function is pinned, by a check that does not go
 * through this file's own formula (tests/):
 *   orc_philox4x64          numpy.random.Philox, 56 counters and keys
 *   orc_randi               the defining partition property at exact
 *                           interval boundaries, in Python integers
 *   orc_draw_*, orc_sample, a pure-Python twin (numpy's Philox, Python
 *   orc_linear_key,         integers, a Python set and dict) for all four
 *   orc_sparse_value,       samplers, 40 random configurations of 2-8
 *   orc_count_observed      modes, candidate counts, the shortfall and the
 *                           exact 64-batch cap
 *   orc_sorted_keys,        every linear key of a small dense tensor
 *   orc_is_nonzero
 *   orc_loss_f, orc_loss_g  scipy's likelihoods, closed forms, central
 *                           differences
 *   orc_model_value,        numpy.einsum MTTKRP of the full gradient (also
 *   orc_full_grad           the textbook 2 (M - X)_(k) Z_k), weighted form
 *   orc_entry_y/f,          enumeration identities (each index once, weight
 *   orc_grad_from_samples,  1, gives the full gradient and objective),
 *   orc_loss_from_samples   finite differences of the estimate, Monte-Carlo
 *                           unbiasedness
 *   orc_*_abs_from_samples  bounds and equalities with sign-definite terms
 *   orc_adam_step           torch.optim.Adam, the closed-form first step,
 *                           the second step's bias correction, projection
 * and tests/test_pins_catch_mistakes.py requires each of 59 planted mistakes
 * in this file to fail one of these pins.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_D 8

/* sampling streams (the tag word of the Philox counter) */
#define ORC_TAG_UNIFORM 0u
#define ORC_TAG_NONZERO 1u
#define ORC_TAG_ZERO_CANDIDATE 2u
#define ORC_TAG_SEMI_ZERO 3u
#define ORC_TAG_OBSERVED 4u

/* sampler kinds */
#define ORC_UNIFORM 0
#define ORC_STRATIFIED 1
#define ORC_SEMI_STRATIFIED 2
#define ORC_OBSERVED 3

/* classes of a drawn entry; they decide which form of y_i applies */
#define ORC_CLS_UNIFORM 0     /* Alg. 1: weight omega/s, g(x,m)            */
#define ORC_CLS_STRAT_NZ 1    /* Alg. 2 nonzero: weight eta/p, g(x,m)      */
#define ORC_CLS_STRAT_ZERO 2  /* Alg. 2 zero: weight zeta/q, g(0,m)        */
#define ORC_CLS_SEMI_NZ 3     /* Alg. 3 nonzero: eta/p, g(x,m) - g(0,m)    */
#define ORC_CLS_SEMI_ZERO 4   /* Alg. 3 "zero": omega/q, g(0,m)            */

/* losses */
#define ORC_GAUSSIAN 0
#define ORC_BERNOULLI_LOGIT 1
#define ORC_POISSON_LOG 2
#define ORC_BERNOULLI_ODDS 3
#define ORC_POISSON_IDENTITY 4
#define ORC_GAMMA 5
#define ORC_BETA_HALF 6

/* The losses with an odds or identity link need m > 0; they are evaluated
   at m + ORC_M_EPS, so that m = 0 (reachable under the projection
   max(A, 0) of Alg. 4) stays finite. */
#define ORC_M_EPS 1e-10

/* status codes */
#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_SHORTFALL 4

/* ------------------------------------------------------------------------ */
/* Philox4x64-10, from the round function published by Salmon et al.       */
/* Pinned at test time against numpy.random.Philox (an independent          */
/* implementation of the same generator).                                   */
/* ------------------------------------------------------------------------ */

static void mul128(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void orc_philox4x64(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t hi0, lo0, hi1, lo1;
        mul128(M0, c0, &hi0, &lo0);
        mul128(M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        uint64_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* randi(n) of Section 4.1, 0-based: floor(W * n / 2^64). */
uint64_t orc_randi(uint64_t word, uint64_t n)
{
    uint64_t hi, lo;
    mul128(word, n, &hi, &lo);
    return hi;
}

/* The d mode indices of draw j (Section 4.1: i_k = randi(n_k)). */
void orc_draw_multi_index(int d, const int64_t *dims, uint64_t seed, uint64_t problem,
                          uint64_t stream, uint32_t tag, uint64_t j, int64_t *idx)
{
    uint64_t key[2] = {seed, problem};
    for (int k = 0; k < d; ++k) {
        uint64_t ctr[4] = {j, stream, (uint64_t)tag, (uint64_t)(k / 4)};
        uint64_t w[4];
        orc_philox4x64(ctr, key, w);
        idx[k] = (int64_t)orc_randi(w[k % 4], (uint64_t)dims[k]);
    }
}

/* xi = randi(eta) of Algs. 2 and 3 (0-based position in the COO list). */
int64_t orc_draw_nonzero(int64_t nnz, uint64_t seed, uint64_t problem, uint64_t stream, uint64_t j)
{
    uint64_t key[2] = {seed, problem};
    uint64_t ctr[4] = {j, stream, (uint64_t)ORC_TAG_NONZERO, 0};
    uint64_t w[4];
    orc_philox4x64(ctr, key, w);
    return (int64_t)orc_randi(w[0], (uint64_t)nnz);
}

/* Row-major linear index of a multi-index (Section 3.2). */
uint64_t orc_linear_key(int d, const int64_t *dims, const int64_t *idx)
{
    uint64_t key = 0;
    for (int k = 0; k < d; ++k) key = key * (uint64_t)dims[k] + (uint64_t)idx[k];
    return key;
}

/* ------------------------------------------------------------------------ */
/* Losses f(x,m) and g = df/dm.                                             */
/* Gaussian: Section 1, f = (x-m)^2.  Bernoulli-logit and Poisson-log are   */
/* the log-link forms of the cited GCP paper (HoKoDu20); this paper prints  */
/* the odds/identity-link forms, also here: Bernoulli-odds, Poisson-        */
/* identity, Gamma (Section 1) and the beta-divergence with beta = 1/2 as   */
/* Section 5.3 prints it.  Pinned by scipy's distributions, closed forms    */
/* and finite differences in the CPU tests.                                 */
/* ------------------------------------------------------------------------ */

double orc_loss_f(int loss, double x, double m)
{
    double mp = m + ORC_M_EPS;
    switch (loss) {
    case ORC_BERNOULLI_ODDS: /* Section 1: log(m + 1) - x log m, m the odds */
        return log(mp + 1.0) - x * log(mp);
    case ORC_POISSON_IDENTITY: /* Section 1: m - x log m */
        return mp - x * log(mp);
    case ORC_GAMMA: /* Section 1 and Section 5.2's caption: x / m + log m */
        return x / mp + log(mp);
    case ORC_BETA_HALF: /* Section 5.3: 2 m^(1/2) + 2 x m^(-1/2) */
        return 2.0 * sqrt(mp) + 2.0 * x / sqrt(mp);
    case ORC_GAUSSIAN:
        return (x - m) * (x - m);
    case ORC_BERNOULLI_LOGIT: {
        /* log(1 + e^m) - x m, with log(1+e^m) = max(m,0) + log1p(e^{-|m|}) */
        double softplus = (m > 0 ? m : 0.0) + log1p(exp(-fabs(m)));
        return softplus - x * m;
    }
    case ORC_POISSON_LOG:
        return exp(m) - x * m;
    }
    return NAN;
}

double orc_loss_g(int loss, double x, double m)
{
    double mp = m + ORC_M_EPS;
    switch (loss) {
    case ORC_BERNOULLI_ODDS:
        return 1.0 / (mp + 1.0) - x / mp;
    case ORC_POISSON_IDENTITY:
        return 1.0 - x / mp;
    case ORC_GAMMA:
        return -x / (mp * mp) + 1.0 / mp;
    case ORC_BETA_HALF:
        return 1.0 / sqrt(mp) - x / (mp * sqrt(mp));
    case ORC_GAUSSIAN:
        return 2.0 * (m - x);
    case ORC_BERNOULLI_LOGIT: {
        double sig = m >= 0 ? 1.0 / (1.0 + exp(-m)) : exp(m) / (1.0 + exp(m));
        return sig - x;
    }
    case ORC_POISSON_LOG:
        return exp(m) - x;
    }
    return NAN;
}

/* ------------------------------------------------------------------------ */
/* Model entry m_i = sum_j prod_k A_k(i_k, j)  (Eq. (1.1); Alg. 1).             */
/* A is all factor matrices concatenated, mode k an n_k x r row-major block. */
/* ------------------------------------------------------------------------ */

static void mode_offsets(int d, const int64_t *dims, int rank, int64_t *off)
{
    off[0] = 0;
    for (int k = 1; k < d; ++k) off[k] = off[k - 1] + dims[k - 1] * rank;
}

double orc_model_value(int d, const int64_t *dims, int rank, const double *A, const int64_t *idx)
{
    int64_t off[ORC_MAX_D];
    mode_offsets(d, dims, rank, off);
    double m = 0.0;
    for (int j = 0; j < rank; ++j) {
        double prod = 1.0;
        for (int k = 0; k < d; ++k) prod *= A[off[k] + idx[k] * rank + j];
        m += prod;
    }
    return m;
}

/* ------------------------------------------------------------------------ */
/* Nonzero membership for stratified zero sampling (Section 4.2): the      */
/* nonzero linear keys, sorted, then a binary search.                       */
/* ------------------------------------------------------------------------ */

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* coo_idx is nnz x d row-major.  Writes the nnz sorted keys. */
void orc_sorted_keys(int d, const int64_t *dims, int64_t nnz, const int64_t *coo_idx, uint64_t *keys)
{
    for (int64_t e = 0; e < nnz; ++e) keys[e] = orc_linear_key(d, dims, coo_idx + e * d);
    qsort(keys, (size_t)nnz, sizeof(uint64_t), cmp_u64);
}

/* Sorts (key, value) pairs by key: the value lookup of uniform sampling
   over a sparse tensor.  vals NULL means all ones. */
typedef struct { uint64_t key; double val; } orc_pair;

static int cmp_pair(const void *a, const void *b)
{
    uint64_t x = ((const orc_pair *)a)->key, y = ((const orc_pair *)b)->key;
    return x < y ? -1 : (x > y ? 1 : 0);
}

void orc_sorted_pairs(int d, const int64_t *dims, int64_t nnz, const int64_t *coo_idx, const double *vals,
                      uint64_t *keys_out, double *vals_out)
{
    orc_pair *p = (orc_pair *)malloc((size_t)nnz * sizeof(orc_pair));
    for (int64_t e = 0; e < nnz; ++e) {
        p[e].key = orc_linear_key(d, dims, coo_idx + e * d);
        p[e].val = vals ? vals[e] : 1.0;
    }
    qsort(p, (size_t)nnz, sizeof(orc_pair), cmp_pair);
    for (int64_t e = 0; e < nnz; ++e) {
        keys_out[e] = p[e].key;
        vals_out[e] = p[e].val;
    }
    free(p);
}

/* x at a linear key of a sparse tensor: its value, or 0 when not a nonzero. */
double orc_sparse_value(int64_t nnz, const uint64_t *sorted_keys, const double *sorted_vals, uint64_t key)
{
    int64_t lo = 0, hi = nnz;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (sorted_keys[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < nnz && sorted_keys[lo] == key) ? sorted_vals[lo] : 0.0;
}

int orc_is_nonzero(int64_t nnz, const uint64_t *sorted_keys, uint64_t key)
{
    int64_t lo = 0, hi = nnz; /* search [lo, hi) */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (sorted_keys[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo < nnz && sorted_keys[lo] == key;
}

/* ------------------------------------------------------------------------ */
/* Sampling: Algs. 1-3, producing the explicit list of drawn entries with   */
/* their value x, weight w and class.  Nonzero draws come first (positions  */
/* 0..p-1), then zero draws.                                                */
/*                                                                          */
/* Stratified zeros (Alg. 2, with the oversampling of Section 4.2 and App.  */
/* B): candidates c = 0, 1, 2, ... are drawn with the zero-candidate tag;   */
/* a candidate is rejected when it is a nonzero; the first q accepted in    */
/* candidate order are kept.  Candidates are examined in batches of          */
/* ceil(rho * q * omega / zeta); after 64 batches without q acceptances the */
/* call fails with ORC_ERR_SHORTFALL.                                       */
/* ------------------------------------------------------------------------ */

int64_t orc_sample_count(int kind, int64_t p, int64_t q)
{
    return (kind == ORC_UNIFORM || kind == ORC_OBSERVED) ? q : p + q;
}

/* Number of entries of nonzero weight (the observed entries of weighted GCP
   for missing data, Section 4.4). */
int64_t orc_count_observed(int64_t n, const double *weights)
{
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i)
        if (weights[i] != 0.0) c++;
    return c;
}

int orc_sample(int d, const int64_t *dims, int sparse,
               const double *dense_vals, const double *dense_weights,
               int64_t nnz, const int64_t *coo_idx, const double *coo_vals,
               const uint64_t *sorted_keys, const double *sorted_vals,
               int kind, int64_t p, int64_t q,
               uint64_t seed, uint64_t problem, uint64_t stream, double rho,
               int64_t *idx_out, double *x_out, double *w_out, int8_t *cls_out,
               int64_t *candidates_used)
{
    if (d < 1 || d > ORC_MAX_D || q < 0 || p < 0) return ORC_ERR_ARG;
    double omega = 1.0;
    for (int k = 0; k < d; ++k) omega *= (double)dims[k];
    if (candidates_used) *candidates_used = 0;

    if (kind == ORC_UNIFORM) {
        /* Alg. 1: s = q draws, weight omega / s; a sparse tensor's value is
           looked up among its nonzeros.  With entry weights v (Eq. (4.5),
           dense tensors) the draw's weight is (omega / s) v_i. */
        for (int64_t j = 0; j < q; ++j) {
            int64_t *ix = idx_out + j * d;
            orc_draw_multi_index(d, dims, seed, problem, stream, ORC_TAG_UNIFORM, (uint64_t)j, ix);
            uint64_t key = orc_linear_key(d, dims, ix);
            if (sparse) {
                x_out[j] = orc_sparse_value(nnz, sorted_keys, sorted_vals, key);
                w_out[j] = omega / (double)q;
            } else {
                x_out[j] = dense_vals[key];
                w_out[j] = (omega / (double)q) * (dense_weights ? dense_weights[key] : 1.0);
            }
            cls_out[j] = ORC_CLS_UNIFORM;
        }
        return ORC_OK;
    }

    if (kind == ORC_OBSERVED) {
        /* Section 4.4: with missing entries given weight 0, sample only the
           entries of nonzero weight.  Reading taken: uniform draws over the
           observed set Omega_obs by rejection, candidates c = 0, 1, ... from
           their own stream, the first q accepted in candidate order (in
           batches of ceil(rho q omega / |Omega_obs|), at most 64), each with
           weight (|Omega_obs| / q) v_i: unbiased for the weighted objective,
           as entries of weight 0 contribute nothing to it. */
        if (sparse || !dense_weights) return ORC_ERR_ARG;
        int64_t n_all = 1;
        for (int k = 0; k < d; ++k) n_all *= dims[k];
        double observed = (double)orc_count_observed(n_all, dense_weights);
        if (q > 0 && observed <= 0) return ORC_ERR_ARG;
        if (rho <= 0) rho = 1.1;
        int64_t batch = q > 0 ? (int64_t)ceil(rho * (double)q * omega / observed) : 0;
        int64_t cap = 64 * batch;
        int64_t accepted = 0, c = 0;
        int64_t ix[ORC_MAX_D];
        while (accepted < q) {
            if (c >= cap) {
                if (candidates_used) *candidates_used = c;
                return ORC_ERR_SHORTFALL;
            }
            orc_draw_multi_index(d, dims, seed, problem, stream, ORC_TAG_OBSERVED, (uint64_t)c, ix);
            c++;
            uint64_t key = orc_linear_key(d, dims, ix);
            if (dense_weights[key] == 0.0) continue; /* missing: reject */
            for (int k = 0; k < d; ++k) idx_out[accepted * d + k] = ix[k];
            x_out[accepted] = dense_vals[key];
            w_out[accepted] = (observed / (double)q) * dense_weights[key];
            cls_out[accepted] = ORC_CLS_UNIFORM;
            accepted++;
        }
        if (candidates_used) *candidates_used = c;
        return ORC_OK;
    }

    if (!sparse || nnz <= 0) return ORC_ERR_ARG;
    double eta = (double)nnz;

    /* nonzeros: xi = randi(eta), weight eta / p (Algs. 2 and 3) */
    for (int64_t j = 0; j < p; ++j) {
        int64_t xi = orc_draw_nonzero(nnz, seed, problem, stream, (uint64_t)j);
        for (int k = 0; k < d; ++k) idx_out[j * d + k] = coo_idx[xi * d + k];
        x_out[j] = coo_vals ? coo_vals[xi] : 1.0;
        w_out[j] = eta / (double)p;
        cls_out[j] = kind == ORC_STRATIFIED ? ORC_CLS_STRAT_NZ : ORC_CLS_SEMI_NZ;
    }

    if (kind == ORC_SEMI_STRATIFIED) {
        /* Alg. 3: q "zeros" drawn from all of Omega, no rejection, weight omega / q */
        for (int64_t j = 0; j < q; ++j) {
            int64_t *ix = idx_out + (p + j) * d;
            orc_draw_multi_index(d, dims, seed, problem, stream, ORC_TAG_SEMI_ZERO, (uint64_t)j, ix);
            x_out[p + j] = 0.0;
            w_out[p + j] = omega / (double)q;
            cls_out[p + j] = ORC_CLS_SEMI_ZERO;
        }
        return ORC_OK;
    }

    if (kind != ORC_STRATIFIED) return ORC_ERR_ARG;
    /* Alg. 2: rejection sampling of zeros, weight zeta / q */
    double zeta = omega - eta;
    if (q > 0 && zeta <= 0) return ORC_ERR_ARG;
    if (rho <= 0) rho = 1.1;
    int64_t batch = q > 0 ? (int64_t)ceil(rho * (double)q * omega / zeta) : 0;
    int64_t cap = 64 * batch;
    int64_t accepted = 0, c = 0;
    int64_t ix[ORC_MAX_D];
    while (accepted < q) {
        if (c >= cap) {
            if (candidates_used) *candidates_used = c;
            return ORC_ERR_SHORTFALL;
        }
        orc_draw_multi_index(d, dims, seed, problem, stream, ORC_TAG_ZERO_CANDIDATE, (uint64_t)c, ix);
        c++;
        if (orc_is_nonzero(nnz, sorted_keys, orc_linear_key(d, dims, ix))) continue; /* reject */
        int64_t pos = p + accepted;
        for (int k = 0; k < d; ++k) idx_out[pos * d + k] = ix[k];
        x_out[pos] = 0.0;
        w_out[pos] = zeta / (double)q;
        cls_out[pos] = ORC_CLS_STRAT_ZERO;
        accepted++;
    }
    if (candidates_used) *candidates_used = c;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Elementwise y of a drawn entry (Eq. (4.1) with the sampling weights of   */
/* Sections 4.1-4.3 and the weights of Eq. (4.5) folded into w):            */
/*   semi-stratified nonzero: y = w [g(x,m) - g(0,m)]   (Alg. 3)            */
/*   every other class:       y = w g(x,m)              (x = 0 for zeros)   */
/* ------------------------------------------------------------------------ */

double orc_entry_y(int loss, int cls, double x, double m, double w)
{
    if (cls == ORC_CLS_SEMI_NZ) return w * (orc_loss_g(loss, x, m) - orc_loss_g(loss, 0.0, m));
    return w * orc_loss_g(loss, x, m);
}

/* The loss-estimate term of a drawn entry (Eqs. (5.1)-(5.2); the semi-     */
/* stratified form is this library's reading, built like Alg. 3's gradient). */
double orc_entry_f(int loss, int cls, double x, double m, double w)
{
    if (cls == ORC_CLS_SEMI_NZ) return w * (orc_loss_f(loss, x, m) - orc_loss_f(loss, 0.0, m));
    return w * orc_loss_f(loss, x, m);
}

/* ------------------------------------------------------------------------ */
/* Sampled gradient (Eq. (4.3), the sparse MTTKRP that closes Alg. 1):      */
/* for each drawn entry, G_k(i_k,:) += y * prod_{l != k} A_l(i_l,:).         */
/* G is written (zeroed first), same layout as A.                           */
/* ------------------------------------------------------------------------ */

int orc_grad_from_samples(int d, const int64_t *dims, int rank, const double *A, int loss,
                          int64_t n, const int64_t *idx, const double *x, const double *w,
                          const int8_t *cls, double *G)
{
    if (d < 1 || d > ORC_MAX_D || rank < 1) return ORC_ERR_ARG;
    int64_t off[ORC_MAX_D];
    mode_offsets(d, dims, rank, off);
    int64_t total = off[d - 1] + dims[d - 1] * rank;
    memset(G, 0, (size_t)total * sizeof(double));
    for (int64_t e = 0; e < n; ++e) {
        const int64_t *ix = idx + e * d;
        double m = orc_model_value(d, dims, rank, A, ix);
        double y = orc_entry_y(loss, cls[e], x[e], m, w[e]);
        for (int k = 0; k < d; ++k) {
            for (int j = 0; j < rank; ++j) {
                double prod = 1.0;
                for (int l = 0; l < d; ++l)
                    if (l != k) prod *= A[off[l] + ix[l] * rank + j];
                G[off[k] + ix[k] * rank + j] += y * prod;
            }
        }
    }
    return ORC_OK;
}

/* Fixed-sample loss estimate F-hat (Eqs. (5.1)-(5.2)). */
double orc_loss_from_samples(int d, const int64_t *dims, int rank, const double *A, int loss,
                             int64_t n, const int64_t *idx, const double *x, const double *w,
                             const int8_t *cls)
{
    double F = 0.0;
    for (int64_t e = 0; e < n; ++e) {
        double m = orc_model_value(d, dims, rank, A, idx + e * d);
        F += orc_entry_f(loss, cls[e], x[e], m, w[e]);
    }
    return F;
}

/* Sum of |term| over the same list: the scale that bounds the rounding     */
/* error of any summation order of F-hat's terms (used for tolerances).     */
double orc_loss_abs_from_samples(int d, const int64_t *dims, int rank, const double *A, int loss,
                                 int64_t n, const int64_t *idx, const double *x, const double *w,
                                 const int8_t *cls)
{
    double S = 0.0;
    for (int64_t e = 0; e < n; ++e) {
        double m = orc_model_value(d, dims, rank, A, idx + e * d);
        S += fabs(orc_entry_f(loss, cls[e], x[e], m, w[e]));
    }
    return S;
}

/* Per-entry sum of |contribution| to the sampled gradient: for every drawn  */
/* entry, Gabs_k(i_k,:) += |y * prod_{l != k} A_l(i_l,:)|.  The scale that  */
/* bounds the rounding error of any summation order of G's terms.           */
int orc_grad_abs_from_samples(int d, const int64_t *dims, int rank, const double *A, int loss,
                              int64_t n, const int64_t *idx, const double *x, const double *w,
                              const int8_t *cls, double *Gabs)
{
    if (d < 1 || d > ORC_MAX_D || rank < 1) return ORC_ERR_ARG;
    int64_t off[ORC_MAX_D];
    mode_offsets(d, dims, rank, off);
    int64_t total = off[d - 1] + dims[d - 1] * rank;
    memset(Gabs, 0, (size_t)total * sizeof(double));
    for (int64_t e = 0; e < n; ++e) {
        const int64_t *ix = idx + e * d;
        double m = orc_model_value(d, dims, rank, A, ix);
        double y = orc_entry_y(loss, cls[e], x[e], m, w[e]);
        for (int k = 0; k < d; ++k)
            for (int j = 0; j < rank; ++j) {
                double prod = 1.0;
                for (int l = 0; l < d; ++l)
                    if (l != k) prod *= A[off[l] + ix[l] * rank + j];
                Gabs[off[k] + ix[k] * rank + j] += fabs(y * prod);
            }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Full (non-stochastic) gradient and objective over all of Omega of a     */
/* dense tensor: G_k = Y_(k) Z_k with y_i = v_i g(x_i, m_i) (Eqs. (4.1),    */
/* (4.2) and the weighted form (4.5); v = NULL means all weights 1).        */
/* Enumerates every index; for tiny tensors only.                           */
/* ------------------------------------------------------------------------ */

int orc_full_grad(int d, const int64_t *dims, int rank, const double *A, int loss,
                  const double *X, const double *v, double *G, double *F_out)
{
    if (d < 1 || d > ORC_MAX_D) return ORC_ERR_ARG;
    int64_t off[ORC_MAX_D];
    mode_offsets(d, dims, rank, off);
    int64_t total = off[d - 1] + dims[d - 1] * rank;
    memset(G, 0, (size_t)total * sizeof(double));
    int64_t omega = 1;
    for (int k = 0; k < d; ++k) omega *= dims[k];
    int64_t ix[ORC_MAX_D];
    double F = 0.0;
    for (int64_t lin = 0; lin < omega; ++lin) {
        int64_t rem = lin;
        for (int k = d - 1; k >= 0; --k) { ix[k] = rem % dims[k]; rem /= dims[k]; }
        double m = orc_model_value(d, dims, rank, A, ix);
        double wt = v ? v[lin] : 1.0;
        F += wt * orc_loss_f(loss, X[lin], m);
        double y = wt * orc_loss_g(loss, X[lin], m);
        for (int k = 0; k < d; ++k)
            for (int j = 0; j < rank; ++j) {
                double prod = 1.0;
                for (int l = 0; l < d; ++l)
                    if (l != k) prod *= A[off[l] + ix[l] * rank + j];
                G[off[k] + ix[k] * rank + j] += y * prod;
            }
    }
    if (F_out) *F_out = F;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* One Adam step with projection (Alg. 4, inner loop over modes), on all    */
/* n entries of the concatenated factor matrices:                          */
/*   B = b1 B + (1-b1) G;  C = b2 C + (1-b2) G^2;                           */
/*   Bh = B / (1 - b1^t');  Ch = C / (1 - b2^t');                          */
/*   A = A - alpha Bh / sqrt(Ch + eps)   (eps inside the root, as printed; */
/*        eps_inside_sqrt = 0 gives sqrt(Ch) + eps instead);               */
/*   A = max(A, lower).                                                     */
/* t' = t + 1 where t counts the steps already taken: the bias correction  */
/* of the first step uses power 1 (the printed counter starts at 0 and      */
/* would divide by 1 - b^0 = 0).                                            */
/* ------------------------------------------------------------------------ */

void orc_adam_step(int64_t n, double *A, double *B, double *C, const double *G,
                   double alpha, double beta1, double beta2, double eps, double lower,
                   int64_t t, int eps_inside_sqrt)
{
    double c1 = 1.0 - pow(beta1, (double)(t + 1));
    double c2 = 1.0 - pow(beta2, (double)(t + 1));
    for (int64_t e = 0; e < n; ++e) {
        B[e] = beta1 * B[e] + (1.0 - beta1) * G[e];
        C[e] = beta2 * C[e] + (1.0 - beta2) * G[e] * G[e];
        double bh = B[e] / c1;
        double ch = C[e] / c2;
        double den = eps_inside_sqrt ? sqrt(ch + eps) : sqrt(ch) + eps;
        A[e] = A[e] - alpha * bh / den;
        if (A[e] < lower) A[e] = lower;
    }
}
