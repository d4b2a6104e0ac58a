/*
 * gcp.h -- C ABI of libgcp_gb300.so, the GB300 (sm_103a) sampled-gradient
 * path of generalized CP decomposition fitted by Adam (GCP-SGD / GCP-Adam,
 * Kolda & Hong, "Stochastic Gradients for Large-Scale Tensor Decomposition",
 * arXiv:1906.01687).
 *
 * Conventions for every entry point:
 *  - Pointers named "device" are CUDA device pointers owned by the caller; the
 *    library never frees them.  Pointers named "host" are host memory.
 *  - Indices are 0-based.  Dense tensors are row-major (last mode fastest).
 *    A linear key is the row-major linear index of a multi-index.
 *  - Arguments are validated on the host before anything is launched; a bad
 *    argument returns GCP_ERR_INVALID_ARG and launches nothing.
 *  - Work is enqueued on the given stream and returns without waiting
 *    (stream-ordered, asynchronous), except where a function says otherwise.
 *    Errors found by a kernel (a stratified shortfall, a non-finite value)
 *    are recorded in a sticky device status word read by
 *    gcp_get_device_status().
 *  - Random draws come from Philox4x64-10 (Salmon, Moraes, Dror and Shaw,
 *    SC'11) with key (seed, problem) and counter (j, stream, tag, k / 4);
 *    mode k of draw j takes word k % 4 of that block and becomes
 *    randi(n_k) = floor(word * n_k / 2^64).  Tags: 0 uniform draw, 1 nonzero
 *    draw (word 0 gives xi = randi(nnz)), 2 stratified zero candidate,
 *    3 semi-stratified "zero", 4 observed-entry candidate.  The sample set
 *    is therefore a pure function of (seed, problem, stream) and the tensor.
 */
#ifndef GCP_GB300_H
#define GCP_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *gcp_stream_t; /* a cudaStream_t; NULL = legacy default stream */

#define GCP_MAX_MODES 8
/* Philox stream word of a fixed loss-estimate sample set (Section 5.1: one
   set serves every epoch and every run). */
#define GCP_STREAM_EST 0xFFFFFFFFFFFFFFFFull

typedef enum gcp_status {
    GCP_OK = 0,
    GCP_ERR_INVALID_ARG = 1,      /* rejected on the host, nothing launched */
    GCP_ERR_CUDA = 2,             /* a CUDA runtime call failed */
    GCP_ERR_NO_MEMORY = 3,        /* a library-owned allocation failed */
    GCP_ERR_SAMPLE_SHORTFALL = 4, /* stratified zeros: fewer than q accepted */
    GCP_ERR_TIMEOUT = 5,          /* a bounded device-side wait gave up: the stratified zero
                                     pass's look-back over earlier tiles (device status of
                                     the handle) or a fused batched iteration's wait for a
                                     problem's gradient (that problem's state->status);
                                     neither can run out while the kernel's own blocks run */
    GCP_ERR_NONFINITE = 6,        /* a non-finite loss estimate was seen */
    GCP_ERR_UNSUPPORTED = 7       /* valid but not supported (e.g. prod(dims) >= 2^64 for stratified) */
} gcp_status;

/* Elementwise losses f(x, m) and g = df/dm.  Gaussian is Section 1's
   (x - m)^2; Bernoulli-logit log(1 + e^m) - x m and Poisson-log e^m - x m are
   the log-link losses of the GCP paper this one builds on (HoKoDu20).  The
   paper's own odds / identity-link losses (Section 1; Sections 5.2-5.4) need
   m > 0 and are evaluated at m + 1e-10: Bernoulli-odds log(m + 1) - x log m,
   Poisson-identity m - x log m, Gamma x / m + log m, and the beta-divergence
   with beta = 1/2 as Section 5.3 prints it, 2 m^(1/2) + 2 x m^(-1/2).  Use
   them with nonnegative factors (lower = 0 in the Adam step). */
typedef enum gcp_loss {
    GCP_LOSS_GAUSSIAN = 0,
    GCP_LOSS_BERNOULLI_LOGIT = 1,
    GCP_LOSS_POISSON_LOG = 2,
    GCP_LOSS_BERNOULLI_ODDS = 3,
    GCP_LOSS_POISSON_IDENTITY = 4,
    GCP_LOSS_GAMMA = 5,
    GCP_LOSS_BETA_HALF = 6
} gcp_loss;

/* Samplers: Alg. 1 (uniform, Section 4.1), Alg. 2 (stratified, Section 4.2),
   Alg. 3 (semi-stratified, Section 4.3), and uniform draws over the entries
   of nonzero weight (Section 4.4: missing data as weight 0, avoided when
   sampling; dense tensors with weights): candidates from their own stream,
   the first q of nonzero weight kept in candidate order (batches of
   ceil(rho q omega / |Omega_obs|), at most 64), weight (|Omega_obs| / q) v_i. */
typedef enum gcp_sampler {
    GCP_SAMPLER_UNIFORM = 0,
    GCP_SAMPLER_STRATIFIED = 1,
    GCP_SAMPLER_SEMI_STRATIFIED = 2,
    GCP_SAMPLER_OBSERVED = 3
} gcp_sampler;

/* Class of a drawn entry; it selects the form of y_i and of the F-hat term:
   semi-stratified nonzeros use w [g(x,m) - g(0,m)] and w [f(x,m) - f(0,m)],
   every other class w g(x,m) and w f(x,m) (x = 0 for zeros). */
typedef enum gcp_class {
    GCP_CLS_UNIFORM = 0,    /* Alg. 1, w = omega / s            */
    GCP_CLS_STRAT_NZ = 1,   /* Alg. 2 nonzero, w = eta / p      */
    GCP_CLS_STRAT_ZERO = 2, /* Alg. 2 zero, w = zeta / q        */
    GCP_CLS_SEMI_NZ = 3,    /* Alg. 3 nonzero, w = eta / p      */
    GCP_CLS_SEMI_ZERO = 4   /* Alg. 3 "zero", w = omega / q     */
} gcp_class;

/* The data tensor X (Section 3.2).
   dense  (sparse = 0): vals = prod(dims) FP32 values, row-major, device.
   sparse (sparse = 1): coordinate format; idx[k][e] = i_k of nonzero e
                        (int32, device, in [0, n_k): not checked on the
                        device), vals = nnz FP32 values or NULL for an
                        all-ones (binary) tensor.  Positions must be unique
                        for the stratified sampler's rejection test. */
typedef struct gcp_tensor {
    int32_t d;                        /* modes, 2..8 (one mode has no leave-one-out
                                         product in Eq. (4.3): rejected) */
    int32_t sparse;
    int64_t dims[GCP_MAX_MODES];      /* n_k, each in [1, 2^31) */
    int64_t nnz;                      /* sparse only */
    const float *vals;
    const int32_t *idx[GCP_MAX_MODES];
    const float *weights;             /* dense only: entry weights v of weighted GCP (Eq. (4.5)),
                                         prod(dims) FP32, row-major, device; NULL = all ones.
                                         A weight of 0 marks a missing entry. */
} gcp_tensor;

/* Factor matrices A_k of the CP model (Eq. (1.1)).  Mode k is an n_k x ld
   row-major FP32 matrix A[k] (device); ld is a multiple of 4 with
   ld >= rank and columns rank..ld-1 hold zeros.  With bf16 = 1 the gradient
   and the loss estimate gather rows from the BF16 copies A_bf16[k]
   (raw bfloat16 bits, same n_k x ld layout), while A stays the FP32 master
   that gcp_adam_step updates and re-rounds into A_bf16 whenever A_bf16[k]
   is non-NULL. */
typedef struct gcp_factors {
    int32_t rank;                     /* r, 1..256 */
    int32_t ld;
    int32_t bf16;
    int32_t reserved;
    float *A[GCP_MAX_MODES];
    uint16_t *A_bf16[GCP_MAX_MODES];
} gcp_factors;

/* What to draw (Sections 4.1-4.4).  uniform: s = q draws (p ignored);
   stratified / semi-stratified: p nonzero draws then q zero draws;
   observed: s = q draws over the entries of nonzero weight (p must be 0).
   oversample is Section 4.2's rho (<= 0 selects 1.1): stratified zeros are
   examined in batches of ceil(rho q omega / zeta) candidates (observed
   entries in batches of ceil(rho q omega / |Omega_obs|)) and the first q
   accepted in candidate order are kept; after 64 batches the draw stops
   with GCP_ERR_SAMPLE_SHORTFALL in the device status. */
typedef struct gcp_sampling {
    int32_t kind;     /* gcp_sampler */
    int32_t reserved;
    int64_t p;        /* 0 .. 2^40 */
    int64_t q;        /* 0 .. 2^40 */
    uint64_t seed;
    uint64_t problem; /* second key word: separates independent runs */
    uint64_t stream;  /* counter word: the iteration, or GCP_STREAM_EST */
    double oversample;
} gcp_sampling;

/* An explicit list of drawn entries, struct of arrays, device memory owned
   by the caller: idx[k][e] (int32), x[e], w[e] (FP32), cls[e] (gcp_class).
   A caller-made list must hold 0 <= idx[k][e] < n_k and a valid class: the
   kernels read the factor rows at these indices without checking them (the
   library's own lists hold them by construction). */
typedef struct gcp_samples {
    int64_t n;
    int32_t *idx[GCP_MAX_MODES];
    float *x;
    float *w;
    int8_t *cls;
} gcp_samples;

/* Adam hyper-parameters (Alg. 4; defaults of Section 5.1: alpha 0.01,
   beta1 0.9, beta2 0.999, eps 1e-8).  eps_inside_sqrt = 1 divides by
   sqrt(Ch + eps) as Alg. 4 prints it, 0 by sqrt(Ch) + eps.  lower is the
   projection bound l (-INFINITY for none). */
typedef struct gcp_adam_params {
    float beta1;
    float beta2;
    float eps;
    float lower;
    int32_t eps_inside_sqrt;
    int32_t reserved;
} gcp_adam_params;

/* Epoch control of Alg. 4: tau iterations per epoch, learning-rate decay nu
   after a failed epoch, stop after more than kappa failed epochs. */
typedef struct gcp_epoch_params {
    int64_t tau;
    float nu;
    int32_t kappa;
} gcp_epoch_params;

/* Optimizer state, resident in DEVICE memory (64 bytes, 8-byte aligned,
   caller-owned), so that whole epochs can be replayed from a CUDA graph
   without host involvement.  Fields are read and written by kernels. */
typedef struct gcp_adam_state {
    double F;        /* current loss estimate F-hat */
    double F_old;    /* F-hat at the start of the epoch */
    int64_t t;       /* Adam steps taken; step t+1's bias correction uses power t+1 */
    int64_t iter;    /* iterations ever run: the Philox stream word of the draws (never wound back) */
    float alpha;     /* current learning rate */
    int32_t bad;     /* failed epochs so far (c in Alg. 4) */
    int32_t done;    /* 1 once more than kappa epochs failed: Adam steps become no-ops */
    int32_t status;  /* sticky gcp_status of the optimizer kernels */
    uint32_t ticket; /* internal completion counter; 0 between launches */
    uint32_t reserved[3];
} gcp_adam_state;

typedef struct gcp_handle gcp_handle; /* opaque: a prepared tensor */

/* ------------------------------------------------------------------------ */
/* Handles                                                                  */
/* ------------------------------------------------------------------------ */

/* Prepares X for sampling (Section 3.2 storage; Section 4.2 lookup).
   Copies the descriptor (the caller keeps X's device arrays alive and
   unchanged for the handle's lifetime) and, for a sparse X, builds in
   library-owned device memory a packed nonzero record per entry (indices and
   value in one 16-, 32- or 48-byte record, so that a nonzero draw reads one
   aligned segment).  The nonzero-key hash table of the stratified sampler is
   built on first stratified use.  Allocates with cudaMalloc and waits for
   the stream; call it before any stream capture.
   Errors: GCP_ERR_INVALID_ARG (d outside 2..8, a dimension outside
   [1, 2^31), nnz < 1 for sparse, NULL arrays), GCP_ERR_NO_MEMORY,
   GCP_ERR_CUDA. */
gcp_status gcp_create(gcp_handle **out, const gcp_tensor *X, gcp_stream_t stream);

/* Takes up new contents of X's device arrays after the caller has rewritten
   them in place (same d, dims, nnz and pointers; Section 3.2 storage): for a
   sparse X it re-packs the nonzero records and, if the stratified
   sampler's nonzero-key hash was built, rebuilds it in place; for a dense X
   with entry weights, the count of entries of nonzero weight is taken
   again on the observed sampler's next use (a host read, as on first use).
   Stream-ordered, allocates nothing and waits for nothing (graph-capturable
   for a sparse X).  The first gradient launch after it draws after its
   dependency wait even with early_draws.  Errors: GCP_ERR_INVALID_ARG (NULL
   handle), GCP_ERR_CUDA. */
gcp_status gcp_refresh(gcp_handle *h, gcp_stream_t stream);

/* Frees the handle and all device memory it owns (waits for the whole
   device first, so no launch of the handle is still running); h must not be
   used afterwards.  Errors: GCP_ERR_INVALID_ARG (NULL handle). */
gcp_status gcp_destroy(gcp_handle *h);

/* Reads and clears the handle's sticky device status word (a gcp_status:
   the first error a kernel of the handle recorded since the last read, or
   GCP_OK).  Synchronises the device.  host_out: host, one int32_t.
   Errors: GCP_ERR_INVALID_ARG (NULL handle or host_out), GCP_ERR_CUDA (a
   failed launch or copy; *host_out is then not written). */
gcp_status gcp_get_device_status(gcp_handle *h, int32_t *host_out);

/* Number of entries a sampling spec draws: q for uniform and observed,
   p + q for stratified and semi-stratified.  Returns -1 for an invalid
   spec. */
int64_t gcp_sample_count(const gcp_sampling *S);

/* ------------------------------------------------------------------------ */
/* Sampling: Algs. 1-3                                                      */
/* ------------------------------------------------------------------------ */

/* Materialises the drawn entries of Alg. 1 (uniform over a dense X),
   Alg. 2 (stratified: p nonzeros with xi = randi(nnz), then q zeros by
   rejection against the nonzero keys), Alg. 3 (semi-stratified: p
   nonzeros, then q indices from all of Omega without rejection) or the
   observed-entry draw of Section 4.4 (q uniform draws over the entries of
   nonzero weight, by rejection of the rest) into out, nonzero draws first.
   Each entry gets its value x (0 for zeros), its weight w (omega/s, eta/p,
   zeta/q, omega/q or (|Omega_obs|/q) v_i, computed in FP64 and rounded
   once) and its class.  out->n must equal gcp_sample_count(S).
   stratified needs a sparse X with prod(dims) < 2^64 (else
   GCP_ERR_UNSUPPORTED); uniform over a sparse X looks each drawn index up
   among the nonzeros (value or 0; also prod(dims) < 2^64); uniform over a
   dense X with entry weights gives the draw weight (omega/s) v_i; observed
   needs a dense X with weights and p = 0 (else GCP_ERR_INVALID_ARG).  May
   allocate library scratch on the first stratified or observed call
   (cudaMalloc), and the first observed call reads the count of entries of
   nonzero weight back to the host: make that first call (or gcp_reserve)
   before any stream capture.  A shortfall sets GCP_ERR_SAMPLE_SHORTFALL in
   the device status; the unfilled slots then hold weight 0.
   Errors: GCP_ERR_INVALID_ARG (a NULL handle, a bad spec or list, out->n
   other than gcp_sample_count(S)), GCP_ERR_UNSUPPORTED, GCP_ERR_NO_MEMORY,
   GCP_ERR_CUDA. */
gcp_status gcp_sample(gcp_handle *h, const gcp_sampling *S, const gcp_samples *out,
                      gcp_stream_t stream);

/* Performs every library-owned allocation and host read that gcp_sample and
   gcp_grad would make for this spec (the stratified sampler's nonzero-key
   hash, the tile words of its ordered compaction and the zero list; for the
   observed-entry sampler the count of entries of nonzero weight, read back
   to the host once), so that
   later calls with the same or a smaller spec allocate nothing, wait for
   nothing and can be captured in a CUDA graph.  Waits for the stream.
   Errors: as gcp_sample; GCP_ERR_INVALID_ARG when no entry has a nonzero
   weight. */
gcp_status gcp_reserve(gcp_handle *h, const gcp_sampling *S, gcp_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Sampled gradient: Eq. (4.3) via Algs. 1-3                               */
/* ------------------------------------------------------------------------ */

/* Accumulates the stochastic gradient G~_k = Y~_(k) Z_k (Eq. (4.3)) into
   G[k] (device, FP32, n_k x F->ld, row-major; the caller zeroes G before a
   fresh gradient -- gcp_adam_step leaves it zeroed).  For every drawn entry
   i: m_i = sum_j prod_k A_k(i_k, j) (Eq. (1.1)); y_i = w g(x_i, m_i), or
   w [g(x_i, m_i) - g(0, m_i)] for a semi-stratified nonzero; and for every
   k, G_k(i_k, j) += y_i * prod_{l != k} A_l(i_l, j) for the columns
   j < rank (the padding columns of G are not written).
   Exactly one of S and list is non-NULL:
     S    -- draws generated inside the kernel from the spec (fused
             sampling, nothing materialised; stratified zeros are picked
             inside the kernel too -- tiles of candidates, ordered by
             decoupled look-back through library scratch -- or, with
             gcp_tuning.zero_pass = 1 or 5 to 8 modes, listed first by a
             separate pass);
     list -- a materialised list (gcp_sample output or the caller's own).
   stream_dev (device, nullable): if non-NULL the Philox stream word is read
   from *stream_dev on the device at run time instead of S->stream (used by
   graph-replayed epochs with &state->iter).
   Modes whose rows are hit often accumulate first in library-owned replica
   slabs that a second kernel (or, with gcp_tuning.tail_work = 1, the
   gradient kernel's last blocks) folds into G and re-zeroes; the slabs are
   allocated on the first call that needs them (cudaMalloc: make that call
   before any stream capture) and are shared by every call on this handle,
   so calls on one handle must not overlap on the GPU.
   Errors: GCP_ERR_INVALID_ARG (a bad loss, spec, list or factor layout, a
   misaligned G), GCP_ERR_NO_MEMORY (replica slabs, scratch), GCP_ERR_CUDA;
   kernel-side shortfall as in gcp_sample. */
gcp_status gcp_grad(gcp_handle *h, const gcp_factors *F, gcp_loss loss,
                    const gcp_sampling *S, const gcp_samples *list,
                    const int64_t *stream_dev, float *const G[GCP_MAX_MODES],
                    gcp_stream_t stream);

/* The part of gcp_grad's sampled gradient (Eq. (4.3), Algs. 1-3) that comes
   from the draws j in [first, first + count) of spec S, accumulated into G
   as gcp_grad does.  Draws are numbered as gcp_sample lists them: uniform
   and observed 0..q-1; stratified and semi-stratified the p nonzero draws
   0..p-1, then the q zero draws p..p+q-1.  Because every draw is a pure
   function of its number (counter-based sampling), the results over any
   partition of [0, gcp_sample_count(S)) sum to gcp_grad's G (up to the
   FP32 summation order): this is the sample-parallel split of one problem
   across GPUs, each GPU taking one range and a sum of G across GPUs
   following -- the parallel use of sampling that Section 6 points to.  With
   a stratified spec each call examines every candidate tile (the zeros of
   a range depend on every earlier candidate) and walks only its range; a
   range of nonzero draws only (first + count <= p) makes no zeros.
   stream_dev, replica slabs, allocation and overlap rules as for gcp_grad.
   Errors: GCP_ERR_INVALID_ARG (S NULL, first < 0, count < 0, or
   first + count beyond gcp_sample_count(S)) and as gcp_grad. */
gcp_status gcp_grad_range(gcp_handle *h, const gcp_factors *F, gcp_loss loss, const gcp_sampling *S,
                          int64_t first, int64_t count, const int64_t *stream_dev,
                          float *const G[GCP_MAX_MODES], gcp_stream_t stream);

/* The full (non-stochastic) gradient G_k = Y_(k) Z_k of a dense X
   (Eq. (4.2); with entry weights, Eq. (4.5)): every index of Omega taken once
   with weight 1 (or v_i) through the gradient kernel, accumulated into G as
   gcp_grad does.  O(r prod(dims)) work: for moderate tensors.
   Errors: GCP_ERR_INVALID_ARG (a sparse X, a bad loss or layout) and as
   gcp_grad. */
gcp_status gcp_full_grad(gcp_handle *h, const gcp_factors *F, gcp_loss loss, float *const G[GCP_MAX_MODES],
                         gcp_stream_t stream);

/* The exact objective F(X, M) of Eq. (1.2) (weighted: Eq. (4.5)) of a dense X
   over every index, FP32 terms summed in FP64, into *out_dev (one device
   double, 8-byte aligned).  Errors: GCP_ERR_INVALID_ARG (a sparse X, a bad
   loss, layout or out_dev), GCP_ERR_NO_MEMORY, GCP_ERR_CUDA. */
gcp_status gcp_full_loss(gcp_handle *h, const gcp_factors *F, gcp_loss loss, double *out_dev, gcp_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Loss estimate: Eqs. (5.1)-(5.2)                                          */
/* ------------------------------------------------------------------------ */

/* F-hat = sum over the fixed list of w f(x, m) (w [f(x,m) - f(0,m)] for
   semi-stratified nonzeros), each term in FP32, summed in FP64 in a fixed
   order (deterministic for a given list), written to *out_dev (device,
   one double, 8-byte aligned).  Uses library scratch for the per-block
   partial sums (allocated on the first call: make it before any stream
   capture).  Errors: GCP_ERR_INVALID_ARG (a bad loss, list, layout or
   out_dev), GCP_ERR_NO_MEMORY, GCP_ERR_CUDA. */
gcp_status gcp_loss_est(gcp_handle *h, const gcp_factors *F, gcp_loss loss,
                        const gcp_samples *list, double *out_dev, gcp_stream_t stream);

/* The loss estimate of gcp_loss_est for callers that cannot allocate device
   memory at the time of the call: it needs no handle and allocates nothing.
   This entry point has no counterpart in the paper.  It exists for callers
   that must not call cudaMalloc when they run the estimate: hosts whose
   device memory is owned by another allocator (a framework's caching
   allocator that has reserved the GPU's memory) and loops that forbid
   allocation after start-up, where a cudaMalloc would stall or fail.  Its
   per-block partial sums live in a file-scope device array of the library:
   1024 doubles and a counter (about 8 KB), held by every GPU that loads the
   library until the process exits.
   d: modes, 2..8; F, list: as for gcp_loss_est (device arrays,
   caller-owned); at most 262,144 listed entries (one per thread of at most
   1024 blocks of 256), longer lists return GCP_ERR_INVALID_ARG.  out_dev:
   one device double.  The first call on a device does a one-time set-up:
   with that device current it looks up the array's device address
   (cudaGetSymbolAddress).  Every call clears the array's counter on the stream before its kernel.
   Every call shares the array: calls whose kernels overlap on the GPU
   (other streams, other threads) race and give wrong results.  Same
   arithmetic as gcp_loss_est (FP32 terms, FP64 sums); the block count may
   differ, so the last bits may too.  Errors: GCP_ERR_INVALID_ARG (d outside
   2..8, a bad loss, factor set or list, a list that is too long, out_dev
   NULL or not 8-byte aligned), GCP_ERR_CUDA (the set-up or the launch). */
gcp_status gcp_loss_est_noalloc(int32_t d, const gcp_factors *F, gcp_loss loss, const gcp_samples *list,
                                double *out_dev, gcp_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Adam with projection and the epoch logic of Alg. 4                       */
/* ------------------------------------------------------------------------ */

/* Sets *state (device, one gcp_adam_state, 8-byte aligned) to the start of
   a run of Alg. 4: F = F_old = 0, t = iter = 0, the given step size alpha,
   bad = done = status = ticket = 0.  Errors: GCP_ERR_INVALID_ARG (state NULL
   or misaligned), GCP_ERR_CUDA. */
gcp_status gcp_state_init(gcp_adam_state *state, float alpha, gcp_stream_t stream);

/* One Adam step for every mode (Alg. 4, inner loop): with t = state->t,
   B = b1 B + (1-b1) G; C = b2 C + (1-b2) G^2; Bh = B / (1 - b1^(t+1));
   Ch = C / (1 - b2^(t+1)); A = max(A - alpha Bh / sqrt(Ch + eps), lower)
   (or sqrt(Ch) + eps); then G = 0, the BF16 copy (where non-NULL) is
   re-rounded from A, and state->t, state->iter advance by one.  alpha is
   read from state.  B, C, G: device FP32 with A's layout.  Does nothing
   but zero G once state->done is set.  dims: host, d entries.  Factor sets
   of 2^31 or more float4 chunks (sum of n_k * ld / 4; 32 GB) are rejected
   with GCP_ERR_INVALID_ARG.  Errors: GCP_ERR_INVALID_ARG (d outside 1..8, a
   bad rank or ld, a NULL or misaligned factor, G, B, C or state, beta1 or
   beta2 outside [0, 1), eps < 0, the size above), GCP_ERR_CUDA. */
gcp_status gcp_adam_step(const gcp_factors *F, int32_t d, const int64_t *dims,
                         float *const G[GCP_MAX_MODES], float *const B[GCP_MAX_MODES],
                         float *const C[GCP_MAX_MODES], const gcp_adam_params *prm,
                         gcp_adam_state *state, gcp_stream_t stream);

/* One GCP-Adam iteration (Alg. 4, inner loop body): the sampled gradient of
   gcp_grad for spec S (with stream_dev as there) followed by the Adam step
   of gcp_adam_step, fused so that replica slabs of the gradient are folded
   inside the Adam kernel (two kernel launches per iteration; a stratified
   spec's zeros are made inside the gradient kernel, or by a third launch
   with gcp_tuning.zero_pass = 1; with tail_work = 1 a small factor set's
   Adam step is taken by the gradient kernel's last blocks and the iteration
   is one launch).  G must be zero on entry and
   is left zero; B, C, state as for gcp_adam_step.  Same results as
   gcp_grad followed by gcp_adam_step up to the summation order.  Between
   the two kernels state->t has already advanced (the gradient kernel does
   it, so that the Adam kernel's blocks need not wait for one another); on
   return both t and iter have advanced by one, as with gcp_adam_step.
   Errors: as gcp_grad and gcp_adam_step, checked before either kernel is
   launched. */
gcp_status gcp_iteration(gcp_handle *h, const gcp_factors *F, gcp_loss loss, const gcp_sampling *S,
                         const int64_t *stream_dev, float *const G[GCP_MAX_MODES], float *const B[GCP_MAX_MODES],
                         float *const C[GCP_MAX_MODES], const gcp_adam_params *prm, gcp_adam_state *state,
                         gcp_stream_t stream);

/* Saves the epoch-start copy of {A, B, C} into {SA, SB, SC} (same layouts)
   and sets F_old = F (the "save copies" step that opens each epoch of
   Alg. 4).  Call once after the first loss estimate.  Errors:
   GCP_ERR_INVALID_ARG (a bad layout, NULL or misaligned arrays or state),
   GCP_ERR_CUDA. */
gcp_status gcp_epoch_begin(const gcp_factors *F, int32_t d, const int64_t *dims,
                           float *const B[GCP_MAX_MODES], float *const C[GCP_MAX_MODES],
                           float *const SA[GCP_MAX_MODES], float *const SB[GCP_MAX_MODES],
                           float *const SC[GCP_MAX_MODES], gcp_adam_state *state,
                           gcp_stream_t stream);

/* Closes an epoch (Alg. 4, after EstObj): if state->F > state->F_old or F
   is not finite, restores {A, B, C} (and the BF16 copy) from {SA, SB, SC},
   sets F = F_old, t -= tau, alpha *= nu, bad += 1, done = (bad > kappa);
   otherwise accepts, copying {A, B, C} into {SA, SB, SC} and setting
   F_old = F for the next epoch.  An equal estimate is accepted.  All on the
   device; graph-capturable.  A non-finite F also records GCP_ERR_NONFINITE
   in state->status.  Errors: as gcp_epoch_begin, and a NULL ep, tau < 0 or
   kappa < 0. */
gcp_status gcp_epoch_end(const gcp_factors *F, int32_t d, const int64_t *dims,
                         float *const B[GCP_MAX_MODES], float *const C[GCP_MAX_MODES],
                         float *const SA[GCP_MAX_MODES], float *const SB[GCP_MAX_MODES],
                         float *const SC[GCP_MAX_MODES], const gcp_epoch_params *ep,
                         gcp_adam_state *state, gcp_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Batched form: many independent decompositions (multi-start runs, uneven  */
/* shapes, ranks and losses) advanced together, one kernel launch per step  */
/* for all of them.  Alg. 4 run per problem; no data crosses problems.      */
/* ------------------------------------------------------------------------ */

/* One problem of a batch.  X dense (uniform sampling, Alg. 1) with 2 <= d <= 4;
   F as for gcp_grad (bf16 allowed); S a uniform spec whose q draws are taken
   per iteration and whose seed and problem words key the Philox draws (the
   stream word is read from state->iter on the device); est the problem's
   fixed loss-estimate list; G, B, C, SA, SB, SC the gradient, moments and
   epoch snapshots with F's layout (G zero on entry); state its optimizer
   state.  All device memory is caller-owned and must outlive the batch. */
typedef struct gcp_batch_problem {
    gcp_tensor X;
    gcp_factors F;
    int32_t loss;
    int32_t reserved;
    gcp_sampling S;
    gcp_samples est;
    float *G[GCP_MAX_MODES];
    float *B[GCP_MAX_MODES];
    float *C[GCP_MAX_MODES];
    float *SA[GCP_MAX_MODES];
    float *SB[GCP_MAX_MODES];
    float *SC[GCP_MAX_MODES];
    gcp_adam_params adam;
    gcp_epoch_params epoch;
    gcp_adam_state *state;
} gcp_batch_problem;

typedef struct gcp_batch gcp_batch; /* opaque: the device-side problem table */

/* Validates count problems (host array) and uploads their table to device
   memory owned by the batch (cudaMalloc; waits for the stream).  Errors:
   GCP_ERR_INVALID_ARG for any invalid problem (sparse X, d outside 2..4,
   entry weights, a non-uniform spec, misaligned pointers) or count outside
   1..1024, GCP_ERR_NO_MEMORY. */
gcp_status gcp_batch_create(gcp_batch **out, const gcp_batch_problem *problems, int32_t count, gcp_stream_t stream);

/* Frees the batch and its device memory (waits for the whole device first;
   the problems' caller-owned memory is not touched).  Errors:
   GCP_ERR_INVALID_ARG (NULL batch). */
gcp_status gcp_batch_destroy(gcp_batch *b);

/* Launch shape of the batched gradient: threads per block (multiple of 32,
   <= 256; 0 = 256) and blocks (0 = one resident wave).  Host-side only.
   Errors: GCP_ERR_INVALID_ARG (NULL batch, values out of range). */
gcp_status gcp_batch_set_tuning(gcp_batch *b, int32_t block, int32_t grid_blocks);

/* Shape of the batched gradient for every problem: chunks_per_lane (1..8;
   0 = 1) float4 chunks of a factor row per lane, so a rank-r problem takes
   L = the power of two (at most 32) covering ceil(ceil(r / 4) / chunks_per_lane)
   lanes per draw and 32 / L draws per warp step (the rows per warp);
   replica_target (0 = 64) and max_replicas (0 = 32; 1 = none): a mode whose
   rows receive more than replica_target updates per iteration on average
   spreads them over ceil(updates / replica_target) replica slabs, at most
   max_replicas (the pre-reduction width before the Adam step's fold).
   Re-uploads the problem table and reallocates the replica slabs
   (cudaMalloc; waits for the stream): call it before any stream capture.
   Changes only the summation order of the gradients.  Errors:
   GCP_ERR_INVALID_ARG (values out of range), GCP_ERR_NO_MEMORY,
   GCP_ERR_CUDA. */
gcp_status gcp_batch_set_shape(gcp_batch *b, int32_t chunks_per_lane, int32_t replica_target, int32_t max_replicas,
                               gcp_stream_t stream);

/* The shape problem `problem` runs with: lanes per draw, chunks per lane and
   the replica slabs of each mode (host outputs; replicas holds 4 entries,
   0 beyond the problem's modes).  Errors: GCP_ERR_INVALID_ARG (NULL batch
   or output, problem outside 0..count-1). */
gcp_status gcp_batch_get_shape(gcp_batch *b, int32_t problem, int32_t *lanes, int32_t *chunks, int32_t *replicas);

/* The sampled gradients of every problem (Eq. (4.3), Alg. 1) into G: warps
   take 32 consecutive draws of one problem at a time from a table of all
   problems' draws; a mode whose rows receive many updates adds them into
   replica slabs, folded into G by a second launch.  Errors:
   GCP_ERR_INVALID_ARG (NULL batch), GCP_ERR_CUDA. */
gcp_status gcp_batch_grad(gcp_batch *b, gcp_stream_t stream);

/* The Adam step of every problem (as gcp_adam_step), one launch.  It also
   folds (and clears) the replica slabs into which gcp_batch_iteration's
   gradient kernel spreads the updates of heavily hit rows; after a plain
   gcp_batch_grad those slabs are already folded and zero.  Errors:
   GCP_ERR_INVALID_ARG (NULL batch), GCP_ERR_CUDA. */
gcp_status gcp_batch_adam_step(gcp_batch *b, gcp_stream_t stream);

/* One GCP-Adam iteration of every problem (Alg. 4, inner loop body):
   gcp_batch_grad then gcp_batch_adam_step.  Errors: as those two. */
gcp_status gcp_batch_iteration(gcp_batch *b, gcp_stream_t stream);

/* gcp_batch_iteration in one persistent launch: warps take every problem's
   gradient batches and then every problem's Adam chunks from one queue, in
   that order; a warp holding an Adam chunk of a problem waits until all of
   that problem's gradient batches are done (they were taken earlier by warps
   that never wait, so the wait ends; it is bounded all the same, and a wait
   that runs out records GCP_ERR_TIMEOUT in that problem's state->status and
   skips the chunk).  The problem's last Adam chunk advances its t and iter.
   Same results as gcp_batch_iteration up to the summation order (the
   replica slabs are folded in order).  Uses library-owned counters that
   every launch leaves zero: launches on one batch must not overlap on the
   GPU.  Errors: GCP_ERR_INVALID_ARG (NULL batch), GCP_ERR_CUDA. */
gcp_status gcp_batch_iteration_fused(gcp_batch *b, gcp_stream_t stream);

/* Every problem's F-hat (Eq. (5.1)) on its fixed list into its state->F
   (FP64), one launch.  Errors: GCP_ERR_INVALID_ARG (NULL batch),
   GCP_ERR_CUDA. */
gcp_status gcp_batch_loss_est(gcp_batch *b, gcp_stream_t stream);

/* gcp_epoch_begin / gcp_epoch_end (Alg. 4, outer loop) for every problem,
   one launch each.  Errors: GCP_ERR_INVALID_ARG (NULL batch),
   GCP_ERR_CUDA. */
gcp_status gcp_batch_epoch_begin(gcp_batch *b, gcp_stream_t stream);
gcp_status gcp_batch_epoch_end(gcp_batch *b, gcp_stream_t stream);

/* Rounds A[k] into A_bf16[k] (round to nearest even) for every mode:
   A_bf16[k] is device BF16 with A[k]'s n_k x ld row-major layout.  dims:
   host, d entries.  Errors: GCP_ERR_INVALID_ARG (the factor checks of
   gcp_adam_step, or a NULL A_bf16[k]), GCP_ERR_CUDA. */
gcp_status gcp_factors_to_bf16(const gcp_factors *F, int32_t d, const int64_t *dims,
                               gcp_stream_t stream);

/* Launch shape of gcp_grad for one handle (0 / -1 fields mean "choose
   automatically").  lanes x chunks float4 column chunks cover a row:
   lanes in {1,2,4,8,16,32} lanes per draw, chunks in {1,2,3,4} per lane
   (only compiled pairs are accepted); block threads (multiple of 32, <= 256);
   grid_blocks CTAs (0 = one resident wave, capped by the draws).
   Accumulation of the row updates, per mode:
     smem_bytes    shared-memory budget for per-CTA accumulation of small
                   G_k, flushed once per CTA (-1 or 0 = off);
     smem_min_hits least expected draws per row per CTA for that (x10);
     max_replicas  most replica slabs a mode's updates are spread over to
                   keep same-address contention low (-1 = 32; 0 or 1 = off);
     replica_target expected updates per 16-byte address per launch above
                   which a mode is replicated (0 = 64).
   group_draws = 1: each group of lanes generates and takes its own draw
   (32 / lanes draws per warp step) instead of a warp generating 32 draws and
   its groups walking them in turn (0): more warps for small draw counts.
   prefetch = 1 (one chunk per lane, 2 or 4 lanes, at most 4 modes): a group
   issues the row loads of all its draws before consuming any (one round
   trip to L2 per group walk instead of one per draw; more registers).
   prefetch = 2 (one chunk per lane, 1 to 8 lanes, 3 or 4 modes, group_draws
   = 0): the staged walk -- every lane copies its chunk of every row of its
   group's draws into shared memory (cp.async) and the group walks them from
   there (one round trip per batch, no registers held; block / 32 x lanes x
   modes x 32 x 16 bytes of shared memory, 8 with BF16 rows; shared-memory
   accumulation of G is off with it).
   early_draws = 1: where the draws read nothing but the data tensor (uniform
   sampling, semi-stratified sampling, the nonzero draws of stratified
   sampling, or uniform over a sparse tensor whose nonzero table was built by
   an earlier call), the kernel makes each warp's first batch of draws
   (Philox, value gather) before it waits for the kernel launched just
   before it on the stream (programmatic dependent launch), so that work
   overlaps the previous kernel's tail.  Contract: the
   data tensor's values and weights are not written by the kernel launched
   immediately before the call (copies and anything further back are
   ordered as usual).  With stream_dev, the kernel starts from a prediction
   (the previous such launch's stream + 1), checks it against *stream_dev
   after the wait and redoes the batch when it differs, so the draws are
   always those of *stream_dev.  Default 0 (wait first).
   zero_pass (stratified and observed-entry sampling, Alg. 2 and Section
   4.4): 0 (automatic) makes the zeros inside the gradient launch where the
   walk is the group walk of 3 or 4 modes -- the grid's first blocks each
   take a tile of block-size consecutive candidates, rank the accepted ones,
   learn the count accepted before their tile by decoupled look-back (bounded
   waits, GCP_ERR_TIMEOUT) and walk the kept ones as draws, with no list
   written; 1 runs the separate ordered pass that lists the zeros first.
   warp_combine (group walk, 3 or 4 modes): modes of at most this many rows
   sum the updates that the groups of one warp step make to the same 16
   bytes of G_k (a match on the row and column chunk, then shuffles) before
   one lane issues the L2 reduction (0 = off).
   tail_work: 1 lets the last blocks of the gradient kernel to finish take
   gcp_grad's replica fold and, where the factor set is small, gcp_iteration's
   Adam step (at most 64 blocks; they wait, bounded, for the other blocks,
   then GCP_ERR_TIMEOUT) instead of launches of their own; 0 (default)
   launches the fold and Adam kernels.
   A tuning choice changes the summation order only, never the draws. */
typedef struct gcp_tuning {
    int32_t lanes;
    int32_t chunks;
    int32_t block;
    int32_t grid_blocks;
    int32_t smem_bytes;
    int32_t smem_min_hits;
    int32_t max_replicas;
    int32_t replica_target;
    int32_t group_draws;
    int32_t prefetch;
    int32_t early_draws;
    int32_t zero_pass;
    int32_t warp_combine;
    int32_t tail_work;
} gcp_tuning;

/* The launch shape gcp_grad chose (gcp_get_launch). */
typedef struct gcp_launch_info {
    int32_t lanes;
    int32_t chunks;
    int32_t block;
    int32_t grid_blocks;
    int32_t smem_bytes;
    uint32_t smem_mode_mask;
    int32_t replicas[GCP_MAX_MODES];
    int32_t group_draws;
    int32_t prefetch;
    int32_t early_draws;
    int32_t zero_tiles;  /* 1: stratified zeros are made inside the gradient launch */
    uint32_t combine_mode_mask;  /* bit k: mode k's updates are combined within a warp step */
    int32_t adam_tail_blocks;    /* gcp_iteration: blocks of the gradient kernel that take the Adam
                                    step (0: a separate Adam launch) */
} gcp_launch_info;

/* Sets (t != NULL) or resets to automatic (t == NULL) the handle's launch
   shape.  Errors: GCP_ERR_INVALID_ARG for a shape that is not compiled. */
gcp_status gcp_set_tuning(gcp_handle *h, const gcp_tuning *t);

/* Reports the launch shape gcp_grad would use for these factors and draw
   count (after automatic choices).  out: host.  Launches nothing.
   Errors: GCP_ERR_INVALID_ARG (NULL handle or out, n_draws < 0, a bad
   rank or ld, a NULL or misaligned factor, a tuned shape that is not
   compiled for this tensor's modes). */
gcp_status gcp_get_launch(gcp_handle *h, const gcp_factors *F, int64_t n_draws, gcp_launch_info *out);

/* Kernel timing for benchmarks.  With enable = 1 the handle creates
   2 x capacity pairs of CUDA events (at most 65536; allocation, so call it
   outside stream capture) and records one pair on the launching stream
   around every fused-gradient kernel launch that follows (gcp_grad,
   gcp_iteration; set 0) and around every Adam kernel launch of
   gcp_iteration (set 1; none when the gradient kernel took the step, see
   gcp_tuning.tail_work), until the pairs are used up; enable = 0 destroys
   them.  gcp_profile_read synchronises the events of set `which` and returns
   the summed device time of its recorded launches in milliseconds and their
   count, then starts a new count.  host outputs.  gcp_profile synchronises
   the device.  Errors: GCP_ERR_INVALID_ARG (NULL handle or output, capacity
   outside 1..65536 with enable = 1, which not 0 or 1), GCP_ERR_NO_MEMORY
   (the host arrays of events), GCP_ERR_CUDA. */
gcp_status gcp_profile(gcp_handle *h, int32_t enable, int32_t capacity);
gcp_status gcp_profile_read(gcp_handle *h, int32_t which, double *total_ms, int64_t *launches);

/* A static string naming a status code ("unknown status" for a value that
   is none); never NULL. */
const char *gcp_status_string(gcp_status s);

/* The CUDA runtime error behind the calling thread's most recent
   GCP_ERR_CUDA or GCP_ERR_NO_MEMORY from any entry point: its numeric code
   (a cudaError_t; 0 when no call of this thread has failed on a CUDA error)
   and the runtime's name for it (a static string).  For diagnostics; the
   status codes stay the interface. */
int32_t gcp_last_cuda_error(void);
const char *gcp_last_cuda_error_name(void);

/* Library version string (static; never NULL). */
const char *gcp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GCP_GB300_H */
