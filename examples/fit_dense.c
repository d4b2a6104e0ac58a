#include <math.h>
#include "gcp.h"

/* GCP-Adam iterations on a dense 3-way tensor: dX holds n[0] n[1] n[2] floats;
   A, G, B, C hold n[k] x ld floats per mode (ld = rank rounded up to 4; G, B, C
   zeroed); state is 64 bytes.  Returns the device status word. */
int fit(const float *dX, const int64_t n[3], int32_t rank, float *A[3], float *G[3], float *B[3],
        float *C[3], gcp_adam_state *state, gcp_stream_t stream, int iterations)
{
    gcp_tensor X = {0};
    X.d = 3;
    for (int k = 0; k < 3; ++k) X.dims[k] = n[k];
    X.vals = dX;
    gcp_handle *h;
    if (gcp_create(&h, &X, stream) != GCP_OK) return -1;
    gcp_factors F = {0};
    F.rank = rank;
    F.ld = (rank + 3) / 4 * 4;
    for (int k = 0; k < 3; ++k) F.A[k] = A[k];
    gcp_sampling S = {0};
    S.kind = GCP_SAMPLER_UNIFORM;
    S.q = 1000;  /* draws per iteration */
    S.seed = 1;
    gcp_adam_params prm = {0.9f, 0.999f, 1e-8f, -INFINITY, 1, 0};
    gcp_state_init(state, 1e-3f, stream);
    for (int t = 0; t < iterations; ++t) {
        S.stream = (uint64_t)t;  /* a new sample set every iteration */
        if (gcp_iteration(h, &F, GCP_LOSS_GAUSSIAN, &S, NULL, G, B, C, &prm, state, stream) != GCP_OK) break;
    }
    int32_t status = 0;
    gcp_get_device_status(h, &status);
    gcp_destroy(h);
    return status;
}
