// Tensor-core (tcgen05) path of the block step. Not built yet: the mixed
// precision is rejected at init with a clear error.
#include "gmf_internal.cuh"

int gmf_tc_prepare(gmf_model* h, cudaStream_t st) {
    (void)h;
    (void)st;
    return GMF_ERR_ARG;
}
int gmf_tc_sweep(gmf_model* h, int w, long long t0, cudaStream_t st) {
    (void)h; (void)w; (void)t0; (void)st;
    return GMF_ERR_STATE;
}
void gmf_tc_free(gmf_model* h) { (void)h; }
