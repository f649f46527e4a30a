// Algorithm 2 (identifiability projection). Not built yet.
#include <string>
#include "gmf_internal.cuh"

int gmf_orth_run(gmf_model* h, int mode, cudaStream_t st, std::string* err) {
    (void)h; (void)mode; (void)st;
    *err = "not available in this build";
    return GMF_ERR_STATE;
}
