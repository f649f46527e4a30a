// Per-cell Fisher scoring. Not built yet.
#include <string>
#include "gmf_internal.cuh"

int gmf_project_run(gmf_model* h, const void* Ynew, int y16, int64_t n_new, const float* Xnew, const float* off,
                    const float* Ustart, int n_steps, float* Uout, float* Gout, float* dev, cudaStream_t st,
                    std::string* err) {
    (void)h; (void)Ynew; (void)y16; (void)n_new; (void)Xnew; (void)off; (void)Ustart; (void)n_steps;
    (void)Uout; (void)Gout; (void)dev; (void)st;
    *err = "not available in this build";
    return GMF_ERR_STATE;
}
