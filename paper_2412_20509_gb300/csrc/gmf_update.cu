// The update launch of a sweep: one CTA per 32-row slice of every row strip and
// column strip of the sweep's blocks (eq. 12, eq. 14), and the once-per-sweep
// NB shape update (App. B) in block 0. It waits for the sweep's tile launch to
// complete (griddepcontrol.wait) before it reads the tiles' partials and moment
// sums; the slice state it loads before that wait is not written by the tile
// launch.
#include "gmf_internal.cuh"
#include "gmf_update.cuh"

using namespace gmfdev;

namespace {

__global__ void __launch_bounds__(UPD_NT) update_kernel(StepArgs a, int w, int T) {
    extern __shared__ __align__(16) float stage[];
    grid_launch_dependents();
    update_unit(a, w, T, blockIdx.x, stage);  // waits for the tile launch inside
    if (blockIdx.x == 0 && threadIdx.x == 0) nb_shape_update(a, w);
}

// Several models sharing the partitions (rank sweep): blockIdx.y = model.
__global__ void __launch_bounds__(UPD_NT) update_multi(const StepArgs* __restrict__ av, int w, int T) {
    extern __shared__ __align__(16) float stage[];
    __shared__ StepArgs s_a;
    grid_launch_dependents();
    if (threadIdx.x == 0) s_a = av[blockIdx.y];
    __syncthreads();
    update_unit(s_a, w, T, blockIdx.x, stage);  // waits for the tile launch inside
    if (blockIdx.x == 0 && threadIdx.x == 0) nb_shape_update(s_a, w);
}

}  // namespace

int gmf_update_units(const StepArgs& a, int T) { return update_units(a.per, a.TI, a.TJ, T); }

size_t gmf_update_smem(const StepArgs& a) { return sizeof(float) * (size_t)update_stage_floats(a.KP, a.fr, a.fc); }

cudaError_t gmf_launch_update(const StepArgs& a, int w, int T, cudaStream_t st) {
    return gmf_launch_pdl(update_kernel, dim3((unsigned)gmf_update_units(a, T)), dim3(UPD_NT), gmf_update_smem(a), st,
                          a, w, T);
}

cudaError_t gmf_launch_update_multi(const StepArgs* d_args, int nmodels, int units, size_t smem, int w, int T,
                                    cudaStream_t st) {
    return gmf_launch_pdl(update_multi, dim3((unsigned)units, (unsigned)nmodels), dim3(UPD_NT), smem, st, d_args, w,
                          T);
}
