// The update launch of a sweep: one CTA per 32-row slice of every row strip and
// column strip of the sweep's blocks (eq. 12, eq. 14), and the once-per-sweep
// NB shape update (App. B) in block 0. It waits for the sweep's tile launch to
// complete (griddepcontrol.wait) before it reads the tiles' partials and moment
// sums; the slice state it loads before that wait is not written by the tile
// launch.
#include <algorithm>

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

// The update launch of the tensor-core path (column-major partial slots). Two
// instances: blocks of up to 384 threads (q + d and p + d up to 24) capped at
// 40 registers, so four CTAs share an SM and a sweep's units run as one wave
// (480 units of 384 threads on 152 SMs for 5 blocks of 2048 x 1024; the
// register cap costs a few spilled values, measured faster than 2 or 3 CTAs
// per SM), and any width up to 1024 threads.
template <int NTMAX, int MINB>
__global__ void __launch_bounds__(NTMAX, MINB) update_tc_kernel(StepArgs a, int w, int T) {
    __shared__ int s_cnt[UTC_SR];
    grid_launch_dependents();
    update_unit_tc(a, w, T, blockIdx.x, s_cnt);  // waits for the tile launch inside
    if (blockIdx.x == 0 && threadIdx.x == 0) nb_shape_update(a, w);
}

// Several models sharing the partitions (rank sweep): blockIdx.y = model.
template <int NTMAX, int MINB>
__global__ void __launch_bounds__(NTMAX, MINB) update_tc_multi(const StepArgs* __restrict__ av, int w, int T) {
    __shared__ StepArgs s_a;
    __shared__ int s_cnt[UTC_SR];
    grid_launch_dependents();
    if (threadIdx.x == 0) s_a = av[blockIdx.y];
    __syncthreads();
    // every thread takes part (the block may be wider than this model needs: the extra threads own no row)
    update_unit_tc(s_a, w, T, blockIdx.x, s_cnt);
    if (blockIdx.x == 0 && threadIdx.x == 0) nb_shape_update(s_a, w);
}

// Copy the state of `rows` consecutive rows starting at `first` of one side
// (row side: L, GbR, HbR, cntR; column side: R, GbC, HbC, cntC) to (write = 0)
// or from (write = 1) a packed buffer, row by row: [KP factor values | nf
// smoothed gradients | nf smoothed curvatures | visit count (int32 bits)].
__global__ void chunk_state_kernel(float* P, float* Gb, float* Hb, int* cnt, int KP, int nf, int64_t first, int rows,
                                   float* buf, int write) {
    const int W = KP + 2 * nf + 1;
    const int64_t total = (int64_t)rows * W;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / W;
        const int c = (int)(e - i * W);
        const int64_t g = first + i;
        float* v;
        if (c < KP)
            v = P + g * KP + c;
        else if (c < KP + nf)
            v = Gb + g * nf + (c - KP);
        else if (c < KP + 2 * nf)
            v = Hb + g * nf + (c - KP - nf);
        else
            v = (float*)(cnt + g);
        if (write)
            *v = buf[e];
        else
            buf[e] = *v;
    }
}

}  // namespace

cudaError_t gmf_launch_chunk_state(float* P, float* Gb, float* Hb, int* cnt, int KP, int nf, int64_t first, int rows,
                                   float* buf, int write, cudaStream_t st) {
    const int64_t total = (int64_t)rows * (KP + 2 * nf + 1);
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
    if (blocks == 0) return cudaSuccess;
    chunk_state_kernel<<<blocks, 256, 0, st>>>(P, Gb, Hb, cnt, KP, nf, first, rows, buf, write);
    return cudaGetLastError();
}

constexpr int UTC_NARROW = 384;  // widest block of the four-per-SM instances

cudaError_t gmf_launch_update_tc(const StepArgs& a, int w, int T, cudaStream_t st) {
    const int threads = UTC_SR * utc_groups(a.fr, a.fc);
    const dim3 grid((unsigned)utc_units(a.nk, a.TI, a.TJ, T));
    if (threads <= UTC_NARROW)
        return gmf_launch_pdl(update_tc_kernel<UTC_NARROW, 4>, grid, dim3((unsigned)threads), 0, st, a, w, T);
    return gmf_launch_pdl(update_tc_kernel<1024, 1>, grid, dim3((unsigned)threads), 0, st, a, w, T);
}

cudaError_t gmf_launch_update_tc_multi(const StepArgs* d_args, int nmodels, int units, int threads, int w, int T,
                                       cudaStream_t st) {
    const dim3 grid((unsigned)units, (unsigned)nmodels);
    if (threads <= UTC_NARROW)
        return gmf_launch_pdl(update_tc_multi<UTC_NARROW, 4>, grid, dim3((unsigned)threads), 0, st, d_args, w, T);
    return gmf_launch_pdl(update_tc_multi<1024, 1>, grid, dim3((unsigned)threads), 0, st, d_args, w, T);
}

int gmf_update_tc_threads(const StepArgs& a) { return UTC_SR * utc_groups(a.fr, a.fc); }
int gmf_update_tc_units(const StepArgs& a, int T) { return utc_units(a.nk, a.TI, a.TJ, T); }

int gmf_update_units(const StepArgs& a, int T) { return update_units(a.nk, a.TI, a.TJ, T); }

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
