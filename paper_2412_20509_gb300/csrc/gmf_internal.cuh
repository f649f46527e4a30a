// Internal declarations of the GB300 GMF library (not part of the C ABI).
//
// Storage (all device, all owned by the handle):
//   Yp  n x m counts, rows and columns permuted by the fixed partitions, so
//       block (I_a, J_b) is the contiguous sub-matrix rows [a*nb_row, ...),
//       columns [b*nb_col, ...).
//   L   n x KP  augmented row factors  [o | X | Gamma | U]   (K = 1+p+q+d, KP = K
//               rounded up to a multiple of 4, the padding columns zero)
//   R   m x KP  augmented column factors [1 | B | Z | V], so eta = L R'.
//       Row-free columns (Gamma, U) of L and their multipliers (Z, V) in R
//       share the indices [1+p, K); column-free columns (B, V) of R and their
//       multipliers (X, U) in L share {1..p} u [1+p+q, K).
//   GbR/HbR n x (q+d), GbC/HbC m x (p+d): smoothed derivatives (eq. 12).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "gmf.h"

#define GMF_TILE 64          // SIMT tile edge (rows and columns)
#define GMF_THREADS 256      // threads per SIMT tile CTA
#define GMF_KMAX 64          // largest K = 1+p+q+d the SIMT path accepts
#define GMF_FREE_MAX 64      // largest q+d or p+d

// Error bits written by kernels into the handle's device status word.
#define GMF_DEVERR_NONFINITE 1u
#define GMF_DEVERR_TIMEOUT 2u
#define GMF_DEVERR_BOUNDS 4u

struct StepArgs {
    int64_t n, m;
    int p, q, d, K, fr, fc;
    int KP;                     // row stride of L and R (K rounded up to a multiple of 4)
    int nb_row, nb_col, r, s, per, swap;
    int TI, TJ;                 // tiles per block along rows / columns (largest block)
    int family, bias_corr, alpha_mode;
    int missing;                // 1: a count equal to ymiss is not observed (imputed by mu, Sec. 3.2)
    float ymiss;                // the missing-count marker as a float: -1 (int32), 65535 (uint16)
    float lam[4];
    float a1, a2, damping, eps, clamp;
    const void* Y;              // Yp (permuted)
    int y16;                    // 1 if uint16 counts
    int yf32;                   // 1 if float32 responses (NaN marks a missing one)
    const float* W;             // permuted weights or nullptr
    float* L;
    float* R;
    float* GbR;
    float* HbR;
    float* GbC;
    float* HbC;
    int* cntR;
    int* cntC;
    float* alpha;               // device scalar (NB shape)
    const float* alpha_col;     // [m] per-gene NB shapes, permuted (alpha_mode 2), else nullptr
    float* partR;               // [per][TI][TJ][TILE][2*fr]: row partials of tile (ti, tj)
    float* partC;               // [per][TJ][TI][TILE][2*fc]: column partials of tile (ti, tj)
    double* nbpart;             // [per*TI*TJ][2]: NB moment sums of each tile
    unsigned* nbctr;            // [1]: tiles of the sweep done (cluster mode's NB shape update)
    const int* sigma;           // device copy of the epoch's sweep offsets
    const float* rhoc;          // [nsw][per]: rho_t * c_t per block (rho_t alone when bias_corr = 1)
    const float* rho1;          // [nsw]: rho at the first block of each sweep (NB shape update)
    const int* need;            // [nsw][per]: earlier visits of each block's moving strip (persistent epochs)
    unsigned* strip_done;       // [max(r, s)]: CTAs done with each moving strip in this launch (persistent epochs)
    unsigned* err;              // device status word
    unsigned long long wait_ns; // limit of one strip wait of the persistent epoch (global timer)
    const int* kmap;            // [nk]: the blocks of the sweep that this launch runs (nullptr: all, k = 0..per-1)
    int nk;                     // blocks this launch runs (grid z of the tile launch)
};

// Block index of launch slot z (a subset of the sweep's blocks, or all of them).
__host__ __device__ __forceinline__ int block_of_slot(const StepArgs& a, int z) { return a.kmap ? a.kmap[z] : z; }

struct gmf_model {
    gmf_config cfg;
    int device;
    int p, q, d, K, fr, fc;
    int KP;                     // row stride of L and R: 16-byte aligned rows
    int64_t n, m;
    int r, s, nsw, per, swap;
    int TI, TJ;
    int y16;
    int yf32;                   // float32 responses (GMF_Y_FLOAT32)
    // device storage
    void* Yp;
    float* Wp;
    float* L;
    float* R;
    float* GbR;
    float* HbR;
    float* GbC;
    float* HbC;
    int* cntR;
    int* cntC;
    float* alpha;
    float* alpha_col;           // [m] per-gene NB shapes, permuted order (alpha_mode 2)
    int* rperm;
    int* cperm;
    void* ystage;               // staging for counts uploaded from the host
    void* ystage2;              // second staging buffer (gmf_update_y_async)
    cudaStream_t copy_stream;   // host-to-device copies of gmf_update_y_async
    cudaEvent_t up_copied[2];   // staging buffer i filled
    cudaEvent_t up_free[2];     // staging buffer i read by its permutation
    int up_idx;                 // staging buffer of the next gmf_update_y_async
    int up_init;
    // counts read straight from mapped host memory into a second count buffer (gmf_update_y_async)
    void* ybuf[2];              // the two count buffers (ybuf[1] allocated on first use); Yp = ybuf[ycur]
    int ycur;
    int y_fixed;                // other handles read Yp: it never moves
    cudaEvent_t y_free[2];      // last work that read ybuf[i] (recorded when it stops being current)
    cudaEvent_t y_ready;        // the gather into the new current buffer
    float* Rorig;               // m x KP: R in the caller's gene order (per-cell projection)
    void* kr_buf;               // BF16 Khatri-Rao product of [Z, V] (tensor-core projection)
    size_t kr_elems;
    int y_shared;               // Yp / Wp belong to another handle (rank sweep)
    float* partR;
    float* partC;
    double* nbpart;
    unsigned* nbctr;
    int* sigma;
    float* rhoc;
    float* rho1;
    int* need;
    int* kmap;                  // [per]: blocks of a gmf_sgd_sweep_blocks launch
    unsigned* strip_done;
    unsigned* err;
    double* devpart;
    double* devtot;
    int devparts;
    // host mirrors
    int32_t* h_rperm;
    int32_t* h_cperm;
    int64_t t;                  // blocks processed so far
    int64_t wait_ns;            // strip-wait limit of the persistent epoch (gmf_set_wait_limit; 0: 2 s)
    int32_t need_extra;         // added to every dependency count of a persistent range (gmf_set_wait_limit)
    int32_t flow_lag;           // dataflow epoch: tile groups between a block's tiles and its updates (gmf_set_flow_lag)
    void* tc;                   // tensor-core path state (gmf_step_tc.cu), or nullptr
    // kernel timing (gmf_trace)
    int trace_on;
    int trace_used;
    cudaEvent_t* trace_ev;      // GMF_TRACE_POOL pairs
    double trace_ms;
    int64_t trace_launches;
    // CUDA graph of one full epoch of FP32 sweeps (captured on first use)
    cudaGraphExec_t epoch_graph[2];   // one per count buffer
    cudaStream_t capture_stream;
};

#define GMF_TRACE_POOL 512

// Launch with programmatic stream serialization: the kernel may start before
// the preceding kernel in the stream has finished and waits for it with
// griddepcontrol.wait before it touches state that kernel writes.
template <typename... Params, typename... Args>
cudaError_t gmf_launch_pdl(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                           Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Raise `kernel`'s dynamic shared-memory limit to what the device allows, after
// checking that `need` bytes fit (cudaErrorInvalidValue if not). The limit
// belongs to the function, not to a handle: every handle sets the same value,
// so creating one model never lowers the limit another model's launches need.
inline cudaError_t gmf_smem_limit(const void* kernel, size_t need) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    const int lim = optin - (int)fa.sharedSizeBytes;
    if (need > (size_t)lim) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

// gmf_update.cu: the strip-update launch that follows each tile launch of a
// sweep (tile edge T); the multi-model form takes one StepArgs per model.
cudaError_t gmf_launch_update(const StepArgs& a, int w, int T, cudaStream_t st);
cudaError_t gmf_launch_update_multi(const StepArgs* d_args, int nmodels, int units, size_t smem, int w, int T,
                                    cudaStream_t st);
int gmf_update_units(const StepArgs& a, int T);
// the tensor-core path's update launch (row-major partial slots, see gmf_update.cuh)
cudaError_t gmf_launch_update_tc(const StepArgs& a, int w, int T, cudaStream_t st);
cudaError_t gmf_launch_update_tc_multi(const StepArgs* d_args, int nmodels, int units, int threads, int w, int T,
                                       cudaStream_t st);
int gmf_update_tc_threads(const StepArgs& a);
int gmf_update_tc_units(const StepArgs& a, int T);
cudaError_t gmf_launch_chunk_state(float* P, float* Gb, float* Hb, int* cnt, int KP, int nf, int64_t first, int rows,
                                   float* buf, int write, cudaStream_t st);
size_t gmf_update_smem(const StepArgs& a);

// gmf_api.cu
int gmf_stage_schedule(gmf_model* h, const int32_t* sigma, int w_begin, int w_end, cudaStream_t st);
int gmf_init_shared(gmf_model** out, const gmf_config* cfg, const gmf_model* owner, const double* X, const double* Z,
                    const double* offset, const double* B0, const double* G0, const double* U0, const double* V0,
                    double alpha0, void* stream);
int gmf_fail(int code, const char* msg);

// gmf_step_simt.cu
StepArgs gmf_make_args(gmf_model* h);
cudaError_t gmf_launch_sweep_simt(gmf_model* h, const StepArgs& a, int w, cudaStream_t st);
cudaError_t gmf_sweep_simt_attr(gmf_model* h);
cudaError_t gmf_launch_deviance(gmf_model* h, double* d_out, cudaStream_t st);
cudaError_t gmf_launch_sum_parts(const double* part, int count, double* out, cudaStream_t st);
// gmf_step_tc.cu: the full deviance on the tensor cores (mixed-precision handles)
int gmf_tc_deviance_ok(const gmf_model* h);
cudaError_t gmf_tc_launch_deviance(gmf_model* h, double* d_out, cudaStream_t st);
cudaError_t gmf_launch_permute_y(const void* src, void* dst, int y16, int64_t n, int64_t m,
                                 const int* rperm, const int* cperm, cudaStream_t st);
// Yp[i][j] = Y[rperm[i]][cperm[j]] with Y in mapped host memory (16-byte
// aligned, rows of a multiple of 16 bytes); gmf_gather_host_ok says whether a
// row fits the kernel's shared memory.
cudaError_t gmf_launch_gather_host(const void* src, void* dst, int y16, int64_t n, int64_t m, const int* rperm,
                                   const int* cperm, cudaStream_t st);
int gmf_gather_host_ok(int y16, int64_t m);
cudaError_t gmf_launch_permute_w(const float* src, float* dst, int64_t n, int64_t m,
                                 const int* rperm, const int* cperm, cudaStream_t st);
