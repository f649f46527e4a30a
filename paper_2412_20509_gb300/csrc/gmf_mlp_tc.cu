// First layer of the warm-start encoder on the tcgen05 tensor cores:
//   z1 = W1 log(1 + y) + b1,  h1 = gelu(z1)      (128 cells per CTA, n_h1 <= 256)
// with BF16 operands and an FP32 accumulator in TMEM. The layer holds ~90% of
// the encoder's products (n_in = 3000 against 256 x 256 and 256 x 20).
//
// Per CTA, a pipeline over K in chunks of 64 with S stages:
//   warp 8 (one thread): TMA of the W1 chunk (BF16, 128-byte swizzle, the
//     B operand) and of the raw count chunk (128 rows x 64 counts);
//   warps 0-7: log(1 + y) of the raw chunk (a table for y < 256), rounded to
//     BF16 into the swizzled A operand; one arrival per warp;
//   warp 9 (one thread): four MMAs of K = 16 per chunk, then a commit that
//     frees the stage for the next TMA;
//   warps 0-3 at the end: TMEM -> + b1 -> z1, gelu(z1) (exact erf form), FP32.
// Every mbarrier wait is bounded; a wait that gives up sets the status word
// and the CTA skips the rest of its work (no hang).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>

#include <algorithm>
#include <string>

#include "gmf_internal.cuh"
#include "gmf_mlp_tc.cuh"
#include "gmf_sm100.cuh"

using namespace sm100;

namespace {

constexpr int BM = 128;                  // cells per CTA (MMA M)
constexpr int BKC = 64;                  // K per chunk: one 128-byte BF16 row
constexpr int NTH = 320;                 // warps 0-7 convert, 8 loads, 9 issues MMAs
constexpr uint32_t A_BYTES = BM * 128;   // A stage: 128 rows x 128 bytes
constexpr uint32_t WAIT_POLLS = 1u << 24;
constexpr int SMAX = 4;

struct L1Args {
    int64_t rows;        // cells of this launch
    int K;               // n_in
    int N;               // n_h1 (multiple of 16, <= 256)
    int nk;              // chunks: ceil(K / 64)
    int S;               // pipeline stages
    uint32_t b_bytes;    // W1 stage: N rows x 128 bytes
    uint32_t y_bytes;    // raw count stage: 128 rows x 64 counts
    uint32_t stage;      // bytes of one stage (A + B + raw counts), 1024-aligned
    const float* b1;
    float* Z1;           // rows x N (may be null)
    float* H1;           // rows x N
    unsigned* err;
};

__device__ __forceinline__ float gelu_f(float t) { return 0.5f * t * (1.f + erff(t * 0.70710678118654752f)); }

__device__ __forceinline__ bool wait_bounded(uint64_t* bar, uint32_t parity, unsigned* err) {
    if (mbar_wait(bar, parity, WAIT_POLLS)) return true;
    atomicOr(err, GMF_DEVERR_TIMEOUT);
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <bool Y16>
__global__ void __launch_bounds__(NTH, 1)
    mlp_l1_tc(L1Args a, const __grid_constant__ CUtensorMap wmap, const __grid_constant__ CUtensorMap ymap) {
    extern __shared__ __align__(1024) uint8_t smraw[];
    __shared__ uint64_t full_tma[SMAX], full_a[SMAX], empty[SMAX], done;
    __shared__ uint32_t tmem_base;
    __shared__ uint16_t tab[256];  // BF16 bits of log(1 + v), v < 256
    __shared__ int s_ok;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t* sm = smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u);
    const int64_t row0 = (int64_t)blockIdx.x * BM;
    const int S = a.S;

    if (tid < 256) tab[tid] = (uint16_t)(pack_bf16x2(log1pf((float)tid), 0.f) & 0xFFFFu);
    if (tid == 0) {
        for (int s = 0; s < S; s++) {
            mbar_init(&full_tma[s], 1);
            mbar_init(&full_a[s], 8);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        fence_mbar_init();
        s_ok = 1;
    }
    if (warp == 9) tmem_alloc(&tmem_base, 256);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tb = tmem_base;

    if (warp == 8) {
        if (lane == 0) {
            for (int kc = 0; kc < a.nk; kc++) {
                const int s = kc % S;
                uint8_t* st = sm + (size_t)s * a.stage;
                if (kc >= S && !wait_bounded(&empty[s], (uint32_t)((kc / S) + 1) & 1u, a.err)) {
                    s_ok = 0;
                    break;
                }
                mbar_arrive_expect_tx(&full_tma[s], a.b_bytes + a.y_bytes);
                tma_load_2d(st + A_BYTES, &wmap, kc * BKC, 0, &full_tma[s]);
                tma_load_2d(st + A_BYTES + a.b_bytes, &ymap, kc * BKC, (int)row0, &full_tma[s]);
            }
        }
    } else if (warp == 9) {
        if (lane == 0) {
            const uint32_t id = idesc_bf16(BM, a.N, 0, 0);
            bool ok = true;
            for (int kc = 0; kc < a.nk && ok; kc++) {
                const int s = kc % S;
                if (!wait_bounded(&full_a[s], (uint32_t)(kc / S) & 1u, a.err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t abase = smem_u32(sm + (size_t)s * a.stage), bbase = abase + A_BYTES;
#pragma unroll
                for (int ks = 0; ks < BKC / 16; ks++)
                    umma_bf16(tb, sdesc(abase + 32u * ks, 16, 1024, SWIZZLE_128B),
                              sdesc(bbase + 32u * ks, 16, 1024, SWIZZLE_128B), id, (kc > 0 || ks > 0) ? 1u : 0u);
                umma_commit(&empty[s]);
            }
            if (!ok) s_ok = 0;
            umma_commit(&done);
        }
    } else {
        // converters: thread c -> row c / 2, counts [32 (c % 2), 32 (c % 2) + 32) of the chunk
        const int c = tid, r = c >> 1, h = c & 1;
        for (int kc = 0; kc < a.nk; kc++) {
            const int s = kc % S;
            uint8_t* st = sm + (size_t)s * a.stage;
            if (!wait_bounded(&full_tma[s], (uint32_t)(kc / S) & 1u, a.err)) {
                s_ok = 0;
                break;
            }
            const uint8_t* raw = st + A_BYTES + a.b_bytes;
            uint32_t pk[16];
#pragma unroll
            for (int q = 0; q < 4; q++) {  // 8 counts per 16-byte chunk of the A row
                float v[8];
                if (Y16) {
                    const uint4 u = *(const uint4*)(raw + (size_t)r * 128 + h * 64 + q * 16);
                    const uint32_t w4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                    for (int t = 0; t < 4; t++) {
                        v[2 * t] = (float)(w4[t] & 0xFFFFu);
                        v[2 * t + 1] = (float)(w4[t] >> 16);
                    }
                } else {
                    const int4 u0 = *(const int4*)(raw + (size_t)r * 256 + h * 128 + q * 32);
                    const int4 u1 = *(const int4*)(raw + (size_t)r * 256 + h * 128 + q * 32 + 16);
                    v[0] = (float)u0.x; v[1] = (float)u0.y; v[2] = (float)u0.z; v[3] = (float)u0.w;
                    v[4] = (float)u1.x; v[5] = (float)u1.y; v[6] = (float)u1.z; v[7] = (float)u1.w;
                }
#pragma unroll
                for (int t = 0; t < 4; t++) {
                    uint32_t lo, hi;
                    const float x0 = v[2 * t], x1 = v[2 * t + 1];
                    lo = (x0 >= 0.f && x0 < 256.f) ? (uint32_t)tab[(int)x0] : (pack_bf16x2(log1pf(x0), 0.f) & 0xFFFFu);
                    hi = (x1 >= 0.f && x1 < 256.f) ? (uint32_t)tab[(int)x1] : (pack_bf16x2(log1pf(x1), 0.f) & 0xFFFFu);
                    pk[4 * q + t] = lo | (hi << 16);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const uint32_t off = sw128_off((uint32_t)r, (uint32_t)(h * 64 + q * 16));
                asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(smem_u32(st + off)), "r"(pk[4 * q]),
                             "r"(pk[4 * q + 1]), "r"(pk[4 * q + 2]), "r"(pk[4 * q + 3])
                             : "memory");
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&full_a[s]);
        }
    }

    // epilogue: warps 0-3 own TMEM lanes 32w .. 32w + 31 = tile rows
    if (warp < 4) {
        const bool ok = wait_bounded(&done, 0, a.err);
        tc_fence_after();
        const int r = 32 * warp + lane;
        const int64_t row = row0 + r;
        if (ok) {
            for (int n0 = 0; n0 < a.N; n0 += 32) {
                uint32_t v[32];
                tmem_ld32(tb + ((uint32_t)(32 * warp) << 16) + (uint32_t)n0, v);
                tmem_wait_ld();
                if (row < a.rows) {
#pragma unroll
                    for (int u = 0; u < 32; u += 4) {
                        float z[4], g[4];
#pragma unroll
                        for (int t = 0; t < 4; t++) {
                            z[t] = __uint_as_float(v[u + t]) + __ldg(a.b1 + n0 + u + t);
                            g[t] = gelu_f(z[t]);
                        }
                        const int64_t o = row * a.N + n0 + u;
                        if (a.Z1) *(float4*)(a.Z1 + o) = make_float4(z[0], z[1], z[2], z[3]);
                        *(float4*)(a.H1 + o) = make_float4(g[0], g[1], g[2], g[3]);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 9) {
        // a CTA that gave up waits once more (bounded) for its own MMAs before freeing TMEM
        if (!s_ok) mbar_wait(&done, 0, WAIT_POLLS);
        tmem_dealloc(tb, 256);
    }
}

__global__ void w1_to_bf16(const float* W, int N, int K, int Kp, __nv_bfloat16* out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)N * Kp;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(e / Kp), k = (int)(e - (int64_t)n * Kp);
        out[e] = __float2bfloat16_rn(k < K ? W[(int64_t)n * K + k] : 0.f);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) ==
                cudaSuccess &&
            p)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

}  // namespace

int gmf_mlp_tc_check(int n_in, int n_h1, std::string* err) {
    if (n_h1 % 16 != 0 || n_h1 < 16 || n_h1 > 256) {
        *err = "the tensor-core encoder needs n_h1 a multiple of 16 in [16, 256]";
        return GMF_ERR_ARG;
    }
    if (n_in < 1) {
        *err = "n_in must be positive";
        return GMF_ERR_ARG;
    }
    return GMF_OK;
}

int gmf_mlp_tc_weights(const float* W1, int n_h1, int n_in, __nv_bfloat16* W1b, cudaStream_t st) {
    const int Kp = (n_in + BKC - 1) / BKC * BKC;
    const int64_t tot = (int64_t)n_h1 * Kp;
    w1_to_bf16<<<(int)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, st>>>(W1, n_h1, n_in, Kp, W1b);
    return cudaGetLastError() == cudaSuccess ? GMF_OK : GMF_ERR_CUDA;
}

size_t gmf_mlp_tc_w1_elems(int n_h1, int n_in) { return (size_t)n_h1 * ((n_in + BKC - 1) / BKC * BKC); }

int gmf_mlp_tc_layer1(const void* Y, int y16, int64_t rows, int n_in, int n_h1, const __nv_bfloat16* W1b,
                      const float* b1, float* Z1, float* H1, unsigned* err_word, cudaStream_t st, std::string* err) {
    const size_t es = y16 ? 2 : 4;
    if (((uintptr_t)Y) % 16 != 0 || ((size_t)n_in * es) % 16 != 0) {
        *err = "the tensor-core encoder needs 16-byte aligned counts and n_in * sizeof(count) a multiple of 16";
        return GMF_ERR_ARG;
    }
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) {
        *err = "cuTensorMapEncodeTiled is not available";
        return GMF_ERR_CUDA;
    }
    L1Args a{};
    a.rows = rows;
    a.K = n_in;
    a.N = n_h1;
    a.nk = (n_in + BKC - 1) / BKC;
    a.b_bytes = (uint32_t)n_h1 * 128u;
    a.y_bytes = (uint32_t)(BM * BKC * es);
    a.stage = (A_BYTES + a.b_bytes + a.y_bytes + 1023u) & ~1023u;
    int optin = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const uint32_t avail = (uint32_t)optin - 2048u - 1024u;  // static shared memory and alignment slack
    a.S = (int)std::min<uint32_t>(SMAX, avail / a.stage);
    if (a.S < 2) {
        *err = "the tensor-core encoder's pipeline does not fit in shared memory";
        return GMF_ERR_ARG;
    }
    a.b1 = b1;
    a.Z1 = Z1;
    a.H1 = H1;
    a.err = err_word;
    const int Kp = a.nk * BKC;
    CUtensorMap wmap, ymap;
    cuuint64_t wd[2] = {(cuuint64_t)Kp, (cuuint64_t)n_h1};
    cuuint64_t ws[1] = {(cuuint64_t)Kp * 2};
    cuuint32_t wb[2] = {(cuuint32_t)BKC, (cuuint32_t)n_h1};
    cuuint32_t one[2] = {1, 1};
    CUresult cr = enc(&wmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)W1b, wd, ws, wb, one,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    cuuint64_t yd[2] = {(cuuint64_t)n_in, (cuuint64_t)rows};
    cuuint64_t ys[1] = {(cuuint64_t)n_in * es};
    cuuint32_t yb[2] = {(cuuint32_t)BKC, (cuuint32_t)BM};
    if (cr == CUDA_SUCCESS)
        cr = enc(&ymap, y16 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_INT32, 2, (void*)Y, yd, ys, yb,
                 one, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) {
        *err = "cuTensorMapEncodeTiled failed for the encoder's operands";
        return GMF_ERR_CUDA;
    }
    const size_t smem = (size_t)a.S * a.stage + 1024;
    const void* fn = y16 ? (const void*)mlp_l1_tc<true> : (const void*)mlp_l1_tc<false>;
    cudaError_t e = gmf_smem_limit(fn, smem);
    if (e == cudaSuccess) {
        const dim3 grid((unsigned)((rows + BM - 1) / BM));
        if (y16)
            mlp_l1_tc<true><<<grid, NTH, smem, st>>>(a, wmap, ymap);
        else
            mlp_l1_tc<false><<<grid, NTH, smem, st>>>(a, wmap, ymap);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        *err = cudaGetErrorString(e);
        return GMF_ERR_CUDA;
    }
    return GMF_OK;
}
