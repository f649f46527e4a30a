// Warm-start encoder for new cells: a small MLP from log(1 + counts) of one cell
// to its latent scores, trained on (counts, fitted U) pairs that the GMF fit
// produces, so that the per-cell projection (gmf_project_cells) can start near
// its optimum. The paper has no network; it supplies the targets (the scores
// of the fitted, orthogonalised model, Sec. 2.1) and the projection it warms up.
//
//   x = log1p(y);  z1 = W1 x + b1, h1 = gelu(z1);  z2 = W2 h1 + b2, h2 = gelu(z2);
//   o = W3 h2 + b3;  loss = mean (o - target)^2;  Adam on all parameters.
// gelu(t) = t Phi(t) (exact, erf). All products run on one FP32 tiled GEMM
// kernel whose operands are read through strides (so A, A', B, B' all work
// without copies), with log1p of the counts fused into the loader and the
// bias / gelu / gelu' epilogues fused into the store. Every reduction has a
// fixed order, so training is bitwise reproducible.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <utility>
#include <vector>

#include "gmf_internal.cuh"
#include "gmf_mlp_tc.cuh"

namespace {

constexpr int TB = 64, BK = 16, NT = 256;

enum { SRC_F32 = 0, SRC_I32 = 1, SRC_U16 = 2 };  // operand source: float, or counts read as log1p
enum { EPI_STORE = 0, EPI_BIAS_GELU = 1, EPI_GELU_BWD = 2, EPI_BIAS = 3 };

struct Gemm {
    int64_t M, N, K;
    const void* A;
    int64_t sam, sak;   // A(m, k) at A[m*sam + k*sak]
    const void* B;
    int64_t sbk, sbn;   // B(k, n) at B[k*sbk + n*sbn]
    float* C;           // C[m*ldc + n]
    int64_t ldc;
    const float* bias;  // [N] (EPI_BIAS_GELU, EPI_BIAS)
    float* H;           // gelu output [m*ldc + n] (EPI_BIAS_GELU)
    const float* Zp;    // pre-activation whose gelu' scales the result (EPI_GELU_BWD)
};

template <int SRC>
__device__ __forceinline__ float ld(const void* p, int64_t i) {
    if (SRC == SRC_F32) return __ldg((const float*)p + i);
    if (SRC == SRC_I32) return log1pf((float)__ldg((const int*)p + i));
    return log1pf((float)__ldg((const unsigned short*)p + i));
}

__device__ __forceinline__ float gelu(float t) { return 0.5f * t * (1.f + erff(t * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_prime(float t) {
    return 0.5f * (1.f + erff(t * 0.70710678118654752f)) + t * expf(-0.5f * t * t) * 0.39894228040143268f;
}

template <int SA, int SB, int EPI>
__global__ void __launch_bounds__(NT) gemm_kernel(Gemm g) {
    __shared__ __align__(16) float As[BK][TB + 4];
    __shared__ __align__(16) float Bs[BK][TB + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * TB, n0 = (int64_t)blockIdx.x * TB;
    float acc[4][4] = {};
    for (int64_t k0 = 0; k0 < g.K; k0 += BK) {
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int e = tid + u * NT;  // 0..1023 over a 64 x 16 tile
            // A tile element (row mm, col kk); consecutive threads walk along k when A is k-contiguous
            const int amm = g.sak == 1 ? e / BK : e % TB, akk = g.sak == 1 ? e % BK : e / TB;
            const int64_t am = m0 + amm, ak = k0 + akk;
            As[akk][amm] = (am < g.M && ak < g.K) ? ld<SA>(g.A, am * g.sam + ak * g.sak) : 0.f;
            const int bnn = g.sbn == 1 ? e % TB : e / BK, bkk = g.sbn == 1 ? e / TB : e % BK;
            const int64_t bn = n0 + bnn, bk = k0 + bkk;
            Bs[bkk][bnn] = (bn < g.N && bk < g.K) ? ld<SB>(g.B, bk * g.sbk + bn * g.sbn) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk++) {
            const float4 a = *(const float4*)&As[kk][4 * ty];
            const float4 b = *(const float4*)&Bs[kk][4 * tx];
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int64_t m = m0 + 4 * ty + i;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int64_t n = n0 + 4 * tx + j;
            if (n >= g.N) continue;
            float v = acc[i][j];
            const int64_t o = m * g.ldc + n;
            if (EPI == EPI_BIAS_GELU) {
                v += g.bias[n];
                g.C[o] = v;
                g.H[o] = gelu(v);
            } else if (EPI == EPI_BIAS) {
                g.C[o] = v + g.bias[n];
            } else if (EPI == EPI_GELU_BWD) {
                g.C[o] = v * gelu_prime(g.Zp[o]);
            } else {
                g.C[o] = v;
            }
        }
    }
}

// Column sums of a rows x cols matrix (bias gradients), one thread per column, rows in order.
__global__ void colsum_kernel(const float* D, int64_t rows, int cols, float* out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int64_t r = 0; r < rows; r++) s += D[r * cols + c];
    out[c] = s;
}

// dO = 2 (O - T) / (rows * cols); loss = mean (O - T)^2 (one block, fixed order).
__global__ void mse_kernel(const float* O, const float* T, int64_t count, float* dO, float* loss) {
    __shared__ float red[NT / 32];
    float s = 0.f;
    const float sc = 2.f / (float)count;
    for (int64_t e = threadIdx.x; e < count; e += NT) {
        const float r = O[e] - T[e];
        dO[e] = sc * r;
        s = fmaf(r, r, s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int u = 0; u < NT / 32; u++) t += red[u];
        *loss = t / (float)count;
    }
}

__global__ void adam_kernel(float* P, const float* G, float* M, float* V, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float g = G[i];
        const float m = b1 * M[i] + (1.f - b1) * g;
        const float v = b2 * V[i] + (1.f - b2) * g * g;
        M[i] = m;
        V[i] = v;
        P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

template <typename Ty>
__global__ void gather_rows(const Ty* src, int64_t ld, const int64_t* idx, int64_t rows, int cols, Ty* dst) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * cols; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / cols;
        const int c = (int)(e - r * cols);
        dst[e] = src[idx[r] * ld + c];
    }
}

int grid1(int64_t n) { return (int)std::min<int64_t>((n + NT - 1) / NT, 8192); }

}  // namespace

struct gmf_mlp {
    int n_in, h1, h2, n_out, max_batch;
    int64_t off[7];        // parameter offsets: W1 b1 W2 b2 W3 b3, total
    float* P = nullptr;    // parameters
    float* G = nullptr;    // gradients
    float* M = nullptr;    // Adam moments
    float* V = nullptr;
    int64_t k = 0;         // Adam step count
    float *Z1 = nullptr, *H1 = nullptr, *Z2 = nullptr, *H2 = nullptr, *O = nullptr, *dO = nullptr;
    float *dZ2 = nullptr, *dZ1 = nullptr, *loss = nullptr;
    void* yb = nullptr;    // gathered batch counts (int32 bytes)
    float* tb = nullptr;   // gathered batch targets
    int64_t* idx = nullptr;
    int prec = GMF_PREC_FP32;        // GMF_PREC_MIXED: first layer on the tensor cores (BF16 W1 and inputs)
    __nv_bfloat16* W1b = nullptr;    // padded BF16 copy of W1 (mixed)
    unsigned* err = nullptr;         // device status word of the tensor-core layer
};

static void mlp_release(gmf_mlp* n) {
    if (!n) return;
    void* ptrs[] = {n->P, n->G, n->M, n->V, n->Z1, n->H1, n->Z2, n->H2, n->O, n->dO, n->dZ2, n->dZ1, n->loss,
                    n->yb, n->tb, n->idx, n->W1b, n->err};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete n;
}

extern "C" void gmf_mlp_free(gmf_mlp* n) { mlp_release(n); }

extern "C" int gmf_mlp_create(gmf_mlp** out, int32_t n_in, int32_t n_h1, int32_t n_h2, int32_t n_out,
                              int32_t max_batch, void* stream) {
    if (!out) return gmf_fail(GMF_ERR_ARG, "gmf_mlp_create: out is NULL");
    *out = nullptr;
    if (n_in < 1 || n_h1 < 1 || n_h2 < 1 || n_out < 1 || max_batch < 1)
        return gmf_fail(GMF_ERR_ARG, "gmf_mlp_create: sizes must be positive");
    gmf_mlp* n = new gmf_mlp();
    n->n_in = n_in;
    n->h1 = n_h1;
    n->h2 = n_h2;
    n->n_out = n_out;
    n->max_batch = max_batch;
    const int64_t sz[6] = {(int64_t)n_h1 * n_in, n_h1, (int64_t)n_h2 * n_h1, n_h2, (int64_t)n_out * n_h2, n_out};
    n->off[0] = 0;
    for (int i = 0; i < 6; i++) n->off[i + 1] = n->off[i] + sz[i];
    const int64_t np = n->off[6], B = max_batch;
    bool ok = cudaMalloc(&n->P, sizeof(float) * np) == cudaSuccess && cudaMalloc(&n->G, sizeof(float) * np) == cudaSuccess &&
              cudaMalloc(&n->M, sizeof(float) * np) == cudaSuccess && cudaMalloc(&n->V, sizeof(float) * np) == cudaSuccess &&
              cudaMalloc(&n->Z1, sizeof(float) * B * n_h1) == cudaSuccess &&
              cudaMalloc(&n->H1, sizeof(float) * B * n_h1) == cudaSuccess &&
              cudaMalloc(&n->Z2, sizeof(float) * B * n_h2) == cudaSuccess &&
              cudaMalloc(&n->H2, sizeof(float) * B * n_h2) == cudaSuccess &&
              cudaMalloc(&n->O, sizeof(float) * B * n_out) == cudaSuccess &&
              cudaMalloc(&n->dO, sizeof(float) * B * n_out) == cudaSuccess &&
              cudaMalloc(&n->dZ2, sizeof(float) * B * n_h2) == cudaSuccess &&
              cudaMalloc(&n->dZ1, sizeof(float) * B * n_h1) == cudaSuccess &&
              cudaMalloc(&n->loss, sizeof(float)) == cudaSuccess &&
              cudaMalloc(&n->yb, sizeof(int) * B * n_in) == cudaSuccess &&
              cudaMalloc(&n->tb, sizeof(float) * B * n_out) == cudaSuccess &&
              cudaMalloc(&n->idx, sizeof(int64_t) * B) == cudaSuccess;
    if (!ok) {
        mlp_release(n);
        return gmf_fail(GMF_ERR_OOM, "gmf_mlp_create: device allocation failed");
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaMemsetAsync(n->P, 0, sizeof(float) * np, st);
    cudaMemsetAsync(n->G, 0, sizeof(float) * np, st);
    cudaMemsetAsync(n->M, 0, sizeof(float) * np, st);
    cudaMemsetAsync(n->V, 0, sizeof(float) * np, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        mlp_release(n);
        return gmf_fail(GMF_ERR_CUDA, "gmf_mlp_create: initialisation failed");
    }
    *out = n;
    return GMF_OK;
}

static int copy_params(gmf_mlp* n, float* base, const float* const* host, bool to_device, cudaStream_t st) {
    for (int i = 0; i < 6; i++) {
        if (!host[i]) continue;
        const size_t bytes = sizeof(float) * (size_t)(n->off[i + 1] - n->off[i]);
        const cudaError_t e = to_device
                                  ? cudaMemcpyAsync(base + n->off[i], host[i], bytes, cudaMemcpyHostToDevice, st)
                                  : cudaMemcpyAsync((void*)host[i], base + n->off[i], bytes, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return gmf_fail(GMF_ERR_CUDA, "gmf_mlp: parameter copy failed");
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return gmf_fail(GMF_ERR_CUDA, "gmf_mlp: parameter copy failed");
    return GMF_OK;
}

extern "C" int gmf_mlp_set_params(gmf_mlp* n, const float* W1, const float* b1, const float* W2, const float* b2,
                                  const float* W3, const float* b3, void* stream) {
    if (!n) return gmf_fail(GMF_ERR_ARG, "gmf_mlp_set_params: NULL handle");
    const float* h[6] = {W1, b1, W2, b2, W3, b3};
    n->k = 0;
    cudaMemsetAsync(n->M, 0, sizeof(float) * n->off[6], (cudaStream_t)stream);
    cudaMemsetAsync(n->V, 0, sizeof(float) * n->off[6], (cudaStream_t)stream);
    const int rc = copy_params(n, n->P, h, true, (cudaStream_t)stream);
    if (rc == GMF_OK && n->prec == GMF_PREC_MIXED &&
        gmf_mlp_tc_weights(n->P + n->off[0], n->h1, n->n_in, n->W1b, (cudaStream_t)stream) != GMF_OK)
        return gmf_fail(GMF_ERR_CUDA, "gmf_mlp_set_params: BF16 copy of W1 failed");
    return rc;
}

extern "C" int gmf_mlp_set_precision(gmf_mlp* n, int32_t precision, void* stream) {
    if (!n) return gmf_fail(GMF_ERR_ARG, "gmf_mlp_set_precision: NULL handle");
    if (precision != GMF_PREC_FP32 && precision != GMF_PREC_MIXED)
        return gmf_fail(GMF_ERR_ARG, "gmf_mlp_set_precision: precision must be GMF_PREC_FP32 or GMF_PREC_MIXED");
    if (precision == GMF_PREC_MIXED) {
        std::string msg;
        if (gmf_mlp_tc_check(n->n_in, n->h1, &msg) != GMF_OK)
            return gmf_fail(GMF_ERR_ARG, ("gmf_mlp_set_precision: " + msg).c_str());
        if (!n->W1b && (cudaMalloc(&n->W1b, sizeof(__nv_bfloat16) * gmf_mlp_tc_w1_elems(n->h1, n->n_in)) != cudaSuccess ||
                        cudaMalloc(&n->err, sizeof(unsigned)) != cudaSuccess))
            return gmf_fail(GMF_ERR_OOM, "gmf_mlp_set_precision: device allocation failed");
        cudaMemsetAsync(n->err, 0, sizeof(unsigned), (cudaStream_t)stream);
        if (gmf_mlp_tc_weights(n->P + n->off[0], n->h1, n->n_in, n->W1b, (cudaStream_t)stream) != GMF_OK)
            return gmf_fail(GMF_ERR_CUDA, "gmf_mlp_set_precision: BF16 copy of W1 failed");
    }
    n->prec = precision;
    return GMF_OK;
}
extern "C" int gmf_mlp_get_params(gmf_mlp* n, float* W1, float* b1, float* W2, float* b2, float* W3, float* b3,
                                  void* stream) {
    if (!n) return gmf_fail(GMF_ERR_ARG, "gmf_mlp_get_params: NULL handle");
    const float* h[6] = {W1, b1, W2, b2, W3, b3};
    return copy_params(n, n->P, h, false, (cudaStream_t)stream);
}
extern "C" int gmf_mlp_get_grads(gmf_mlp* n, float* W1, float* b1, float* W2, float* b2, float* W3, float* b3,
                                 void* stream) {
    if (!n) return gmf_fail(GMF_ERR_ARG, "gmf_mlp_get_grads: NULL handle");
    const float* h[6] = {W1, b1, W2, b2, W3, b3};
    return copy_params(n, n->G, h, false, (cudaStream_t)stream);
}

template <int SA, int SB, int EPI>
static cudaError_t run_gemm(const Gemm& g, cudaStream_t st) {
    dim3 grid((unsigned)((g.N + TB - 1) / TB), (unsigned)((g.M + TB - 1) / TB));
    gemm_kernel<SA, SB, EPI><<<grid, NT, 0, st>>>(g);
    return cudaGetLastError();
}

// Message of the last failure inside the tensor-core first layer (reported by the ABI call).
static thread_local std::string tl_layer_msg;

// ABI status for a failed forward / backward pass.
static int pass_fail(const char* fn, cudaError_t e) {
    std::string m = std::string(fn) + ": " + (tl_layer_msg.empty() ? cudaGetErrorString(e) : tl_layer_msg);
    const int code = tl_layer_msg.empty() ? GMF_ERR_CUDA : GMF_ERR_ARG;
    tl_layer_msg.clear();
    return gmf_fail(code, m.c_str());
}

static cudaError_t forward_l1_simt(gmf_mlp* n, const void* Y, int y16, int64_t ldy, int64_t rows, cudaStream_t st);
static cudaError_t forward_l23(gmf_mlp* n, int64_t rows, float* out, cudaStream_t st);

// Forward pass of `rows` cells whose counts start at Y (row stride ldy); output rows x n_out.
static cudaError_t forward(gmf_mlp* n, const void* Y, int y16, int64_t ldy, int64_t rows, float* out, cudaStream_t st) {
    float* P = n->P;
    cudaError_t e = cudaSuccess;
    if (n->prec == GMF_PREC_MIXED) {
        std::string msg;
        if (ldy != n->n_in) msg = "the tensor-core encoder reads contiguous rows of n_in counts";
        if (!msg.empty() ||
            gmf_mlp_tc_layer1(Y, y16, rows, n->n_in, n->h1, n->W1b, P + n->off[1], n->Z1, n->H1, n->err, st, &msg) !=
                GMF_OK) {
            tl_layer_msg = msg;
            return cudaErrorInvalidValue;
        }
    } else {
        e = forward_l1_simt(n, Y, y16, ldy, rows, st);
        if (e != cudaSuccess) return e;
    }
    return forward_l23(n, rows, out, st);
}

// First layer on the FP32 CUDA-core GEMM.
static cudaError_t forward_l1_simt(gmf_mlp* n, const void* Y, int y16, int64_t ldy, int64_t rows, cudaStream_t st) {
    float* P = n->P;
    Gemm g{};
    g.M = rows;
    g.N = n->h1;
    g.K = n->n_in;
    g.A = Y;
    g.sam = ldy;
    g.sak = 1;
    g.B = P + n->off[0];
    g.sbk = 1;
    g.sbn = n->n_in;
    g.C = n->Z1;
    g.ldc = n->h1;
    g.bias = P + n->off[1];
    g.H = n->H1;
    return y16 ? run_gemm<SRC_U16, SRC_F32, EPI_BIAS_GELU>(g, st) : run_gemm<SRC_I32, SRC_F32, EPI_BIAS_GELU>(g, st);
}

// Layers 2 and 3 (FP32 CUDA-core GEMM) from H1.
static cudaError_t forward_l23(gmf_mlp* n, int64_t rows, float* out, cudaStream_t st) {
    float* P = n->P;
    cudaError_t e = cudaSuccess;
    Gemm g{};
    g.M = rows;
    g.N = n->h2;
    g.K = n->h1;
    g.A = n->H1;
    g.sam = n->h1;
    g.sak = 1;
    g.B = P + n->off[2];
    g.sbk = 1;
    g.sbn = n->h1;
    g.C = n->Z2;
    g.ldc = n->h2;
    g.bias = P + n->off[3];
    g.H = n->H2;
    if ((e = run_gemm<SRC_F32, SRC_F32, EPI_BIAS_GELU>(g, st)) != cudaSuccess) return e;
    g = Gemm{};
    g.M = rows;
    g.N = n->n_out;
    g.K = n->h2;
    g.A = n->H2;
    g.sam = n->h2;
    g.sak = 1;
    g.B = P + n->off[4];
    g.sbk = 1;
    g.sbn = n->h2;
    g.C = out;
    g.ldc = n->n_out;
    g.bias = P + n->off[5];
    return run_gemm<SRC_F32, SRC_F32, EPI_BIAS>(g, st);
}

// Loss and gradients of a batch already laid out contiguously (rows <= max_batch).
static cudaError_t backward(gmf_mlp* n, const void* Y, int y16, int64_t ldy, int64_t rows, const float* T,
                            cudaStream_t st) {
    cudaError_t e = forward(n, Y, y16, ldy, rows, n->O, st);
    if (e != cudaSuccess) return e;
    mse_kernel<<<1, NT, 0, st>>>(n->O, T, rows * n->n_out, n->dO, n->loss);
    float* P = n->P;
    float* G = n->G;
    Gemm g{};
    // dW3 = dO' H2
    g.M = n->n_out; g.N = n->h2; g.K = rows;
    g.A = n->dO; g.sam = 1; g.sak = n->n_out;
    g.B = n->H2; g.sbk = n->h2; g.sbn = 1;
    g.C = G + n->off[4]; g.ldc = n->h2;
    if ((e = run_gemm<SRC_F32, SRC_F32, EPI_STORE>(g, st)) != cudaSuccess) return e;
    colsum_kernel<<<(n->n_out + NT - 1) / NT, NT, 0, st>>>(n->dO, rows, n->n_out, G + n->off[5]);
    // dZ2 = (dO W3) * gelu'(Z2)
    g = Gemm{};
    g.M = rows; g.N = n->h2; g.K = n->n_out;
    g.A = n->dO; g.sam = n->n_out; g.sak = 1;
    g.B = P + n->off[4]; g.sbk = n->h2; g.sbn = 1;
    g.C = n->dZ2; g.ldc = n->h2; g.Zp = n->Z2;
    if ((e = run_gemm<SRC_F32, SRC_F32, EPI_GELU_BWD>(g, st)) != cudaSuccess) return e;
    // dW2 = dZ2' H1
    g = Gemm{};
    g.M = n->h2; g.N = n->h1; g.K = rows;
    g.A = n->dZ2; g.sam = 1; g.sak = n->h2;
    g.B = n->H1; g.sbk = n->h1; g.sbn = 1;
    g.C = G + n->off[2]; g.ldc = n->h1;
    if ((e = run_gemm<SRC_F32, SRC_F32, EPI_STORE>(g, st)) != cudaSuccess) return e;
    colsum_kernel<<<(n->h2 + NT - 1) / NT, NT, 0, st>>>(n->dZ2, rows, n->h2, G + n->off[3]);
    // dZ1 = (dZ2 W2) * gelu'(Z1)
    g = Gemm{};
    g.M = rows; g.N = n->h1; g.K = n->h2;
    g.A = n->dZ2; g.sam = n->h2; g.sak = 1;
    g.B = P + n->off[2]; g.sbk = n->h1; g.sbn = 1;
    g.C = n->dZ1; g.ldc = n->h1; g.Zp = n->Z1;
    if ((e = run_gemm<SRC_F32, SRC_F32, EPI_GELU_BWD>(g, st)) != cudaSuccess) return e;
    // dW1 = dZ1' log1p(Y)
    g = Gemm{};
    g.M = n->h1; g.N = n->n_in; g.K = rows;
    g.A = n->dZ1; g.sam = 1; g.sak = n->h1;
    g.B = Y; g.sbk = ldy; g.sbn = 1;
    g.C = G + n->off[0]; g.ldc = n->n_in;
    e = y16 ? run_gemm<SRC_F32, SRC_U16, EPI_STORE>(g, st) : run_gemm<SRC_F32, SRC_I32, EPI_STORE>(g, st);
    if (e != cudaSuccess) return e;
    colsum_kernel<<<(n->h1 + NT - 1) / NT, NT, 0, st>>>(n->dZ1, rows, n->h1, G + n->off[1]);
    return cudaGetLastError();
}

extern "C" int gmf_mlp_forward(gmf_mlp* n, const void* Y, int32_t y_dtype, int64_t rows, float* out, void* stream) {
    if (!n || rows < 0) return gmf_fail(GMF_ERR_ARG, "gmf_mlp_forward: bad argument");
    if (rows == 0) return GMF_OK;  // an empty batch (its pointers may be NULL)
    if (!Y || !out) return gmf_fail(GMF_ERR_ARG, "gmf_mlp_forward: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    const int y16 = y_dtype == GMF_Y_UINT16;
    const size_t es = y16 ? 2 : 4;
    for (int64_t r0 = 0; r0 < rows; r0 += n->max_batch) {
        const int64_t nr = std::min<int64_t>(n->max_batch, rows - r0);
        const cudaError_t e = forward(n, (const char*)Y + (size_t)r0 * n->n_in * es, y16, n->n_in, nr,
                                      out + r0 * n->n_out, st);
        if (e != cudaSuccess) return pass_fail("gmf_mlp_forward", e);
    }
    return GMF_OK;
}

extern "C" int gmf_mlp_loss_grad(gmf_mlp* n, const void* Y, int32_t y_dtype, int64_t rows, const float* target,
                                 float* loss, void* stream) {
    if (!n || !Y || !target || rows < 1 || rows > n->max_batch)
        return gmf_fail(GMF_ERR_ARG, "gmf_mlp_loss_grad: bad argument (rows must be <= max_batch)");
    cudaStream_t st = (cudaStream_t)stream;
    const cudaError_t e = backward(n, Y, y_dtype == GMF_Y_UINT16, n->n_in, rows, target, st);
    if (e != cudaSuccess) return pass_fail("gmf_mlp_loss_grad", e);
    if (loss && cudaMemcpyAsync(loss, n->loss, sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return gmf_fail(GMF_ERR_CUDA, "gmf_mlp_loss_grad: copy failed");
    return GMF_OK;
}

extern "C" int gmf_mlp_adam(gmf_mlp* n, float lr, float beta1, float beta2, float eps, void* stream) {
    if (!n || !(lr > 0.f)) return gmf_fail(GMF_ERR_ARG, "gmf_mlp_adam: bad argument");
    n->k++;
    const float c1 = 1.f - (float)pow((double)beta1, (double)n->k);
    const float c2 = 1.f - (float)pow((double)beta2, (double)n->k);
    adam_kernel<<<grid1(n->off[6]), NT, 0, (cudaStream_t)stream>>>(n->P, n->G, n->M, n->V, n->off[6], lr, beta1, beta2,
                                                                   eps, c1, c2);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return gmf_fail(GMF_ERR_CUDA, cudaGetErrorString(e));
    if (n->prec == GMF_PREC_MIXED &&
        gmf_mlp_tc_weights(n->P + n->off[0], n->h1, n->n_in, n->W1b, (cudaStream_t)stream) != GMF_OK)
        return gmf_fail(GMF_ERR_CUDA, "gmf_mlp_adam: BF16 copy of W1 failed");
    return GMF_OK;
}

// SplitMix64: the host-side generator of the minibatch order.
static uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// acc += loss * w  (one thread; the batches of an epoch add in order)
static __global__ void loss_acc_kernel(const float* loss, double w, double* acc) { *acc += (double)*loss * w; }

extern "C" int gmf_mlp_train(gmf_mlp* n, const void* Y, int32_t y_dtype, int64_t rows, const float* target,
                             int32_t epochs, int32_t batch, float lr, uint64_t seed, float* losses, void* stream) {
    if (!n || !Y || !target || rows < 1 || epochs < 0 || batch < 1 || batch > n->max_batch || !(lr > 0.f))
        return gmf_fail(GMF_ERR_ARG, "gmf_mlp_train: bad argument (batch must be <= max_batch)");
    if (epochs == 0) return GMF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int y16 = y_dtype == GMF_Y_UINT16;
    // One shuffled order per epoch, drawn on the host while the device trains
    // on the previous one; the epoch losses accumulate on the device and are
    // read once at the end.
    int64_t* d_perm = nullptr;
    double* d_acc = nullptr;
    if (cudaMalloc(&d_perm, sizeof(int64_t) * rows) != cudaSuccess ||
        cudaMalloc(&d_acc, sizeof(double) * epochs) != cudaSuccess) {
        cudaFree(d_perm);
        return gmf_fail(GMF_ERR_OOM, "gmf_mlp_train: device allocation failed");
    }
    auto done = [&](int rc) {
        cudaStreamSynchronize(st);
        cudaFree(d_perm);
        cudaFree(d_acc);
        return rc;
    };
    std::vector<int64_t> perm(rows);
    uint64_t s = seed;
    auto shuffle = [&]() {
        for (int64_t i = 0; i < rows; i++) perm[i] = i;
        for (int64_t i = rows - 1; i > 0; i--) std::swap(perm[i], perm[splitmix(s) % (uint64_t)(i + 1)]);
    };
    if (cudaMemsetAsync(d_acc, 0, sizeof(double) * epochs, st) != cudaSuccess)
        return done(gmf_fail(GMF_ERR_CUDA, "gmf_mlp_train: memset failed"));
    shuffle();
    for (int ep = 0; ep < epochs; ep++) {
        // pageable source: the copy waits for the stream, so the previous epoch is done with d_perm
        if (cudaMemcpyAsync(d_perm, perm.data(), sizeof(int64_t) * rows, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return done(gmf_fail(GMF_ERR_CUDA, "gmf_mlp_train: copy failed"));
        for (int64_t b0 = 0; b0 < rows; b0 += batch) {
            const int64_t nb = std::min<int64_t>(batch, rows - b0);
            const int64_t* idx = d_perm + b0;
            if (y16)
                gather_rows<unsigned short><<<grid1(nb * n->n_in), NT, 0, st>>>(
                    (const unsigned short*)Y, n->n_in, idx, nb, n->n_in, (unsigned short*)n->yb);
            else
                gather_rows<int><<<grid1(nb * n->n_in), NT, 0, st>>>((const int*)Y, n->n_in, idx, nb, n->n_in,
                                                                     (int*)n->yb);
            gather_rows<float><<<grid1(nb * n->n_out), NT, 0, st>>>(target, n->n_out, idx, nb, n->n_out, n->tb);
            cudaError_t e = backward(n, n->yb, y16, n->n_in, nb, n->tb, st);
            if (e != cudaSuccess) return done(pass_fail("gmf_mlp_train", e));
            const int rc = gmf_mlp_adam(n, lr, 0.9f, 0.999f, 1e-8f, stream);
            if (rc) return done(rc);
            loss_acc_kernel<<<1, 1, 0, st>>>(n->loss, (double)nb, d_acc + ep);
        }
        if (ep + 1 < epochs) shuffle();
    }
    std::vector<double> acc(epochs);
    if (cudaMemcpyAsync(acc.data(), d_acc, sizeof(double) * epochs, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return done(gmf_fail(GMF_ERR_CUDA, "gmf_mlp_train: loss read failed"));
    if (losses)
        for (int ep = 0; ep < epochs; ep++) losses[ep] = (float)(acc[ep] / (double)rows);
    if (n->err) {
        unsigned w = 0;
        if (cudaMemcpy(&w, n->err, sizeof w, cudaMemcpyDeviceToHost) == cudaSuccess && w)
            return done(gmf_fail(GMF_ERR_TIMEOUT, "gmf_mlp_train: a bounded wait in the tensor-core layer gave up"));
    }
    return done(GMF_OK);
}
