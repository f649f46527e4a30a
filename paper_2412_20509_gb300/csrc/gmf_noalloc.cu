// gmf_deviance_noalloc: the total-deviance kernel in a form that performs no
// device allocation, for callers that cannot call cudaMalloc -- for example a
// plug-in hosted by a framework that owns all device memory through its own
// pool, or a monitoring call that must not change the memory a running fit
// sees.
//
// Its per-tile partial sums live in the file-scope array below instead of in a
// handle's workspace. Every GPU that loads the library holds this array until
// the process exits.
#include <mutex>

#include "gmf_internal.cuh"
#include "gmf_update.cuh"

// One FP64 partial sum per 64 x 64 tile: at most 262144 tiles (2 MiB), i.e.
// ceil(n/64) * ceil(m/64) <= 262144 (for example 200000 x 5000).
#define GMF_NOALLOC_MAX_TILES 262144
static __device__ __align__(256) double g_noalloc_scratch[GMF_NOALLOC_MAX_TILES];

namespace {

constexpr int NT = 256;
constexpr int T = 64;
constexpr int LDS = T + 4;

// Unit deviance / 2w (Table S1; App. B for the negative binomial) in FP32:
// the shared ratio form for a positive count (no difference of two large
// logarithms), alpha log1p(mu/alpha) or mu for a zero count.
__device__ __forceinline__ float unit_dev(bool nb, float y, float e, float mu, float alpha) {
    if (y > 0.f) return gmfdev::half_dev_ratio(nb, y, e, mu, alpha);
    return nb ? alpha * log1pf(mu / alpha) : mu;
}

// One 64 x 64 tile: eta = L R' (FP32), unit deviances, compensated per-thread
// sums, FP32 block sum, written to part[tile] (every tile writes its slot).
__global__ void __launch_bounds__(NT) noalloc_tile_kernel(const void* Y, int y16, const float* W, int64_t n, int64_t m,
                                                          const float* L, const float* R, int K, int ld, int nb,
                                                          float alpha, float clamp, double* part) {
    __shared__ __align__(16) float Ls[64 * LDS];
    __shared__ __align__(16) float Rs[64 * LDS];
    __shared__ float red[NT / 32];
    const int tid = threadIdx.x;
    const int64_t row0 = (int64_t)blockIdx.y * T, col0 = (int64_t)blockIdx.x * T;
    const int nr = (int)min((int64_t)T, n - row0), nc = (int)min((int64_t)T, m - col0);
    for (int e = tid; e < T * K; e += NT) {
        const int i = e / K, c = e - i * K;
        Ls[c * LDS + i] = i < nr ? __ldg(L + (row0 + i) * ld + c) : 0.f;
        Rs[c * LDS + i] = i < nc ? __ldg(R + (col0 + i) * ld + c) : 0.f;
    }
    __syncthreads();
    const int tx = tid & 15, ty = tid >> 4;
    float acc[4][4] = {};
    for (int c = 0; c < K; c++) {
        const float4 lv = *(const float4*)(Ls + c * LDS + 4 * ty);
        const float4 rv = *(const float4*)(Rs + c * LDS + 4 * tx);
        const float l4[4] = {lv.x, lv.y, lv.z, lv.w}, r4[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
        for (int u = 0; u < 4; u++)
#pragma unroll
            for (int v = 0; v < 4; v++) acc[u][v] = fmaf(l4[u], r4[v], acc[u][v]);
    }
    float sum = 0.f, comp = 0.f;
#pragma unroll
    for (int u = 0; u < 4; u++) {
#pragma unroll
        for (int v = 0; v < 4; v++) {
            const int il = 4 * ty + u, jl = 4 * tx + v;
            if (il < nr && jl < nc) {
                const int64_t idx = (row0 + il) * m + col0 + jl;
                const float y = y16 ? (float)__ldg((const unsigned short*)Y + idx) : (float)__ldg((const int*)Y + idx);
                const float wv = W ? __ldg(W + idx) : 1.f;
                const float e = fminf(fmaxf(acc[u][v], -clamp), clamp);
                const float dv = 2.f * wv * unit_dev(nb != 0, y, e, expf(e), alpha);
                const float yk = dv - comp;
                const float tk = sum + yk;
                comp = (tk - sum) - yk;
                sum = tk;
            }
        }
    }
    const float s = gmfdev::block_sum_f<NT>(sum, red);
    if (tid == 0) part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = (double)s;
}

__global__ void noalloc_sum_kernel(const double* part, int count, double* out) {
    __shared__ double red[NT / 32];
    double s = 0.0;
    for (int c = threadIdx.x; c < count; c += NT) s += part[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int u = 0; u < NT / 32; u++) t += red[u];
        *out = t;
    }
}

// Device address of the scratch array, looked up once per device.
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double* g_scratch_ptr[MAX_DEVICES] = {};

int scratch_for_current_device(double** out, const char** why) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        *why = "no usable current CUDA device";
        return GMF_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            *why = cudaGetErrorString(e);
            return GMF_ERR_CUDA;
        }
        g_scratch_ptr[dev] = (double*)p;
    }
    *out = g_scratch_ptr[dev];
    return GMF_OK;
}

}  // namespace

int gmf_noalloc_fail(int code, const char* msg);  // gmf_api.cu: sets the thread's last-error text

extern "C" int gmf_deviance_noalloc(const void* Y, int32_t y_dtype, const float* W, int64_t n, int64_t m,
                                    const float* L, const float* R, int32_t K, int32_t ld, int32_t family,
                                    float alpha, float eta_clamp, double* d_out, void* stream) {
    if (!Y || !L || !R || !d_out) return gmf_noalloc_fail(GMF_ERR_ARG, "gmf_deviance_noalloc: NULL argument");
    if (n <= 0 || m <= 0) return gmf_noalloc_fail(GMF_ERR_ARG, "gmf_deviance_noalloc: n and m must be positive");
    if (y_dtype != GMF_Y_INT32 && y_dtype != GMF_Y_UINT16)
        return gmf_noalloc_fail(GMF_ERR_ARG, "gmf_deviance_noalloc: bad y_dtype");
    if (K < 1 || K > 64 || ld < K) return gmf_noalloc_fail(GMF_ERR_ARG, "gmf_deviance_noalloc: need 1 <= K <= 64, ld >= K");
    if (family != GMF_POISSON && family != GMF_NEGBIN)
        return gmf_noalloc_fail(GMF_ERR_ARG, "gmf_deviance_noalloc: unknown family");
    if (family == GMF_NEGBIN && !(alpha > 0.f))
        return gmf_noalloc_fail(GMF_ERR_ARG, "gmf_deviance_noalloc: alpha must be > 0");
    if (!(eta_clamp > 0.f)) return gmf_noalloc_fail(GMF_ERR_ARG, "gmf_deviance_noalloc: eta_clamp must be > 0");
    const int64_t tiles_x = (m + T - 1) / T, tiles_y = (n + T - 1) / T;
    if (tiles_x > 65535 || tiles_y > 65535 || tiles_x * tiles_y > GMF_NOALLOC_MAX_TILES)
        return gmf_noalloc_fail(GMF_ERR_ARG,
                                "gmf_deviance_noalloc: ceil(n/64) * ceil(m/64) exceeds the 262144-tile scratch limit");
    double* scratch = nullptr;
    const char* why = "";
    const int rc = scratch_for_current_device(&scratch, &why);
    if (rc != GMF_OK) return gmf_noalloc_fail(rc, why);
    cudaStream_t st = (cudaStream_t)stream;
    noalloc_tile_kernel<<<dim3((unsigned)tiles_x, (unsigned)tiles_y), NT, 0, st>>>(
        Y, y_dtype == GMF_Y_UINT16, W, n, m, L, R, K, ld, family == GMF_NEGBIN, alpha, eta_clamp, scratch);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        noalloc_sum_kernel<<<1, NT, 0, st>>>(scratch, (int)(tiles_x * tiles_y), d_out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return gmf_noalloc_fail(GMF_ERR_CUDA, cudaGetErrorString(e));
    return GMF_OK;
}
