// Out-of-sample metrics of a fit trained with held-out entries marked missing
// (Sec. 5.2): on the held-out set V,
//   Error    = sum_V [log1p(y) - log1p(mu)]^2 / sum_V [log1p(y) - log1p(ybar_T)]^2
//   Deviance = sum_V D(y, mu) / sum_V D(y, ybar_T)      (Poisson unit deviance, Table S1)
// with ybar_T the mean of the observed (training) counts. Two passes over 64 x
// 64 tiles of the handle's permuted count matrix: the first finds the missing
// entries, gathers their true counts from the caller's matrix (original order)
// and forms eta = L R' for them, and sums the observed counts; the second,
// once ybar_T is known, forms the denominators. FP32 terms, FP64 sums per
// thread and per CTA, combined on the host in CTA order.
#include <math.h>

#include <algorithm>
#include <vector>

#include "gmf_internal.cuh"

namespace {

constexpr int T = 64;
constexpr int NT = 256;
constexpr int LDT = T + 4;
constexpr int NPART = 5;

__device__ __forceinline__ float yval(const void* Y, int y16, int64_t idx) {
    return y16 ? (float)__ldg((const unsigned short*)Y + idx) : (float)__ldg((const int*)Y + idx);
}

// Poisson unit deviance 2 [y (log y - log mu) - (y - mu)], 0 log 0 = 0, with log mu given.
__device__ __forceinline__ float pois_dev(float y, float mu, float lmu) {
    return 2.f * ((y > 0.f ? y * (logf(y) - lmu) : 0.f) - (y - mu));
}

__device__ __forceinline__ double block_sum_d(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < NT / 32; u++) s += red[u];
    return s;
}

// pass 0: part = {sum of observed y, observed count, sum_V err(mu), sum_V D(y, mu), |V|}
// pass 1: part = {sum_V err(ybar), sum_V D(y, ybar), 0, 0, 0}
__global__ void __launch_bounds__(NT) holdout_kernel(StepArgs a, const void* Ytrue, const int* __restrict__ rperm,
                                                     const int* __restrict__ cperm, int pass, float ybar,
                                                     double* part) {
    __shared__ __align__(16) float Ls[GMF_KMAX * LDT];
    __shared__ __align__(16) float Rs[GMF_KMAX * LDT];
    __shared__ double red[NT / 32];
    const int tid = threadIdx.x;
    const int64_t tiles_c = (a.m + T - 1) / T, tiles = ((a.n + T - 1) / T) * tiles_c;
    const float lybar = logf(ybar), l1ybar = log1pf(ybar);
    double acc[NPART] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t row0 = (tile / tiles_c) * T, col0 = (tile % tiles_c) * T;
        const int nr = (int)min((int64_t)T, a.n - row0), nc = (int)min((int64_t)T, a.m - col0);
        if (pass == 0) {
            __syncthreads();  // the previous tile's factors are no longer read
            for (int e = tid; e < T * a.K; e += NT) {
                const int i = e / a.K, c = e - i * a.K;
                Ls[c * LDT + i] = i < nr ? a.L[(row0 + i) * a.KP + c] : 0.f;
                Rs[c * LDT + i] = i < nc ? a.R[(col0 + i) * a.KP + c] : 0.f;
            }
            __syncthreads();
        }
        for (int e = tid; e < T * T; e += NT) {
            const int i = e / T, j = e - i * T;
            if (i >= nr || j >= nc) continue;
            const float yp = yval(a.Y, a.y16, (row0 + i) * a.m + col0 + j);
            if (yp != a.ymiss) {
                if (pass == 0) {
                    acc[0] += (double)yp;
                    acc[1] += 1.0;
                }
                continue;
            }
            const float y = yval(Ytrue, a.y16, (int64_t)rperm[row0 + i] * a.m + cperm[col0 + j]);
            const float ly1 = log1pf(y);
            if (pass == 0) {
                float eta = 0.f;
                for (int c = 0; c < a.K; c++) eta = fmaf(Ls[c * LDT + i], Rs[c * LDT + j], eta);
                const float e2 = fminf(fmaxf(eta, -a.clamp), a.clamp);
                const float mu = expf(e2);
                const float d = ly1 - log1pf(mu);
                acc[2] += (double)(d * d);
                acc[3] += (double)pois_dev(y, mu, e2);
                acc[4] += 1.0;
            } else {
                const float d = ly1 - l1ybar;
                acc[0] += (double)(d * d);
                acc[1] += (double)pois_dev(y, ybar, lybar);
            }
        }
    }
    for (int k = 0; k < NPART; k++) {
        const double s = block_sum_d(acc[k], red);
        if (tid == 0) part[(int64_t)blockIdx.x * NPART + k] = s;
    }
}

// Log-likelihood and Pearson statistic of the observed entries at the current
// parameters: part = {sum w log f(y; mu), sum w (y - mu)^2 / nu(mu), observed
// entries, 0, 0} per CTA. log f of Table S1's families with the log link:
//   Poisson  y eta - mu - lgamma(y + 1)
//   NB       lgamma(y + a) - lgamma(a) - lgamma(y + 1) + a (log a - log(a + mu)) + y (eta - log(a + mu))
// with nu(mu) = mu and mu (1 + mu / a).
__global__ void __launch_bounds__(NT) loglik_kernel(StepArgs a, double* part) {
    __shared__ __align__(16) float Ls[GMF_KMAX * LDT];
    __shared__ __align__(16) float Rs[GMF_KMAX * LDT];
    __shared__ double red[NT / 32];
    const int tid = threadIdx.x;
    const bool nb = a.family == GMF_NEGBIN;
    const float alpha = *a.alpha;
    const float la = logf(alpha), lga = lgammaf(alpha);
    const int64_t tiles_c = (a.m + T - 1) / T, tiles = ((a.n + T - 1) / T) * tiles_c;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t row0 = (tile / tiles_c) * T, col0 = (tile % tiles_c) * T;
        const int nr = (int)min((int64_t)T, a.n - row0), nc = (int)min((int64_t)T, a.m - col0);
        __syncthreads();
        for (int e = tid; e < T * a.K; e += NT) {
            const int i = e / a.K, c = e - i * a.K;
            Ls[c * LDT + i] = i < nr ? a.L[(row0 + i) * a.KP + c] : 0.f;
            Rs[c * LDT + i] = i < nc ? a.R[(col0 + i) * a.KP + c] : 0.f;
        }
        __syncthreads();
        for (int e = tid; e < T * T; e += NT) {
            const int i = e / T, j = e - i * T;
            if (i >= nr || j >= nc) continue;
            const int64_t idx = (row0 + i) * a.m + col0 + j;
            const float y = yval(a.Y, a.y16, idx);
            if (a.missing && y == a.ymiss) continue;
            const float w = a.W ? __ldg(a.W + idx) : 1.f;
            float eta = 0.f;
            for (int c = 0; c < a.K; c++) eta = fmaf(Ls[c * LDT + i], Rs[c * LDT + j], eta);
            const float ec = fminf(fmaxf(eta, -a.clamp), a.clamp);
            const float mu = expf(ec);
            float lf, nu;
            if (nb) {
                const bool pg = a.alpha_col != nullptr;   // per-gene shapes
                const float aj = pg ? __ldg(a.alpha_col + col0 + j) : alpha;
                const float laj = pg ? logf(aj) : la, lgaj = pg ? lgammaf(aj) : lga;
                const float lam = laj + log1pf(mu / aj);   // log(alpha + mu)
                lf = lgammaf(y + aj) - lgaj - lgammaf(y + 1.f) + aj * (laj - lam) + y * (ec - lam);
                nu = mu * (1.f + mu / aj);
            } else {
                lf = y * ec - mu - lgammaf(y + 1.f);
                nu = mu;
            }
            acc[0] += (double)(w * lf);
            acc[1] += (double)(w * (y - mu) * (y - mu) / nu);
            acc[2] += 1.0;
        }
    }
    for (int k = 0; k < 3; k++) {
        const double s = block_sum_d(acc[k], red);
        if (tid == 0) part[(int64_t)blockIdx.x * 3 + k] = s;
    }
}

// Per-gene moment sums of App. B's shape estimator at the current parameters:
// part[ry][j] = {sum_i w mu^2, sum_i w ((y - mu)^2 - mu)} over the observed
// entries of the row tiles ry, ry + gridDim.y, ... of column tile blockIdx.x.
// Thread t always owns column t % 64 of the tile, so its sums need no atomics.
__global__ void __launch_bounds__(NT) gene_moments_kernel(StepArgs a, double* part) {
    __shared__ __align__(16) float Ls[GMF_KMAX * LDT];
    __shared__ __align__(16) float Rs[GMF_KMAX * LDT];
    __shared__ double red[NT][2];
    const int tid = threadIdx.x;
    const int64_t col0 = (int64_t)blockIdx.x * T;
    const int nc = (int)min((int64_t)T, a.m - col0);
    const int64_t tiles_r = (a.n + T - 1) / T;
    const int j = tid % T;
    double s1 = 0.0, s2 = 0.0;
    for (int e = tid; e < T * a.K; e += NT) {
        const int i = e / a.K, c = e - i * a.K;
        Rs[c * LDT + i] = i < nc ? a.R[(col0 + i) * a.KP + c] : 0.f;
    }
    for (int64_t rt = blockIdx.y; rt < tiles_r; rt += gridDim.y) {
        const int64_t row0 = rt * T;
        const int nr = (int)min((int64_t)T, a.n - row0);
        __syncthreads();
        for (int e = tid; e < T * a.K; e += NT) {
            const int i = e / a.K, c = e - i * a.K;
            Ls[c * LDT + i] = i < nr ? a.L[(row0 + i) * a.KP + c] : 0.f;
        }
        __syncthreads();
        if (j < nc) {
            for (int i = tid / T; i < nr; i += NT / T) {
                const int64_t idx = (row0 + i) * a.m + col0 + j;
                const float y = yval(a.Y, a.y16, idx);
                if (a.missing && y == a.ymiss) continue;
                const float w = a.W ? __ldg(a.W + idx) : 1.f;
                float eta = 0.f;
                for (int c = 0; c < a.K; c++) eta = fmaf(Ls[c * LDT + i], Rs[c * LDT + j], eta);
                const float mu = expf(fminf(fmaxf(eta, -a.clamp), a.clamp));
                s1 += (double)(w * mu * mu);
                s2 += (double)(w * ((y - mu) * (y - mu) - mu));
            }
        }
    }
    red[tid][0] = s1;
    red[tid][1] = s2;
    __syncthreads();
    if (tid < T && tid < nc) {
        double t1 = 0.0, t2 = 0.0;
        for (int u = tid; u < NT; u += T) {
            t1 += red[u][0];
            t2 += red[u][1];
        }
        part[((int64_t)blockIdx.y * a.m + col0 + tid) * 2] = t1;
        part[((int64_t)blockIdx.y * a.m + col0 + tid) * 2 + 1] = t2;
    }
}

// ---- maximum-likelihood NB shape per gene (App. B's likelihood, one gene's
// shape alpha with the fit's means held fixed). With l(alpha) the NB
// log-likelihood of the gene's observed entries, Newton's method in
// theta = log alpha needs per gene
//   l'  = sum_i w [psi(y + a) - psi(a) - log1p(mu / a) + (mu - y) / (a + mu)]
//   l'' = sum_i w [psi'(y + a) - psi'(a) + mu / (a (a + mu)) + (y - mu) / (a + mu)^2].
// The digamma and trigamma differences are sums of 1 / (a + k) and -1 / (a + k)^2
// over k < y (psi(x + 1) = psi(x) + 1 / x); from k = 16 on, for y > 16, the
// shifted differences psi(y + a) - psi(a + 16) come from the asymptotic series
// of psi and psi' (Abramowitz and Stegun 6.3.18 and 6.4.12), whose arguments
// are then at least 16. Terms in FP32, compensated (Kahan) FP32 sums per thread.
constexpr int ML_DIRECT = 16;

__device__ __forceinline__ float psi_asym(float x) {  // x >= 16: ln x - 1/(2x) - 1/(12x^2) + 1/(120x^4) - 1/(252x^6)
    const float r = 1.f / x, r2 = r * r;
    return logf(x) - 0.5f * r - r2 * (1.f / 12.f - r2 * (1.f / 120.f - r2 * (1.f / 252.f)));
}
__device__ __forceinline__ float psi1_asym(float x) {  // x >= 16: 1/x + 1/(2x^2) + 1/(6x^3) - 1/(30x^5) + 1/(42x^7)
    const float r = 1.f / x, r2 = r * r;
    return r + 0.5f * r2 + r * r2 * (1.f / 6.f - r2 * (1.f / 30.f - r2 * (1.f / 42.f)));
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
    const float yv = v - c;
    const float t = s + yv;
    c = (t - s) - yv;
    s = t;
}

// part[ry][j] = {l'_j, l''_j} over the observed entries of row tiles ry, ry + gridDim.y, ... of column tile
// blockIdx.x; alpha: the current shape of each (permuted) gene.
__global__ void __launch_bounds__(NT) gene_ml_kernel(StepArgs a, const float* __restrict__ alpha, double* part) {
    __shared__ __align__(16) float Ls[GMF_KMAX * LDT];
    __shared__ __align__(16) float Rs[GMF_KMAX * LDT];
    __shared__ double red[NT][2];
    const int tid = threadIdx.x;
    const int64_t col0 = (int64_t)blockIdx.x * T;
    const int nc = (int)min((int64_t)T, a.m - col0);
    const int64_t tiles_r = (a.n + T - 1) / T;
    const int j = tid % T;
    const float aj = j < nc ? __ldg(alpha + col0 + j) : 1.f;
    float s1 = 0.f, c1 = 0.f, s2 = 0.f, c2 = 0.f;
    for (int e = tid; e < T * a.K; e += NT) {
        const int i = e / a.K, c = e - i * a.K;
        Rs[c * LDT + i] = i < nc ? a.R[(col0 + i) * a.KP + c] : 0.f;
    }
    for (int64_t rt = blockIdx.y; rt < tiles_r; rt += gridDim.y) {
        const int64_t row0 = rt * T;
        const int nr = (int)min((int64_t)T, a.n - row0);
        __syncthreads();
        for (int e = tid; e < T * a.K; e += NT) {
            const int i = e / a.K, c = e - i * a.K;
            Ls[c * LDT + i] = i < nr ? a.L[(row0 + i) * a.KP + c] : 0.f;
        }
        __syncthreads();
        if (j < nc) {
            for (int i = tid / T; i < nr; i += NT / T) {
                const int64_t idx = (row0 + i) * a.m + col0 + j;
                const float y = yval(a.Y, a.y16, idx);
                if (a.missing && y == a.ymiss) continue;
                const float w = a.W ? __ldg(a.W + idx) : 1.f;
                float eta = 0.f;
                for (int c = 0; c < a.K; c++) eta = fmaf(Ls[c * LDT + i], Rs[c * LDT + j], eta);
                const float mu = expf(fminf(fmaxf(eta, -a.clamp), a.clamp));
                const int yi = (int)y;
                const int kd = min(yi, ML_DIRECT);
                float d1 = 0.f, d2 = 0.f;
                for (int k = 0; k < kd; k++) {
                    const float r = 1.f / (aj + (float)k);
                    d1 += r;
                    d2 -= r * r;
                }
                if (yi > ML_DIRECT) {
                    d1 += psi_asym(y + aj) - psi_asym(aj + (float)ML_DIRECT);
                    d2 += psi1_asym(y + aj) - psi1_asym(aj + (float)ML_DIRECT);
                }
                const float am = aj + mu;
                const float g = d1 - log1pf(mu / aj) + (mu - y) / am;
                const float hh = d2 + mu / (aj * am) + (y - mu) / (am * am);
                kahan_add(s1, c1, w * g);
                kahan_add(s2, c2, w * hh);
            }
        }
    }
    red[tid][0] = (double)s1;
    red[tid][1] = (double)s2;
    __syncthreads();
    if (tid < T && tid < nc) {
        double t1 = 0.0, t2 = 0.0;
        for (int u = tid; u < NT; u += T) {
            t1 += red[u][0];
            t2 += red[u][1];
        }
        part[((int64_t)blockIdx.y * a.m + col0 + tid) * 2] = t1;
        part[((int64_t)blockIdx.y * a.m + col0 + tid) * 2 + 1] = t2;
    }
}

}  // namespace

int gmf_gene_moments_run(gmf_model* h, double* sums, cudaStream_t st, const char** why) {
    StepArgs a = gmf_make_args(h);
    const int RY = 16;
    double* part = nullptr;
    if (cudaMallocAsync((void**)&part, sizeof(double) * 2 * RY * (size_t)h->m, st) != cudaSuccess) {
        *why = "device allocation of the partial sums failed";
        return GMF_ERR_OOM;
    }
    std::vector<double> hp((size_t)2 * RY * h->m);
    gene_moments_kernel<<<dim3((unsigned)((h->m + T - 1) / T), RY), NT, 0, st>>>(a, part);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(part, st);
    if (e != cudaSuccess) {
        *why = cudaGetErrorString(e);
        return GMF_ERR_CUDA;
    }
    for (int64_t j = 0; j < h->m; j++) {
        double t1 = 0.0, t2 = 0.0;
        for (int r = 0; r < RY; r++) {
            t1 += hp[((size_t)r * h->m + j) * 2];
            t2 += hp[((size_t)r * h->m + j) * 2 + 1];
        }
        sums[2 * j] = t1;
        sums[2 * j + 1] = t2;
    }
    return GMF_OK;
}

int gmf_loglik_run(gmf_model* h, double* out, cudaStream_t st, const char** why) {
    StepArgs a = gmf_make_args(h);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::max(1, sms) * 4;
    double* part = nullptr;
    if (cudaMallocAsync((void**)&part, sizeof(double) * 3 * grid, st) != cudaSuccess) {
        *why = "device allocation of the partial sums failed";
        return GMF_ERR_OOM;
    }
    std::vector<double> hp((size_t)3 * grid);
    loglik_kernel<<<grid, NT, 0, st>>>(a, part);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(part, st);
    if (e != cudaSuccess) {
        *why = cudaGetErrorString(e);
        return GMF_ERR_CUDA;
    }
    out[0] = out[1] = out[2] = 0.0;
    for (int b = 0; b < grid; b++)
        for (int k = 0; k < 3; k++) out[k] += hp[(size_t)b * 3 + k];
    return GMF_OK;
}

int gmf_holdout_run(gmf_model* h, const void* Ytrue, double* out, cudaStream_t st, const char** why) {
    StepArgs a = gmf_make_args(h);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::max(1, sms) * 4;
    double* part = nullptr;
    if (cudaMallocAsync((void**)&part, sizeof(double) * NPART * grid, st) != cudaSuccess) {
        *why = "device allocation of the partial sums failed";
        return GMF_ERR_OOM;
    }
    std::vector<double> hp((size_t)NPART * grid);
    double tot[2][NPART] = {};
    for (int pass = 0; pass < 2; pass++) {
        const float ybar = pass == 0 ? 1.f : (float)(tot[0][0] / tot[0][1]);
        holdout_kernel<<<grid, NT, 0, st>>>(a, Ytrue, h->rperm, h->cperm, pass, ybar, part);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            cudaFreeAsync(part, st);
            *why = cudaGetErrorString(e);
            return GMF_ERR_CUDA;
        }
        for (int b = 0; b < grid; b++)
            for (int k = 0; k < NPART; k++) tot[pass][k] += hp[(size_t)b * NPART + k];
        if (pass == 0 && (tot[0][1] == 0.0 || tot[0][4] == 0.0)) {
            cudaFreeAsync(part, st);
            *why = tot[0][4] == 0.0 ? "no entry of the counts is marked missing" : "no entry is observed";
            return GMF_ERR_STATE;
        }
    }
    cudaFreeAsync(part, st);
    out[0] = tot[0][2] / tot[1][0];
    out[1] = tot[0][3] / tot[1][1];
    out[2] = tot[0][0] / tot[0][1];
    out[3] = tot[0][4];
    return GMF_OK;
}

// Newton's method in theta = log alpha for every gene at once: per iteration
// one pass of gene_ml_kernel (FP64 sums over the row-tile partials in order),
// then per gene dtheta = -g / h with g = a l', h = a l' + a^2 l'' where h < 0,
// else a step of +-1 in the direction of g; steps capped at 1 in theta, theta
// kept in [log lo, log hi]. alpha (permuted order, FP64) holds the start and
// receives the estimate; iters_done the passes made.
int gmf_gene_ml_run(gmf_model* h, double* alpha, int iters, double tol, double lo, double hi, int* iters_done,
                    cudaStream_t st, const char** why) {
    StepArgs a = gmf_make_args(h);
    const int RY = 16;
    const size_t m = (size_t)h->m;
    double* part = nullptr;
    float* ad = nullptr;
    if (cudaMallocAsync((void**)&part, sizeof(double) * 2 * RY * m, st) != cudaSuccess ||
        cudaMallocAsync((void**)&ad, sizeof(float) * m, st) != cudaSuccess) {
        if (part) cudaFreeAsync(part, st);
        *why = "device allocation of the per-gene sums failed";
        return GMF_ERR_OOM;
    }
    std::vector<double> hp(2 * RY * m);
    std::vector<float> af(m);
    std::vector<char> done(m, 0);
    const double tlo = log(lo), thi = log(hi);
    cudaError_t e = cudaSuccess;
    int it = 0;
    for (; it < iters; it++) {
        for (size_t jp = 0; jp < m; jp++) af[jp] = (float)alpha[jp];
        e = cudaMemcpyAsync(ad, af.data(), sizeof(float) * m, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) break;
        gene_ml_kernel<<<dim3((unsigned)((h->m + T - 1) / T), RY), NT, 0, st>>>(a, ad, part);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) break;
        bool all = true;
        for (size_t jp = 0; jp < m; jp++) {
            if (done[jp]) continue;
            double g1 = 0.0, g2 = 0.0;
            for (int r = 0; r < RY; r++) {
                g1 += hp[((size_t)r * m + jp) * 2];
                g2 += hp[((size_t)r * m + jp) * 2 + 1];
            }
            const double al = alpha[jp], th = log(al);
            const double g = al * g1, hs = al * g1 + al * al * g2;
            double step = hs < 0.0 ? -g / hs : (g > 0.0 ? 1.0 : g < 0.0 ? -1.0 : 0.0);
            step = std::min(1.0, std::max(-1.0, step));
            const double tn = std::min(thi, std::max(tlo, th + step));
            alpha[jp] = exp(tn);
            if (fabs(tn - th) <= tol) done[jp] = 1;
            else all = false;
        }
        if (all) {
            it++;
            break;
        }
    }
    cudaFreeAsync(part, st);
    cudaFreeAsync(ad, st);
    if (e != cudaSuccess) {
        *why = cudaGetErrorString(e);
        return GMF_ERR_CUDA;
    }
    *iters_done = it;
    return GMF_OK;
}
