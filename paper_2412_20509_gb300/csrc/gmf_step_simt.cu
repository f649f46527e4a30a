// FP32 CUDA-core path of the block step (Algorithm 1, eq. 15 / App. B,
// eq. 12, eq. 14) and the full deviance (Table S1, App. B).
//
// One launch per sweep. Grid (TJ, TI, per): CTA (tj, ti, k) owns a 64 x 64
// tile of block k of the sweep. Per tile:
//   1. the L and R rows of the tile go to shared memory (transposed);
//   2. each thread forms a 4 x 4 micro-tile of eta = L R' in FP32, then
//      mu = exp(eta), Ddot, Dddot (Sec. 3, log link) -> shared memory;
//   3. row partials sum_j Ddot_ij R_jc, sum_j Dddot_ij R_jc^2 (c row-free) and
//      column partials sum_i Ddot_ij L_ic, sum_i Dddot_ij L_ic^2 (c column-free)
//      are written to a workspace, one slot per tile (fixed order, no atomics
//      on values);
//   4. an arrival counter per row strip and per column strip elects the last
//      CTA of the strip, which sums that strip's partials in tile order and
//      applies the scale factor, penalty, damping, EMA and step to its rows
//      (columns). Every reader of those parameters in this sweep has arrived,
//      so the update cannot race with a reader; no CTA waits on another.
// The NB shape is updated once per sweep by the last CTA of the launch from
// per-CTA moment sums (FP64) reduced in CTA order.
#include <math.h>

#include "gmf_internal.cuh"

namespace {

constexpr int T = GMF_TILE;
constexpr int LD = T + 4;   // leading dimension of the transposed factor tiles
constexpr int LDD = T + 1;  // leading dimension of the Ddot / Dddot tiles (odd)
constexpr int NW = GMF_THREADS / 32;

struct BlockGeo {
    int64_t r0, nI, c0, mJ;
};

__device__ __forceinline__ BlockGeo block_geo(const StepArgs& a, int w, int k) {
    const int sg = a.sigma[w];
    int rc, cc;
    if (!a.swap) {
        rc = (sg + k) % a.r;
        cc = k;
    } else {
        rc = k;
        cc = (sg + k) % a.s;
    }
    BlockGeo g;
    g.r0 = (int64_t)rc * a.nb_row;
    g.nI = min((int64_t)a.nb_row, a.n - g.r0);
    g.c0 = (int64_t)cc * a.nb_col;
    g.mJ = min((int64_t)a.nb_col, a.m - g.c0);
    return g;
}

__device__ __forceinline__ float load_y(const void* Y, int y16, int64_t idx) {
    return y16 ? (float)__ldg((const unsigned short*)Y + idx) : (float)__ldg((const int*)Y + idx);
}

// L (or R) rows [row0, row0+nr) -> S[c*LD + i], zero-filled to T rows.
__device__ __forceinline__ void load_factor_tile(float* S, const float* F, int K, int64_t row0, int nr) {
    for (int e = threadIdx.x; e < T * K; e += GMF_THREADS) {
        const int i = e / K, c = e - i * K;
        S[c * LD + i] = i < nr ? F[(row0 + i) * K + c] : 0.f;
    }
}

// 4 x 4 micro-tile of eta: rows ty + 16a, columns tx + 16b.
__device__ __forceinline__ void eta_microtile(const float* Ls, const float* Rs, int K, int tx, int ty,
                                              float acc[4][4]) {
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) acc[a][b] = 0.f;
    for (int c = 0; c < K; c++) {
        float lv[4], rv[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            lv[u] = Ls[c * LD + ty + 16 * u];
            rv[u] = Rs[c * LD + tx + 16 * u];
        }
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int b = 0; b < 4; b++) acc[a][b] = fmaf(lv[a], rv[b], acc[a][b]);
    }
}

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    for (int u = 0; u < NW; u++) s += red[u];  // fixed order, every thread the same value
    return s;
}

__device__ __forceinline__ double bias_factor(int mode, double a1, double a2, long long t, int visits) {
    if (mode == 0) return (1.0 - pow(a2, (double)t)) / (1.0 - pow(a1, (double)t));
    return (1.0 - pow(1.0 - a2, (double)visits)) / (1.0 - pow(1.0 - a1, (double)visits));
}

// Smoothed local step of eq. 12 / eq. 14 for one free parameter.
__device__ __forceinline__ void smoothed_step(float* theta, float* gbar, float* hbar, float gsum, float hsum,
                                              float scale, float lam, const StepArgs& a, float rho_c,
                                              unsigned* err) {
    const float th = *theta;
    const float gh = -scale * gsum + lam * th;
    const float hh = scale * hsum + lam + a.damping;
    const float gb = (1.f - a.a1) * (*gbar) + a.a1 * gh;
    const float hb = (1.f - a.a2) * (*hbar) + a.a2 * hh;
    const float nt = th - rho_c * (gb / hb);
    *gbar = gb;
    *hbar = hb;
    *theta = nt;
    if (!isfinite(nt)) atomicOr(err, GMF_DEVERR_NONFINITE);
}

__global__ void __launch_bounds__(GMF_THREADS) sweep_kernel(StepArgs a, int w, long long t0) {
    extern __shared__ float smem[];
    float* Ls = smem;
    float* Rs = Ls + a.K * LD;
    float* Ds = Rs + a.K * LD;
    float* DDs = Ds + T * LDD;
    __shared__ double red[NW];
    __shared__ int s_flag[3];
    __shared__ int s_visits[T];
    __shared__ float s_rc[T];

    const int tid = threadIdx.x;
    const int tj = blockIdx.x, ti = blockIdx.y, k = blockIdx.z;
    const BlockGeo g = block_geo(a, w, k);
    const int nTI = (int)((g.nI + T - 1) / T), nTJ = (int)((g.mJ + T - 1) / T);
    const bool active = ti < nTI && tj < nTJ;
    const bool nb = a.family == GMF_NEGBIN;
    const bool moments = nb && a.alpha_mode == 1;
    const float alpha = *a.alpha;
    const long long t = t0 + (long long)w * a.per + k + 1;
    double s1 = 0.0, s2 = 0.0;

    const int64_t row0 = g.r0 + (int64_t)ti * T, col0 = g.c0 + (int64_t)tj * T;
    const int nr = active ? (int)min((int64_t)T, g.nI - (int64_t)ti * T) : 0;
    const int nc = active ? (int)min((int64_t)T, g.mJ - (int64_t)tj * T) : 0;

    if (active) {
        load_factor_tile(Ls, a.L, a.K, row0, nr);
        load_factor_tile(Rs, a.R, a.K, col0, nc);
        __syncthreads();
        const int tx = tid & 15, ty = tid >> 4;
        float acc[4][4];
        eta_microtile(Ls, Rs, a.K, tx, ty, acc);
#pragma unroll
        for (int u = 0; u < 4; u++) {
#pragma unroll
            for (int v = 0; v < 4; v++) {
                const int il = ty + 16 * u, jl = tx + 16 * v;
                float dd = 0.f, ddd = 0.f;
                if (il < nr && jl < nc) {
                    const int64_t idx = (row0 + il) * a.m + col0 + jl;
                    const float y = load_y(a.Y, a.y16, idx);
                    const float wv = a.W ? __ldg(a.W + idx) : 1.f;
                    const float e = fminf(fmaxf(acc[u][v], -a.clamp), a.clamp);
                    const float mu = expf(e);
                    if (nb) {
                        const float f = alpha / (alpha + mu);
                        dd = wv * (y - mu) * f;
                        ddd = wv * mu * f;
                    } else {
                        dd = wv * (y - mu);
                        ddd = wv * mu;
                    }
                    if (moments) {
                        s1 += (double)(wv * mu * mu);
                        s2 += (double)(wv * ((y - mu) * (y - mu) - mu));
                    }
                }
                Ds[il * LDD + jl] = dd;
                DDs[il * LDD + jl] = ddd;
            }
        }
        __syncthreads();
        // Row partials: thread (il, cg) handles row-free columns c = cg, cg+4, ...
        {
            const int il = tid & (T - 1), cg = tid >> 6;
            const int cR = 1 + a.p;
            float gacc[GMF_FREE_MAX / 4], hacc[GMF_FREE_MAX / 4];
#pragma unroll
            for (int u = 0; u < GMF_FREE_MAX / 4; u++) gacc[u] = hacc[u] = 0.f;
            for (int j = 0; j < nc; j++) {
                const float dv = Ds[il * LDD + j], ddv = DDs[il * LDD + j];
#pragma unroll
                for (int u = 0; u < GMF_FREE_MAX / 4; u++) {
                    const int c = cg + 4 * u;
                    if (c < a.fr) {
                        const float rv = Rs[(cR + c) * LD + j];
                        gacc[u] = fmaf(dv, rv, gacc[u]);
                        hacc[u] = fmaf(ddv, rv * rv, hacc[u]);
                    }
                }
            }
            if (il < nr) {
                float* dst = a.partR + ((size_t)(k * a.TJ + tj) * T + il) * 2 * a.fr;
#pragma unroll
                for (int u = 0; u < GMF_FREE_MAX / 4; u++) {
                    const int c = cg + 4 * u;
                    if (c < a.fr) {
                        dst[c] = gacc[u];
                        dst[a.fr + c] = hacc[u];
                    }
                }
            }
        }
        // Column partials: thread (jl, cg) handles column-free columns c = cg, cg+4, ...
        {
            const int jl = tid & (T - 1), cg = tid >> 6;
            float gacc[GMF_FREE_MAX / 4], hacc[GMF_FREE_MAX / 4];
#pragma unroll
            for (int u = 0; u < GMF_FREE_MAX / 4; u++) gacc[u] = hacc[u] = 0.f;
            for (int i = 0; i < nr; i++) {
                const float dv = Ds[i * LDD + jl], ddv = DDs[i * LDD + jl];
#pragma unroll
                for (int u = 0; u < GMF_FREE_MAX / 4; u++) {
                    const int c = cg + 4 * u;
                    if (c < a.fc) {
                        const int lc = c < a.p ? 1 + c : 1 + a.q + c;
                        const float lv = Ls[lc * LD + i];
                        gacc[u] = fmaf(dv, lv, gacc[u]);
                        hacc[u] = fmaf(ddv, lv * lv, hacc[u]);
                    }
                }
            }
            if (jl < nc) {
                float* dst = a.partC + ((size_t)(k * a.TI + ti) * T + jl) * 2 * a.fc;
#pragma unroll
                for (int u = 0; u < GMF_FREE_MAX / 4; u++) {
                    const int c = cg + 4 * u;
                    if (c < a.fc) {
                        dst[c] = gacc[u];
                        dst[a.fc + c] = hacc[u];
                    }
                }
            }
        }
    }

    // ---- arrivals: elect the last CTA of each row strip and column strip
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        s_flag[0] = s_flag[1] = 0;
        if (active) {
            unsigned prev = atomicAdd(&a.ctrR[k * a.TI + ti], 1u);
            s_flag[0] = prev == (unsigned)(nTJ - 1);
            prev = atomicAdd(&a.ctrC[k * a.TJ + tj], 1u);
            s_flag[1] = prev == (unsigned)(nTI - 1);
        }
    }
    __syncthreads();
    const double rho = a.k0 / pow(1.0 + a.k0 * a.k1 * (double)t, a.tau);

    if (s_flag[0]) {  // this CTA updates rows [row0, row0 + nr) of block k
        __threadfence();
        if (tid < nr) {
            const int v = a.cntR[row0 + tid] + 1;
            s_visits[tid] = v;
            s_rc[tid] = (float)(rho * bias_factor(a.bias_corr, a.a1, a.a2, t, v));
        }
        __syncthreads();
        const float scale = (float)((double)a.m / (double)g.mJ);
        for (int e = tid; e < nr * a.fr; e += GMF_THREADS) {
            const int il = e / a.fr, c = e - il * a.fr;
            float sg = 0.f, sh = 0.f;
            for (int u = 0; u < nTJ; u++) {
                const float* src = a.partR + ((size_t)(k * a.TJ + u) * T + il) * 2 * a.fr;
                sg += __ldcg(src + c);
                sh += __ldcg(src + a.fr + c);
            }
            const int64_t row = row0 + il;
            const float lam = c < a.q ? a.lam[1] : a.lam[2];
            smoothed_step(a.L + row * a.K + 1 + a.p + c, a.GbR + row * a.fr + c, a.HbR + row * a.fr + c, sg, sh,
                          scale, lam, a, s_rc[il], a.err);
        }
        __syncthreads();
        if (tid < nr) a.cntR[row0 + tid] = s_visits[tid];
        if (tid == 0) a.ctrR[k * a.TI + ti] = 0u;
    }
    if (s_flag[1]) {  // this CTA updates columns [col0, col0 + nc) of block k
        __threadfence();
        __syncthreads();
        if (tid < nc) {
            const int v = a.cntC[col0 + tid] + 1;
            s_visits[tid] = v;
            s_rc[tid] = (float)(rho * bias_factor(a.bias_corr, a.a1, a.a2, t, v));
        }
        __syncthreads();
        const float scale = (float)((double)a.n / (double)g.nI);
        for (int e = tid; e < nc * a.fc; e += GMF_THREADS) {
            const int jl = e / a.fc, c = e - jl * a.fc;
            float sg = 0.f, sh = 0.f;
            for (int u = 0; u < nTI; u++) {
                const float* src = a.partC + ((size_t)(k * a.TI + u) * T + jl) * 2 * a.fc;
                sg += __ldcg(src + c);
                sh += __ldcg(src + a.fc + c);
            }
            const int64_t col = col0 + jl;
            const int rcol = c < a.p ? 1 + c : 1 + a.q + c;
            const float lam = c < a.p ? a.lam[0] : a.lam[3];
            smoothed_step(a.R + col * a.K + rcol, a.GbC + col * a.fc + c, a.HbC + col * a.fc + c, sg, sh, scale,
                          lam, a, s_rc[jl], a.err);
        }
        __syncthreads();
        if (tid < nc) a.cntC[col0 + tid] = s_visits[tid];
        if (tid == 0) a.ctrC[k * a.TJ + tj] = 0u;
    }

    // ---- NB shape: moment sums pooled over the sweep, one update per sweep (App. B)
    if (moments) {
        const double S1 = block_sum(s1, red);
        const double S2 = block_sum(s2, red);
        const int cta = (k * a.TI + ti) * a.TJ + tj;
        if (tid == 0) {
            a.nbpart[2 * cta] = S1;
            a.nbpart[2 * cta + 1] = S2;
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            const unsigned total = gridDim.x * gridDim.y * gridDim.z;
            s_flag[2] = atomicAdd(a.ctrSweep, 1u) == total - 1;
        }
        __syncthreads();
        if (s_flag[2] && tid == 0) {
            __threadfence();
            const int total = gridDim.x * gridDim.y * gridDim.z;
            double T1 = 0.0, T2 = 0.0;
            for (int c = 0; c < total; c++) {
                T1 += __ldcg(a.nbpart + 2 * c);
                T2 += __ldcg(a.nbpart + 2 * c + 1);
            }
            if (T2 > 0.0) {
                double ahat = T1 / T2;
                if (ahat < (double)a.eps) ahat = (double)a.eps;
                const long long tf = t0 + (long long)w * a.per + 1;
                const double rf = a.k0 / pow(1.0 + a.k0 * a.k1 * (double)tf, a.tau);
                *a.alpha = (float)((1.0 - rf) * (double)alpha + rf * ahat);
            }
            *a.ctrSweep = 0u;
        }
    }
}

// Deviance of one 64 x 64 tile of the whole (permuted) matrix.
__global__ void __launch_bounds__(GMF_THREADS) deviance_kernel(StepArgs a, double* part) {
    extern __shared__ float smem[];
    float* Ls = smem;
    float* Rs = Ls + a.K * LD;
    __shared__ double red[NW];
    const int tid = threadIdx.x;
    const int64_t row0 = (int64_t)blockIdx.y * T, col0 = (int64_t)blockIdx.x * T;
    const int nr = (int)min((int64_t)T, a.n - row0), nc = (int)min((int64_t)T, a.m - col0);
    load_factor_tile(Ls, a.L, a.K, row0, nr);
    load_factor_tile(Rs, a.R, a.K, col0, nc);
    __syncthreads();
    const int tx = tid & 15, ty = tid >> 4;
    float acc[4][4];
    eta_microtile(Ls, Rs, a.K, tx, ty, acc);
    const float alpha = *a.alpha;
    const bool nb = a.family == GMF_NEGBIN;
    float sum = 0.f, comp = 0.f;  // compensated (Kahan) per-thread sum
#pragma unroll
    for (int u = 0; u < 4; u++) {
#pragma unroll
        for (int v = 0; v < 4; v++) {
            const int il = ty + 16 * u, jl = tx + 16 * v;
            if (il < nr && jl < nc) {
                const int64_t idx = (row0 + il) * a.m + col0 + jl;
                const float y = load_y(a.Y, a.y16, idx);
                const float wv = a.W ? __ldg(a.W + idx) : 1.f;
                const float e = fminf(fmaxf(acc[u][v], -a.clamp), a.clamp);
                const float mu = expf(e);
                float dv;
                if (nb) {
                    if (y > 0.f)
                        dv = y * log1pf((y - mu) / mu) - (y + alpha) * log1pf((y - mu) / (mu + alpha));
                    else
                        dv = alpha * log1pf(mu / alpha);
                } else {
                    dv = (y > 0.f ? y * log1pf((y - mu) / mu) : 0.f) - (y - mu);
                }
                dv *= 2.f * wv;
                const float yk = dv - comp;
                const float tk = sum + yk;
                comp = (tk - sum) - yk;
                sum = tk;
            }
        }
    }
    const double s = block_sum((double)sum, red);
    if (tid == 0) part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
}

__global__ void sum_parts_kernel(const double* part, int count, double* out) {
    __shared__ double red[NW];
    double s = 0.0;
    for (int c = threadIdx.x; c < count; c += GMF_THREADS) s += part[c];
    s = block_sum(s, red);
    if (threadIdx.x == 0) *out = s;
}

template <typename Ty>
__global__ void permute_kernel(const Ty* __restrict__ src, Ty* __restrict__ dst, int64_t n, int64_t m,
                               const int* __restrict__ rperm, const int* __restrict__ cperm) {
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const Ty* s = src + (int64_t)rperm[i] * m;
        Ty* d = dst + i * m;
        for (int64_t j = threadIdx.x; j < m; j += blockDim.x) d[j] = s[cperm[j]];
    }
}

}  // namespace

StepArgs gmf_make_args(gmf_model* h) {
    StepArgs a{};
    const gmf_config& c = h->cfg;
    a.n = h->n;
    a.m = h->m;
    a.p = h->p;
    a.q = h->q;
    a.d = h->d;
    a.K = h->K;
    a.fr = h->fr;
    a.fc = h->fc;
    a.nb_row = c.nb_row;
    a.nb_col = c.nb_col;
    a.r = h->r;
    a.s = h->s;
    a.per = h->per;
    a.swap = h->swap;
    a.TI = h->TI;
    a.TJ = h->TJ;
    a.family = c.family;
    a.bias_corr = c.bias_corr;
    a.alpha_mode = c.alpha_mode;
    for (int i = 0; i < 4; i++) a.lam[i] = (float)c.lambda[i];
    a.a1 = (float)c.a1;
    a.a2 = (float)c.a2;
    a.damping = (float)c.damping;
    a.eps = (float)c.eps;
    a.clamp = (float)c.eta_clamp;
    a.k0 = c.k0;
    a.k1 = c.k1;
    a.tau = c.tau;
    a.Y = h->Yp;
    a.y16 = h->y16;
    a.W = h->Wp;
    a.L = h->L;
    a.R = h->R;
    a.GbR = h->GbR;
    a.HbR = h->HbR;
    a.GbC = h->GbC;
    a.HbC = h->HbC;
    a.cntR = h->cntR;
    a.cntC = h->cntC;
    a.alpha = h->alpha;
    a.partR = h->partR;
    a.partC = h->partC;
    a.ctrR = h->ctrR;
    a.ctrC = h->ctrC;
    a.ctrSweep = h->ctrSweep;
    a.nbpart = h->nbpart;
    a.sigma = h->sigma;
    a.err = h->err;
    return a;
}

static size_t sweep_smem(int K) { return sizeof(float) * (2 * (size_t)K * LD + 2 * (size_t)T * LDD); }

cudaError_t gmf_launch_sweep_simt(gmf_model* h, const StepArgs& a, int w, long long t0, cudaStream_t st) {
    const size_t smem = sweep_smem(h->K);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sweep_smem(GMF_KMAX));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid(h->TJ, h->TI, h->per);
    sweep_kernel<<<grid, GMF_THREADS, smem, st>>>(a, w, t0);
    return cudaGetLastError();
}

cudaError_t gmf_launch_deviance(gmf_model* h, double* d_out, cudaStream_t st) {
    StepArgs a = gmf_make_args(h);
    dim3 grid((unsigned)((h->m + T - 1) / T), (unsigned)((h->n + T - 1) / T));
    const size_t smem = sizeof(float) * 2 * (size_t)h->K * LD;
    deviance_kernel<<<grid, GMF_THREADS, smem, st>>>(a, h->devpart);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_parts_kernel<<<1, GMF_THREADS, 0, st>>>(h->devpart, (int)(grid.x * grid.y), d_out);
    return cudaGetLastError();
}

cudaError_t gmf_launch_permute_y(const void* src, void* dst, int y16, int64_t n, int64_t m, const int* rperm,
                                 const int* cperm, cudaStream_t st) {
    const int blocks = (int)(n < 65535 ? n : 65535);
    if (y16)
        permute_kernel<unsigned short><<<blocks, 256, 0, st>>>((const unsigned short*)src, (unsigned short*)dst, n, m,
                                                               rperm, cperm);
    else
        permute_kernel<int><<<blocks, 256, 0, st>>>((const int*)src, (int*)dst, n, m, rperm, cperm);
    return cudaGetLastError();
}

cudaError_t gmf_launch_permute_w(const float* src, float* dst, int64_t n, int64_t m, const int* rperm,
                                 const int* cperm, cudaStream_t st) {
    const int blocks = (int)(n < 65535 ? n : 65535);
    permute_kernel<float><<<blocks, 256, 0, st>>>(src, dst, n, m, rperm, cperm);
    return cudaGetLastError();
}
