// Per-cell projection of new cells (the row problem of Sec. 3, solved by the
// Fisher-scoring row step of AIRWLS, Sec. 3.1) with the column side fixed.
//
// For cell i with theta_i = [gamma_i, u_i] (f = q + d free values) and
// r_j = [z_j, v_j]:  eta_ij = o_i + x_i'beta_j + theta_i'r_j, and one step is
//   theta <- theta + (sum_j Dddot_ij r_j r_j' + Lambda)^-1 (sum_j Ddot_ij r_j - Lambda theta).
// A CTA owns 32 cells and streams the genes in chunks of 32: it forms eta, mu,
// Ddot, Dddot for the 32 x 32 chunk, then accumulates each cell's Fisher matrix
// (packed lower triangle, f(f+1)/2 entries; warp w owns cells 4w..4w+3, lane l
// the pairs l, l+32, ...) against the chunk's precomputed pair products
// r_ja r_jb, and its score. Each of 32 threads then solves one cell's system by
// an in-place packed Cholesky. Start: u from the caller (or 0); gamma_0 (the
// first Z column) in closed form log(max(sum_j y_ij, 0.5) / sum_j exp(eta_ij
// without gamma)), other gamma 0. FP32 throughout.
//
// Step control: every pass also sums the cell's unit deviances, giving the
// penalised objective f = 0.5 dev + 0.5 theta' Lambda theta at the current
// point. A point with f <= f_best + 1e-5 (1 + |f_best|) is accepted and the
// Fisher step is taken from it; otherwise the last step is halved and tried
// from the best point. The best point and its deviance are the output. Plain
// Fisher scoring overshoots from far starts; accepted steps are exact Fisher
// steps, so cells whose steps descend take the same path as without control.
#include <math.h>

#include <algorithm>
#include <string>

#include <cuda_bf16.h>

#include "gmf_internal.cuh"

namespace {

constexpr int NT = 256;
constexpr int CC = 32;     // cells per CTA
constexpr int GC = 32;     // genes per chunk
constexpr int FMAX = 32;   // largest q + d
constexpr float SLACK = 1e-5f;  // relative slack of the acceptance test

struct ProjArgs {
    const void* Y;
    int y16;
    int64_t n, m;
    int p, q, d, KP;
    const float* X;       // n x p
    const float* off;     // n or null
    const float* Ustart;  // n x d or null
    const float* R;       // m x KP, original gene order: [1 | B | Z | V]
    const float* alpha;
    int nb;
    float clamp, lam_g, lam_u;
    int n_steps;
    float* Uout;
    float* Gout;
    float* dev;
};

__device__ __forceinline__ int pidx(int i, int j) { return i * (i + 1) / 2 + j; }  // i >= j

template <int PP>
__global__ void __launch_bounds__(NT) project_kernel(ProjArgs a) {
    extern __shared__ __align__(16) float sm[];
    const int f = a.q + a.d, np = f * (f + 1) / 2;
    float* Rs = sm;                              // GC x KP gene rows
    float* RR = Rs + GC * a.KP;                  // GC x np pair products; later CC x np Fisher matrices
    float* Dd = RR + (size_t)max(GC, CC) * np;   // CC x (GC+1)
    float* DDd = Dd + CC * (GC + 1);
    float* TH = DDd + CC * (GC + 1);             // CC x f  theta
    float* GR = TH + CC * FMAX;                  // CC x f  score
    float* BASE = GR + CC * FMAX;                // CC x (GC+1)  o_i + x_i'beta_j
    float* S1 = BASE + CC * (GC + 1);            // CC: sum y (init) / deviance
    float* S2 = S1 + CC;                         // CC: sum exp(rest) (init)
    float* DV = S2 + CC;                         // CC x (GC+1)  unit deviances of the chunk
    float* BEST = DV + CC * (GC + 1);            // CC x f  best accepted theta
    float* DEL = BEST + CC * FMAX;               // CC x f  last step
    float* FB = DEL + CC * FMAX;                 // CC: best objective
    float* DB = FB + CC;                         // CC: deviance at the best point

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t cell0 = (int64_t)blockIdx.x * CC;
    const int ncell = (int)min((int64_t)CC, a.n - cell0);
    const float alpha = *a.alpha;

    for (int e = tid; e < CC * f; e += NT) {
        const int c = e / f, k = e - c * f;
        float v = 0.f;
        if (c < ncell && k >= a.q && a.Ustart) v = a.Ustart[(cell0 + c) * a.d + (k - a.q)];
        TH[c * FMAX + k] = v;
    }
    if (tid < CC) FB[tid] = DB[tid] = 0.f;
    // passes: 0 = closed-form gamma; 1..n_steps+1 evaluate the objective at the
    // current point, and 1..n_steps also form the Fisher system there
    for (int pass = 0; pass <= a.n_steps + 1; pass++) {
        const bool init = pass == 0, fisher = pass >= 1 && pass <= a.n_steps;
        if (init && a.q == 0) continue;
        float facc[4][PP], gacc[4], dacc[4];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            gacc[c] = dacc[c] = 0.f;
#pragma unroll
            for (int t = 0; t < PP; t++) facc[c][t] = 0.f;
        }
        if (tid < CC) S1[tid] = S2[tid] = 0.f;
        __syncthreads();
        for (int g0 = 0; g0 < a.m; g0 += GC) {
            const int ng = (int)min((int64_t)GC, a.m - g0);
            for (int e = tid; e < GC * a.KP; e += NT) {
                const int g = e / a.KP, c = e - g * a.KP;
                Rs[e] = g < ng ? __ldg(a.R + (int64_t)(g0 + g) * a.KP + c) : 0.f;
            }
            __syncthreads();
            if (fisher)
                for (int e = tid; e < GC * np; e += NT) {
                    const int g = e / np, pr = e - g * np;
                    int i = (int)((sqrtf(8.f * pr + 1.f) - 1.f) * 0.5f);
                    while (i * (i + 1) / 2 > pr) i--;
                    while ((i + 1) * (i + 2) / 2 <= pr) i++;
                    const int j = pr - i * (i + 1) / 2;
                    RR[e] = Rs[g * a.KP + 1 + a.p + i] * Rs[g * a.KP + 1 + a.p + j];
                }
            // eta, mu and the per-entry quantities of the 32 x 32 chunk
            for (int e = tid; e < CC * GC; e += NT) {
                const int c = e / GC, g = e - c * GC;
                float dd = 0.f, ddd = 0.f, dvu = 0.f;
                if (c < ncell && g < ng) {
                    const int64_t cell = cell0 + c;
                    float base = a.off ? a.off[cell] : 0.f;
                    for (int k = 0; k < a.p; k++) base = fmaf(a.X[cell * a.p + k], Rs[g * a.KP + 1 + k], base);
                    float eta = base;
                    for (int k = 0; k < f; k++) eta = fmaf(TH[c * FMAX + k], Rs[g * a.KP + 1 + a.p + k], eta);
                    const int64_t yi = cell * a.m + g0 + g;
                    const float y = a.y16 ? (float)((const unsigned short*)a.Y)[yi] : (float)((const int*)a.Y)[yi];
                    if (init) {
                        // rest = eta without gamma
                        float rest = eta;
                        for (int k = 0; k < a.q; k++) rest -= TH[c * FMAX + k] * Rs[g * a.KP + 1 + a.p + k];
                        dd = y;
                        ddd = expf(fminf(fmaxf(rest, -a.clamp), a.clamp));
                    } else {
                        const float ec = fminf(fmaxf(eta, -a.clamp), a.clamp);
                        const float mu = expf(ec);
                        {
                            float dv;
                            if (y > 0.f) {
                                const float r1 = (y - mu) / mu;
                                const float l1 = fabsf(r1) < 0.5f ? log1pf(r1) : logf(y) - ec;
                                if (!a.nb) {
                                    dv = y * l1 - (y - mu);
                                } else {
                                    const float r2 = (y - mu) / (mu + alpha);
                                    const float lma = mu > alpha ? ec + log1pf(alpha / mu) : logf(alpha) + log1pf(mu / alpha);
                                    const float l2 = fabsf(r2) < 0.5f ? log1pf(r2) : logf(y + alpha) - lma;
                                    dv = y * l1 - (y + alpha) * l2;
                                }
                            } else {
                                dv = a.nb ? alpha * log1pf(mu / alpha) : mu;
                            }
                            dvu = 2.f * dv;
                        }
                        if (fisher) {
                            const float fct = a.nb ? alpha / (alpha + mu) : 1.f;
                            dd = (y - mu) * fct;
                            ddd = mu * fct;
                        }
                    }
                }
                Dd[c * (GC + 1) + g] = dd;
                DDd[c * (GC + 1) + g] = ddd;
                DV[c * (GC + 1) + g] = dvu;
            }
            __syncthreads();
            if (!init) {
                // warp w: cells 4w..4w+3; lane: gene lane of the chunk for the deviance
#pragma unroll
                for (int c = 0; c < 4; c++) dacc[c] += DV[(4 * warp + c) * (GC + 1) + lane];
            }
            if (fisher) {
                // warp w: cells 4w..4w+3; lane: pairs lane + 32t, score component lane
                for (int g = 0; g < ng; g++) {
                    float w4[4], d4[4];
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        w4[c] = DDd[(4 * warp + c) * (GC + 1) + g];
                        d4[c] = Dd[(4 * warp + c) * (GC + 1) + g];
                    }
                    const float rl = lane < f ? Rs[g * a.KP + 1 + a.p + lane] : 0.f;
#pragma unroll
                    for (int c = 0; c < 4; c++) gacc[c] = fmaf(d4[c], rl, gacc[c]);
#pragma unroll
                    for (int t = 0; t < PP; t++) {
                        const int pr = lane + 32 * t;
                        const float rr = pr < np ? RR[g * np + pr] : 0.f;
#pragma unroll
                        for (int c = 0; c < 4; c++) facc[c][t] = fmaf(w4[c], rr, facc[c][t]);
                    }
                }
            } else if (init && tid < CC) {
                // S1 = sum y, S2 = sum exp(rest)
                float s1 = S1[tid], s2 = S2[tid];
                for (int g = 0; g < ng; g++) {
                    s1 += Dd[tid * (GC + 1) + g];
                    s2 += DDd[tid * (GC + 1) + g];
                }
                S1[tid] = s1;
                S2[tid] = s2;
            }
            __syncthreads();
        }
        if (init) {
            if (tid < ncell) TH[tid * FMAX + 0] = logf(fmaxf(S1[tid], 0.5f) / S2[tid]);
            __syncthreads();
            continue;
        }
#pragma unroll
        for (int c = 0; c < 4; c++) {
            float v = dacc[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) S1[4 * warp + c] = v;
        }
        float* F = RR;  // CC x np
        if (fisher) {
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const int cell = 4 * warp + c;
#pragma unroll
                for (int t = 0; t < PP; t++) {
                    const int pr = lane + 32 * t;
                    if (pr < np) F[cell * np + pr] = facc[c][t];
                }
                if (lane < f) GR[cell * FMAX + lane] = gacc[c];
            }
        }
        __syncthreads();
        if (tid < ncell) {
            float* th = TH + tid * FMAX;
            float* be = BEST + tid * FMAX;
            float* de = DEL + tid * FMAX;
            float pen = 0.f;
            for (int k = 0; k < f; k++) pen += (k < a.q ? a.lam_g : a.lam_u) * th[k] * th[k];
            const float obj = 0.5f * S1[tid] + 0.5f * pen;
            const float fb = FB[tid];
            if (pass == 1 || obj <= fb + SLACK * (1.f + fabsf(fb))) {
                for (int k = 0; k < f; k++) be[k] = th[k];
                FB[tid] = obj;
                DB[tid] = S1[tid];
                if (fisher) {
                    float* A = F + tid * np;
                    float* b = GR + tid * FMAX;
                    for (int k = 0; k < f; k++) {
                        const float lam = k < a.q ? a.lam_g : a.lam_u;
                        A[pidx(k, k)] += lam;
                        b[k] -= lam * th[k];
                    }
                    bool ok = true;
                    for (int j = 0; j < f; j++) {  // packed lower Cholesky in place
                        float s = A[pidx(j, j)];
                        for (int k = 0; k < j; k++) s -= A[pidx(j, k)] * A[pidx(j, k)];
                        if (!(s > 0.f)) {
                            ok = false;
                            break;
                        }
                        const float ljj = sqrtf(s);
                        A[pidx(j, j)] = ljj;
                        for (int i = j + 1; i < f; i++) {
                            float t = A[pidx(i, j)];
                            for (int k = 0; k < j; k++) t -= A[pidx(i, k)] * A[pidx(j, k)];
                            A[pidx(i, j)] = t / ljj;
                        }
                    }
                    if (ok) {
                        for (int i = 0; i < f; i++) {  // L z = b
                            float s = b[i];
                            for (int k = 0; k < i; k++) s -= A[pidx(i, k)] * b[k];
                            b[i] = s / A[pidx(i, i)];
                        }
                        for (int i = f - 1; i >= 0; i--) {  // L' x = z
                            float s = b[i];
                            for (int k = i + 1; k < f; k++) s -= A[pidx(k, i)] * b[k];
                            b[i] = s / A[pidx(i, i)];
                        }
                    }
                    for (int k = 0; k < f; k++) {
                        de[k] = ok ? b[k] : 0.f;
                        th[k] = be[k] + de[k];
                    }
                }
            } else {
                for (int k = 0; k < f; k++) {
                    de[k] *= 0.5f;
                    th[k] = be[k] + de[k];
                }
            }
        }
        __syncthreads();
    }
    if (tid < ncell && a.dev) a.dev[cell0 + tid] = DB[tid];
    for (int e = tid; e < ncell * f; e += NT) {
        const int c = e / f, k = e - c * f;
        const float v = BEST[c * FMAX + k];
        if (k < a.q)
            a.Gout[(cell0 + c) * a.q + k] = v;
        else
            a.Uout[(cell0 + c) * a.d + (k - a.q)] = v;
    }
}

__global__ void unpermute_rows(const float* R, const int* cperm, int64_t m, int KP, float* Rorig) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m * KP; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t jp = e / KP;
        const int c = (int)(e - jp * KP);
        Rorig[(int64_t)cperm[jp] * KP + c] = R[e];
    }
}

size_t project_smem(int KP, int f) {
    const int np = f * (f + 1) / 2;
    return sizeof(float) * ((size_t)GC * KP + (size_t)std::max(GC, CC) * np + 4 * (size_t)CC * (GC + 1) +
                            4 * (size_t)CC * FMAX + 4 * (size_t)CC);
}

}  // namespace

// gmf_project_tc.cu
int gmf_project_tc_run(const float* Rorig, int64_t m, int p, int q, int d, int KP, const void* Ynew, int y16,
                       int64_t n_new, const float* Xnew, const float* off, const float* Ustart, const float* alpha,
                       int nb, float clamp, float lam_g, float lam_u, int n_steps, float* Uout, float* Gout, float* dev,
                       unsigned* err_word, __nv_bfloat16** kr_buf, size_t* kr_elems, cudaStream_t st,
                       std::string* err);

int gmf_project_run(gmf_model* h, const void* Ynew, int y16, int64_t n_new, const float* Xnew, const float* off,
                    const float* Ustart, int n_steps, float* Uout, float* Gout, float* dev, cudaStream_t st,
                    std::string* err) {
    const int f = h->q + h->d;
    if (f > FMAX || f < 1) {
        *err = "q + d must be between 1 and 32";
        return GMF_ERR_ARG;
    }
    if (!h->Rorig) {
        if (cudaMalloc(&h->Rorig, sizeof(float) * (size_t)h->m * h->KP) != cudaSuccess) {
            *err = "device allocation failed";
            return GMF_ERR_OOM;
        }
    }
    unpermute_rows<<<(int)std::min<int64_t>((h->m * h->KP + 255) / 256, 4096), 256, 0, st>>>(h->R, h->cperm, h->m,
                                                                                             h->KP, h->Rorig);
    if (h->cfg.precision == GMF_PREC_MIXED) {
        // Fisher matrices on the tensor cores where the shapes allow (f <= 22, uint16 counts, ...)
        const int rc = gmf_project_tc_run(h->Rorig, h->m, h->p, h->q, h->d, h->KP, Ynew, y16, n_new, Xnew, off, Ustart,
                                          h->alpha, h->cfg.family == GMF_NEGBIN, (float)h->cfg.eta_clamp,
                                          (float)h->cfg.lambda[1], (float)h->cfg.lambda[2], n_steps, Uout, Gout, dev,
                                          h->err, (__nv_bfloat16**)&h->kr_buf, &h->kr_elems, st, err);
        if (rc != GMF_ERR_STATE) return rc;
    }
    ProjArgs a{};
    a.Y = Ynew;
    a.y16 = y16;
    a.n = n_new;
    a.m = h->m;
    a.p = h->p;
    a.q = h->q;
    a.d = h->d;
    a.KP = h->KP;
    a.X = Xnew;
    a.off = off;
    a.Ustart = Ustart;
    a.R = h->Rorig;
    a.alpha = h->alpha;
    a.nb = h->cfg.family == GMF_NEGBIN;
    a.clamp = (float)h->cfg.eta_clamp;
    a.lam_g = (float)h->cfg.lambda[1];
    a.lam_u = (float)h->cfg.lambda[2];
    a.n_steps = n_steps;
    a.Uout = Uout;
    a.Gout = Gout;
    a.dev = dev;
    const size_t smem = project_smem(h->KP, f);
    const int np = f * (f + 1) / 2;
    const dim3 grid((unsigned)((n_new + CC - 1) / CC));
    cudaError_t e;
    if (np <= 32 * 8) {
        e = gmf_smem_limit((const void*)project_kernel<8>, smem);
        if (e == cudaSuccess) project_kernel<8><<<grid, NT, smem, st>>>(a);
    } else {
        e = gmf_smem_limit((const void*)project_kernel<17>, smem);
        if (e == cudaSuccess) project_kernel<17><<<grid, NT, smem, st>>>(a);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        *err = cudaGetErrorString(e);
        return GMF_ERR_CUDA;
    }
    return GMF_OK;
}
