// FP32 CUDA-core path of the block step (Algorithm 1, eq. 15 / App. B,
// eq. 12, eq. 14) and the full deviance (Table S1, App. B).
//
// One launch per sweep. Grid (TJ, TI, per): CTA (tj, ti, k) owns a 64 x 64
// tile of block k of the sweep. Per tile:
//   1. the L and R rows of the tile go to shared memory, transposed for the
//      eta product and row-major (with squares) for the two contractions;
//   2. each thread forms a 4 x 4 micro-tile of eta = L R' in FP32, then
//      mu = exp(eta), Ddot, Dddot (Sec. 3, log link) -> shared memory;
//   3. row partials sum_j Ddot_ij R_jc, sum_j Dddot_ij R_jc^2 (c row-free) and
//      column partials sum_i Ddot_ij L_ic, sum_i Dddot_ij L_ic^2 (c column-free):
//      four lanes split the 64-long sum, registers hold the Ddot values, the
//      factor operands arrive as 128-bit broadcast loads, and the four lane
//      partials are combined by shuffles in a fixed order;
//   4. the partials go to a workspace slot per tile (no atomics on values); an
//      arrival counter per row strip and per column strip elects the last CTA
//      of the strip, which sums the strip's partials in tile order and applies
//      scale factor, penalty, damping, EMA and step to its rows (columns).
//      Every reader of those parameters in this sweep has arrived, so the
//      update cannot race with a reader, and no CTA waits on another.
// rho_t * c_t of each block comes precomputed from the host (FP64 there); the
// device does no FP64 arithmetic except the cross-CTA sums of the NB moments.
#include <math.h>

#include <algorithm>

#include "gmf_internal.cuh"
#include "gmf_update.cuh"

namespace {

using namespace gmfdev;

constexpr int T = GMF_TILE;
constexpr int LD = T + 4;   // transposed factor tiles: 16-byte aligned rows
constexpr int LDD = T + 4;  // Ddot / Dddot tiles (row-major)
constexpr int NW = GMF_THREADS / 32;
constexpr int CHP = 2;      // 4-column chunks per contraction pass

__device__ __forceinline__ float load_y(const void* Y, int y16, int64_t idx, int yf32 = 0) {
    if (yf32) return __ldg((const float*)Y + idx);
    return y16 ? (float)__ldg((const unsigned short*)Y + idx) : (float)__ldg((const int*)Y + idx);
}

// Four consecutive counts of one row (vector load when aligned).
__device__ __forceinline__ void load_y4(const void* Y, int y16, int64_t idx, bool vec, int valid, float y[4],
                                        int yf32 = 0) {
    if (vec && valid == 4) {
        if (yf32) {
            const float4 v = __ldg((const float4*)((const float*)Y + idx));
            y[0] = v.x; y[1] = v.y; y[2] = v.z; y[3] = v.w;
        } else if (y16) {
            const ushort4 v = __ldg((const ushort4*)((const unsigned short*)Y + idx));
            y[0] = v.x; y[1] = v.y; y[2] = v.z; y[3] = v.w;
        } else {
            const int4 v = __ldg((const int4*)((const int*)Y + idx));
            y[0] = (float)v.x; y[1] = (float)v.y; y[2] = (float)v.z; y[3] = (float)v.w;
        }
        return;
    }
#pragma unroll
    for (int b = 0; b < 4; b++) y[b] = b < valid ? load_y(Y, y16, idx + b, yf32) : 0.f;
}

// Rows [row0, row0+nr) of F (row stride KP, a multiple of 4) -> St[c*LD + i]
// (transposed), zero-filled beyond nr. All loads of a thread are issued before
// any store (one L2 round trip).
__device__ __forceinline__ void load_factor_T(float* St, const float* F, int KP, int64_t row0, int nr) {
    const int q4 = KP >> 2;                 // float4 per row
    const int total = T * q4;               // <= 1024 for KP <= 64
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
        const int e = threadIdx.x + u * GMF_THREADS;
        const int i = e / q4;
        v[u] = (e < total && i < nr) ? __ldg((const float4*)(F + (row0 + i) * KP) + (e - i * q4))
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
        const int e = threadIdx.x + u * GMF_THREADS;
        if (e < total) {
            const int i = e / q4, c = 4 * (e - i * q4);
            St[(c + 0) * LD + i] = v[u].x;
            St[(c + 1) * LD + i] = v[u].y;
            St[(c + 2) * LD + i] = v[u].z;
            St[(c + 3) * LD + i] = v[u].w;
        }
    }
}

// Free-column operands of a contraction: O[i*2P + c] = F[i, col(c)], O[i*2P + P + c] = its square.
// col(c) = c0 + c for row-free columns; c < p ? 1 + c : 1 + q + c for column-free ones.
__device__ __forceinline__ void load_operands(float* O, const float* St, int nf, int P, int c_lo, int p, int q,
                                              bool colfree) {
    for (int e = threadIdx.x; e < T * P; e += GMF_THREADS) {
        const int i = e / P, c = e - i * P;
        float v = 0.f;
        if (c < nf) {
            const int col = colfree ? (c < p ? 1 + c : 1 + q + c) : c_lo + c;
            v = St[col * LD + i];
        }
        O[i * 2 * P + c] = v;
        O[i * 2 * P + P + c] = v * v;
    }
}

// Contraction of one tile side. Thread (o = tid >> 2, q4 = tid & 3) owns output
// row o (a tile row for the row side, a tile column for the column side) and
// the summation indices kk = 4*s + q4, s < 16. D(o, kk) is read through
// dstride_o / dstride_k. Operands O[kk][2P] (values then squares).
// Writes sums for c < nf to dst[c*T + o] (G) and dst[(nf + c)*T + o] (H).
__device__ __forceinline__ void contract_side(const float* __restrict__ Ds, const float* __restrict__ DDs,
                                              int dstride_o, int dstride_k, const float* __restrict__ O, int P,
                                              int nf, int nvalid_k, int nvalid_o, float* __restrict__ dst) {
    const int o = threadIdx.x >> 2, q4 = threadIdx.x & 3;
    float dv[16], ddv[16];
#pragma unroll
    for (int s = 0; s < 16; s++) {
        const int kk = 4 * s + q4;
        dv[s] = Ds[o * dstride_o + kk * dstride_k];
        ddv[s] = DDs[o * dstride_o + kk * dstride_k];
    }
    const int nch = P >> 2;
    const int kmax = (nvalid_k + 3) >> 2;  // s beyond this only sees zeros
    for (int ch0 = 0; ch0 < nch; ch0 += CHP) {
        float g[CHP][4], h[CHP][4];
#pragma unroll
        for (int u = 0; u < CHP; u++)
#pragma unroll
            for (int v = 0; v < 4; v++) g[u][v] = h[u][v] = 0.f;
#pragma unroll
        for (int s = 0; s < 16; s++) {
            if (s >= kmax) break;
            const int kk = 4 * s + q4;
            const float4* row = (const float4*)(O + kk * 2 * P);
#pragma unroll
            for (int u = 0; u < CHP; u++) {
                if (ch0 + u < nch) {
                    const float4 r = row[ch0 + u];
                    const float4 r2 = row[(P >> 2) + ch0 + u];
                    g[u][0] = fmaf(dv[s], r.x, g[u][0]);
                    g[u][1] = fmaf(dv[s], r.y, g[u][1]);
                    g[u][2] = fmaf(dv[s], r.z, g[u][2]);
                    g[u][3] = fmaf(dv[s], r.w, g[u][3]);
                    h[u][0] = fmaf(ddv[s], r2.x, h[u][0]);
                    h[u][1] = fmaf(ddv[s], r2.y, h[u][1]);
                    h[u][2] = fmaf(ddv[s], r2.z, h[u][2]);
                    h[u][3] = fmaf(ddv[s], r2.w, h[u][3]);
                }
            }
        }
        // combine the four lanes of this output row: ((q0 + q1) + (q2 + q3)), identical on all four
#pragma unroll
        for (int u = 0; u < CHP; u++)
#pragma unroll
            for (int v = 0; v < 4; v++) {
                g[u][v] += __shfl_xor_sync(0xffffffffu, g[u][v], 1);
                g[u][v] += __shfl_xor_sync(0xffffffffu, g[u][v], 2);
                h[u][v] += __shfl_xor_sync(0xffffffffu, h[u][v], 1);
                h[u][v] += __shfl_xor_sync(0xffffffffu, h[u][v], 2);
            }
        if (o < nvalid_o) {
#pragma unroll
            for (int u = 0; u < CHP; u++)
#pragma unroll
                for (int v = 0; v < 4; v++) {
                    const int c = 4 * (ch0 + u) + v;
                    if (v == q4 && c < nf) {
                        dst[c * T + o] = g[u][v];
                        dst[(nf + c) * T + o] = h[u][v];
                    }
                }
        }
    }
}

struct Smem {
    float *Ls, *Rs, *RF, *LF, *Ds, *DDs;
};

__device__ __forceinline__ Smem carve(float* base, int K, int FRP, int FCP) {
    Smem s;
    s.Ls = base;
    s.Rs = s.Ls + K * LD;   // K here is the padded KP
    s.RF = s.Rs + K * LD;
    s.LF = s.RF + T * 2 * FRP;
    s.Ds = s.LF + T * 2 * FCP;
    s.DDs = s.Ds + T * LDD;
    return s;
}

__device__ __forceinline__ void simt_tile(const StepArgs& a, int w, int k, float* smem) {
    const int FRP = (a.fr + 3) & ~3, FCP = (a.fc + 3) & ~3;
    const Smem S = carve(smem, a.KP, FRP, FCP);
    const int tid = threadIdx.x;
    const int tj = blockIdx.x, ti = blockIdx.y;
    const BlockGeo g = block_geo(a, w, k);
    const int nTI = (int)((g.nI + T - 1) / T), nTJ = (int)((g.mJ + T - 1) / T);
    const bool active = ti < nTI && tj < nTJ;
    const bool nb = a.family == GMF_NEGBIN;
    const bool glm = a.family >= GMF_GAUSSIAN;  // the other families of Table S1
    const bool moments = scalar_estimated(a.family, a.alpha_mode);
    grid_dependency_wait();  // the previous sweep's update launch writes the model state
    grid_launch_dependents();  // this sweep's update may start: the previous one has completed
    const float alpha = *a.alpha;
    float s1 = 0.f, s2 = 0.f;

    const int64_t row0 = g.r0 + (int64_t)ti * T, col0 = g.c0 + (int64_t)tj * T;
    const int nr = active ? (int)min((int64_t)T, g.nI - (int64_t)ti * T) : 0;
    const int nc = active ? (int)min((int64_t)T, g.mJ - (int64_t)tj * T) : 0;

    if (active) {
        // eta micro-tile of this thread: rows 4ty..4ty+3, columns 4tx..4tx+3.
        // Its counts (and weights) are requested first so that the HBM latency
        // overlaps the factor loads and the eta product.
        const int tx = tid & 15, ty = tid >> 4;
        const bool vec = ((a.m & 3) == 0) && ((col0 & 3) == 0);
        float yv[4][4], wv[4][4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int il = 4 * ty + u, jl0 = 4 * tx;
            const int valid = il < nr ? max(0, min(4, nc - jl0)) : 0;
            const int64_t idx = (row0 + il) * a.m + col0 + jl0;
            if (valid > 0) load_y4(a.Y, a.y16, idx, vec, valid, yv[u], a.yf32);
#pragma unroll
            for (int v = 0; v < 4; v++) {
                if (valid == 0) yv[u][v] = 0.f;
                wv[u][v] = (a.W && v < valid) ? __ldg(a.W + idx + v) : 1.f;
            }
        }
        load_factor_T(S.Ls, a.L, a.KP, row0, nr);
        load_factor_T(S.Rs, a.R, a.KP, col0, nc);
        __syncthreads();
        load_operands(S.RF, S.Rs, a.fr, FRP, 1 + a.p, a.p, a.q, false);
        load_operands(S.LF, S.Ls, a.fc, FCP, 0, a.p, a.q, true);
        float acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; u++)
#pragma unroll
            for (int v = 0; v < 4; v++) acc[u][v] = 0.f;
        for (int c = 0; c < a.K; c++) {
            const float4 lv = *(const float4*)(S.Ls + c * LD + 4 * ty);
            const float4 rv = *(const float4*)(S.Rs + c * LD + 4 * tx);
            const float l4[4] = {lv.x, lv.y, lv.z, lv.w}, r4[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int v = 0; v < 4; v++) acc[u][v] = fmaf(l4[u], r4[v], acc[u][v]);
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int il = 4 * ty + u;
            const int jl0 = 4 * tx;
            const int valid = il < nr ? max(0, min(4, nc - jl0)) : 0;
            float dd[4], ddd[4];
#pragma unroll
            for (int v = 0; v < 4; v++) {
                dd[v] = ddd[v] = 0.f;
                if (v < valid && glm) {
                    const float w8 = wv[u][v];
                    const float e = fminf(fmaxf(acc[u][v], -a.clamp), a.clamp);
                    const float mu = glm_mean(a.family, e);
                    const bool miss = y_missing(a, yv[u][v]);
                    const float y = miss ? mu : yv[u][v];
                    float d1, d2;
                    glm_derivs(a.family, y, mu, alpha, d1, d2);
                    dd[v] = w8 * d1;
                    ddd[v] = w8 * d2;
                    if (moments && !miss) {
                        s1 += w8 * (y - mu) * (y - mu) / glm_variance(a.family, mu);
                        s2 += 1.f;
                    }
                } else if (v < valid) {
                    const float w8 = wv[u][v];
                    const float e = fminf(fmaxf(acc[u][v], -a.clamp), a.clamp);
                    const float mu = expf(e);
                    // an unobserved entry is imputed by the current mean (Sec. 3.2)
                    const float y = (a.missing && yv[u][v] == a.ymiss) ? mu : yv[u][v];
                    const float aj = a.alpha_col ? __ldg(a.alpha_col + col0 + jl0 + v) : alpha;
                    const float f = nb ? aj / (aj + mu) : 1.f;
                    dd[v] = w8 * (y - mu) * f;
                    ddd[v] = w8 * mu * f;
                    if (moments) {
                        s1 = fmaf(w8 * mu, mu, s1);
                        s2 += w8 * ((y - mu) * (y - mu) - mu);
                    }
                }
            }
            *(float4*)(S.Ds + il * LDD + jl0) = make_float4(dd[0], dd[1], dd[2], dd[3]);
            *(float4*)(S.DDs + il * LDD + jl0) = make_float4(ddd[0], ddd[1], ddd[2], ddd[3]);
        }
        __syncthreads();
        float* prow = a.partR + ((size_t)((k * a.TI + ti) * a.TJ + tj) * T) * 2 * a.fr;
        float* pcol = a.partC + ((size_t)((k * a.TJ + tj) * a.TI + ti) * T) * 2 * a.fc;
        // row side: output row o = tile row, summation over tile columns
        contract_side(S.Ds, S.DDs, LDD, 1, S.RF, FRP, a.fr, nc, nr, prow);
        // column side: output o = tile column, summation over tile rows
        contract_side(S.Ds, S.DDs, 1, LDD, S.LF, FCP, a.fc, nr, nc, pcol);
    }

    tile_moments<GMF_THREADS>(a, k, ti, tj, s1, s2);
}

__global__ void __launch_bounds__(GMF_THREADS, 3) sweep_kernel(StepArgs a, int w) {
    extern __shared__ __align__(16) float smem[];
    simt_tile(a, w, block_of_slot(a, blockIdx.z), smem);
}

// Several models sharing the count matrix: blockIdx.z = slot * per + k (see sweep_tc_multi).
__global__ void __launch_bounds__(GMF_THREADS, 3) sweep_multi(const StepArgs* __restrict__ av,
                                                             const int* __restrict__ order, int per, int w) {
    extern __shared__ __align__(16) float smem[];
    __shared__ StepArgs s_a;
    if (threadIdx.x == 0) s_a = av[order[blockIdx.z / per]];
    __syncthreads();
    simt_tile(s_a, w, blockIdx.z % per, smem);
}

// Deviance of one 64 x 64 tile of the whole (permuted) matrix.
__global__ void __launch_bounds__(GMF_THREADS) deviance_kernel(StepArgs a, double* part) {
    extern __shared__ __align__(16) float smem[];
    float* Ls = smem;
    float* Rs = Ls + a.KP * LD;
    __shared__ float red[NW];
    __shared__ float tlog[256], tloga[256];  // log(v), log(v + alpha), v < 256
    const int tid = threadIdx.x;
    {
        const float al = *a.alpha;
        tlog[tid] = tid > 0 ? logf((float)tid) : 0.f;
        tloga[tid] = logf((float)tid + al);
    }
    const int64_t row0 = (int64_t)blockIdx.y * T, col0 = (int64_t)blockIdx.x * T;
    const int nr = (int)min((int64_t)T, a.n - row0), nc = (int)min((int64_t)T, a.m - col0);
    load_factor_T(Ls, a.L, a.KP, row0, nr);
    load_factor_T(Rs, a.R, a.KP, col0, nc);
    __syncthreads();
    const int tx = tid & 15, ty = tid >> 4;
    float acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
        for (int v = 0; v < 4; v++) acc[u][v] = 0.f;
    for (int c = 0; c < a.K; c++) {
        const float4 lv = *(const float4*)(Ls + c * LD + 4 * ty);
        const float4 rv = *(const float4*)(Rs + c * LD + 4 * tx);
        const float l4[4] = {lv.x, lv.y, lv.z, lv.w}, r4[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
        for (int u = 0; u < 4; u++)
#pragma unroll
            for (int v = 0; v < 4; v++) acc[u][v] = fmaf(l4[u], r4[v], acc[u][v]);
    }
    const float alpha = *a.alpha;
    const float la = tloga[0];  // log(alpha), the same rounding as the table's y = 0 entry
    const bool nb = a.family == GMF_NEGBIN;
    const bool vec = ((a.m & 3) == 0) && ((col0 & 3) == 0);
    float sum = 0.f, comp = 0.f;  // compensated (Kahan) per-thread sum
#pragma unroll
    for (int u = 0; u < 4; u++) {
        const int il = 4 * ty + u, jl0 = 4 * tx;
        const int valid = il < nr ? max(0, min(4, nc - jl0)) : 0;
        if (valid == 0) continue;
        const int64_t idx = (row0 + il) * a.m + col0 + jl0;
        float y[4];
        load_y4(a.Y, a.y16, idx, vec, valid, y, a.yf32);
#pragma unroll
        for (int v = 0; v < 4; v++) {
            if (v < valid && !y_missing(a, y[v])) {   // y <- mu: D(mu, mu) = 0
                const float wv = a.W ? __ldg(a.W + idx + v) : 1.f;
                const float e = fminf(fmaxf(acc[u][v], -a.clamp), a.clamp);
                float hd;
                if (a.family >= GMF_GAUSSIAN) {
                    hd = 0.5f * glm_unit_dev(a.family, y[v], e, glm_mean(a.family, e));
                } else if (a.alpha_col) {   // per-gene shapes: no tables of log(y + alpha)
                    const float aj = __ldg(a.alpha_col + col0 + jl0 + v), mu = expf(e);
                    hd = y[v] > 0.f ? half_dev_ratio(nb, y[v], e, mu, aj) : (nb ? aj * log1pf(mu / aj) : mu);
                } else {
                    hd = half_dev_tab(nb, y[v], e, expf(e), alpha, la, tlog, tloga);
                }
                const float dv = 2.f * wv * hd;
                const float yk = dv - comp;
                const float tk = sum + yk;
                comp = (tk - sum) - yk;
                sum = tk;
            }
        }
    }
    const float s = block_sum_f<GMF_THREADS>(sum, red);
    if (tid == 0) part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = (double)s;
}

__global__ void sum_parts_kernel(const double* part, int count, double* out) {
    __shared__ double red[NW];
    double s = 0.0;
    for (int c = threadIdx.x; c < count; c += GMF_THREADS) s += part[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int u = 0; u < NW; u++) t += red[u];
        *out = t;
    }
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

// Mapped host rows -> permuted device rows. Each CTA takes `rows` destination
// rows at a time: their source rows come over the host link as 16-byte loads
// into shared memory (all loads of the group in flight before the first use),
// then the destination rows are written in column order.
constexpr int GH_THREADS = 512;
template <typename Ty>
__global__ void __launch_bounds__(GH_THREADS)
    gather_host_kernel(const Ty* __restrict__ src, Ty* __restrict__ dst, int64_t n, int64_t m,
                       const int* __restrict__ rperm, const int* __restrict__ cperm, int rows) {
    extern __shared__ uint4 gh_smem[];
    const Ty* srow = (const Ty*)gh_smem;
    const int chunks = (int)(m * (int64_t)sizeof(Ty) / 16);  // 16-byte chunks per row
    for (int64_t i0 = (int64_t)blockIdx.x * rows; i0 < n; i0 += (int64_t)gridDim.x * rows) {
        const int nr = (int)min((int64_t)rows, n - i0);
        for (int e = threadIdx.x; e < nr * chunks; e += blockDim.x) {
            const int r = e / chunks, c = e - r * chunks;
            gh_smem[e] = ((const uint4*)(src + (int64_t)rperm[i0 + r] * m))[c];
        }
        __syncthreads();
        for (int64_t e = threadIdx.x; e < (int64_t)nr * m; e += blockDim.x) {
            const int r = (int)(e / m);
            const int64_t j = e - (int64_t)r * m;
            dst[(i0 + r) * m + j] = srow[(int64_t)r * m + cperm[j]];
        }
        __syncthreads();
    }
}

size_t sweep_smem(int K, int fr, int fc) {
    const int FRP = (fr + 3) & ~3, FCP = (fc + 3) & ~3;
    K = (K + 3) & ~3;
    return sizeof(float) * (2 * (size_t)K * LD + (size_t)T * 2 * FRP + (size_t)T * 2 * FCP + 2 * (size_t)T * LDD);
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
    a.KP = h->KP;
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
    a.alpha_col = c.alpha_mode == 2 ? h->alpha_col : nullptr;
    a.missing = c.missing;
    a.ymiss = h->y16 ? 65535.f : -1.f;
    for (int i = 0; i < 4; i++) a.lam[i] = (float)c.lambda[i];
    a.a1 = (float)c.a1;
    a.a2 = (float)c.a2;
    a.damping = (float)c.damping;
    a.eps = (float)c.eps;
    a.clamp = (float)c.eta_clamp;
    a.Y = h->Yp;
    a.y16 = h->y16;
    a.yf32 = h->yf32;
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
    a.nbpart = h->nbpart;
    a.nbctr = h->nbctr;
    a.sigma = h->sigma;
    a.wait_ns = h->wait_ns > 0 ? (unsigned long long)h->wait_ns : 2000000000ull;
    a.kmap = nullptr;
    a.nk = h->per;
    a.rhoc = h->rhoc;
    a.rho1 = h->rho1;
    a.need = h->need;
    a.strip_done = h->strip_done;
    a.err = h->err;
    return a;
}

cudaError_t gmf_sweep_simt_attr(gmf_model* h) {
    return gmf_smem_limit((const void*)sweep_kernel, sweep_smem(h->K, h->fr, h->fc));
}

size_t gmf_sweep_simt_smem(const gmf_model* h) { return sweep_smem(h->K, h->fr, h->fc); }

cudaError_t gmf_simt_multi_attr(size_t smem) { return gmf_smem_limit((const void*)sweep_multi, smem); }

cudaError_t gmf_simt_launch_multi(const gmf_model* h0, const StepArgs* d_args, const int* d_order, int nmodels,
                                  size_t smem, int w, cudaStream_t st) {
    dim3 grid(h0->TJ, h0->TI, h0->per * nmodels);
    return gmf_launch_pdl(sweep_multi, grid, dim3(GMF_THREADS), smem, st, d_args, d_order, h0->per, w);
}

cudaError_t gmf_launch_sweep_simt(gmf_model* h, const StepArgs& a, int w, cudaStream_t st) {
    const size_t smem = sweep_smem(h->K, h->fr, h->fc);
    dim3 grid(h->TJ, h->TI, a.nk);
    const cudaError_t e = gmf_launch_pdl(sweep_kernel, grid, dim3(GMF_THREADS), smem, st, a, w);
    return e;
}

cudaError_t gmf_launch_sum_parts(const double* part, int count, double* out, cudaStream_t st) {
    sum_parts_kernel<<<1, GMF_THREADS, 0, st>>>(part, count, out);
    return cudaGetLastError();
}

// Mixed-precision handles take eta from the tensor cores (deviance_tc) unless
// GMF_FLAG_SIMT_DEVIANCE asks for this kernel (FP32 eta on the CUDA cores).
cudaError_t gmf_launch_deviance(gmf_model* h, double* d_out, cudaStream_t st) {
    if (gmf_tc_deviance_ok(h)) return gmf_tc_launch_deviance(h, d_out, st);
    StepArgs a = gmf_make_args(h);
    dim3 grid((unsigned)((h->m + T - 1) / T), (unsigned)((h->n + T - 1) / T));
    const size_t smem = sizeof(float) * 2 * (size_t)h->KP * LD;
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

int gmf_gather_host_ok(int y16, int64_t m) {
    const int64_t rb = m * (y16 ? 2 : 4);
    return rb % 16 == 0 && rb <= 48 * 1024;
}

// One CTA per SM (fewer reach only ~80 % of the link's rate), two rows per
// round: up to 16 KB of shared memory and 26 registers a thread, so that the
// CTAs share SMs with the block-step kernels running at the same time.
cudaError_t gmf_launch_gather_host(const void* src, void* dst, int y16, int64_t n, int64_t m, const int* rperm,
                                   const int* cperm, cudaStream_t st) {
    const int64_t rb = m * (y16 ? 2 : 4);
    const int rows = (int)std::max<int64_t>(1, std::min<int64_t>(2, 16384 / rb));
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = (int)std::min<int64_t>((n + rows - 1) / rows, nsm);
    const size_t smem = (size_t)rows * (size_t)rb;
    if (y16)
        gather_host_kernel<unsigned short><<<blocks, GH_THREADS, smem, st>>>(
            (const unsigned short*)src, (unsigned short*)dst, n, m, rperm, cperm, rows);
    else
        gather_host_kernel<int><<<blocks, GH_THREADS, smem, st>>>((const int*)src, (int*)dst, n, m, rperm, cperm,
                                                                  rows);
    return cudaGetLastError();
}

cudaError_t gmf_launch_permute_w(const float* src, float* dst, int64_t n, int64_t m, const int* rperm,
                                 const int* cperm, cudaStream_t st) {
    const int blocks = (int)(n < 65535 ? n : 65535);
    permute_kernel<float><<<blocks, 256, 0, st>>>(src, dst, n, m, rperm, cperm);
    return cudaGetLastError();
}
