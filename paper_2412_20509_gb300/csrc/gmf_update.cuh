// Block geometry, arrival counting and the smoothed local update shared by the
// FP32 and tensor-core block-step kernels (eq. 12, eq. 14, App. B).
//
// Each tile kernel writes its row partials (sum_j Ddot_ij R_jc, sum_j Dddot_ij
// R_jc^2 for the row-free columns c) and column partials to a per-tile slot
// (column-major: G(o, c) at slot[c*T + o], H(o, c) at slot[(nf + c)*T + o]),
// then calls tile_arrive_update(): an arrival counter per row strip and per
// column strip elects the last CTA of the strip, which sums the strip's
// partials in tile order and applies scale factor, penalty, damping, EMA and
// step to its rows (columns). Every reader of those parameters in this sweep
// has arrived before the update starts, so it cannot race with a reader, and
// no CTA ever waits on another.
#pragma once

#include "gmf_internal.cuh"

namespace gmfdev {

struct BlockGeo {
    int64_t r0, nI, c0, mJ;
};

// Block k of sweep w (Algorithm 1 schedule; roles swap when r < s).
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

template <int NT>
__device__ __forceinline__ float block_sum_f(float v, float* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    float s = 0.f;
#pragma unroll
    for (int u = 0; u < NT / 32; u++) s += red[u];  // fixed order: every thread the same value
    return s;
}

// (1 - (1-a2)^k) / (1 - (1-a1)^k): per-visit bias correction, k >= 1.
__device__ __forceinline__ float bias_visit(float a1, float a2, int visits) {
    const float k = (float)visits;
    return (1.f - expf(k * log1pf(-a2))) / (1.f - expf(k * log1pf(-a1)));
}

// Smoothed local step of eq. 12 / eq. 14 for one free parameter.
__device__ __forceinline__ void smoothed_step(float& theta, float& gbar, float& hbar, float gsum, float hsum,
                                              float scale, float lam, const StepArgs& a, float rho_c) {
    const float gh = -scale * gsum + lam * theta;
    const float hh = scale * hsum + lam + a.damping;
    gbar = (1.f - a.a1) * gbar + a.a1 * gh;
    hbar = (1.f - a.a2) * hbar + a.a2 * hh;
    theta = theta - rho_c * (gbar / hbar);
    if (!isfinite(theta)) atomicOr(a.err, GMF_DEVERR_NONFINITE);
}

// Update of one strip (rows of a row strip, or columns of a column strip).
// Per-tile partial slots hold G(o, c) at slot[c*T + o] and H(o, c) at
// slot[(nf + c)*T + o]; the nslots slots of the strip are nslot_stride apart
// and are summed in slot order. Items (o, c) go to threads c-major so that the
// partial loads coalesce; each thread issues the loads of IB items at once.
template <int T, int NT, int IB>
__device__ __forceinline__ void strip_update(const StepArgs& a, const float* __restrict__ part, size_t slot_stride,
                                             int nslots, int no, int nf, int64_t first, bool rowside, float scale,
                                             const float* s_rc) {
    const int total = no * nf;
    for (int e0 = threadIdx.x; e0 < total; e0 += NT * IB) {
        float* pth[IB];
        float* pgb[IB];
        float* phb[IB];
        float th[IB], gb[IB], hb[IB], sg[IB], sh[IB], lam[IB];
        int oo[IB], cc[IB];
        bool ok[IB];
#pragma unroll
        for (int b = 0; b < IB; b++) {
            const int e = e0 + b * NT;
            ok[b] = e < total;
            const int c = ok[b] ? e / no : 0, o = ok[b] ? e - c * no : 0;
            oo[b] = o;
            cc[b] = c;
            const int64_t x = first + o;
            if (rowside) {
                pth[b] = a.L + x * a.KP + 1 + a.p + c;
                pgb[b] = a.GbR + x * a.fr + c;
                phb[b] = a.HbR + x * a.fr + c;
                lam[b] = c < a.q ? a.lam[1] : a.lam[2];
            } else {
                pth[b] = a.R + x * a.KP + (c < a.p ? 1 + c : 1 + a.q + c);
                pgb[b] = a.GbC + x * a.fc + c;
                phb[b] = a.HbC + x * a.fc + c;
                lam[b] = c < a.p ? a.lam[0] : a.lam[3];
            }
            th[b] = ok[b] ? *pth[b] : 0.f;
            gb[b] = ok[b] ? *pgb[b] : 0.f;
            hb[b] = ok[b] ? *phb[b] : 1.f;
            sg[b] = sh[b] = 0.f;
        }
        for (int u0 = 0; u0 < nslots; u0 += 4) {
            float gv[IB][4], hv[IB][4];
#pragma unroll
            for (int b = 0; b < IB; b++)
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const bool l = ok[b] && u0 + u < nslots;
                    const float* src = part + (size_t)(u0 + u) * slot_stride + (size_t)cc[b] * T + oo[b];
                    gv[b][u] = l ? __ldcg(src) : 0.f;
                    hv[b][u] = l ? __ldcg(src + (size_t)nf * T) : 0.f;
                }
#pragma unroll
            for (int b = 0; b < IB; b++)
#pragma unroll
                for (int u = 0; u < 4; u++)
                    if (u0 + u < nslots) {
                        sg[b] += gv[b][u];
                        sh[b] += hv[b][u];
                    }
        }
#pragma unroll
        for (int b = 0; b < IB; b++) {
            if (ok[b]) {
                smoothed_step(th[b], gb[b], hb[b], sg[b], sh[b], scale, lam[b], a, s_rc[oo[b]]);
                *pth[b] = th[b];
                *pgb[b] = gb[b];
                *phb[b] = hb[b];
            }
        }
    }
}

// Arrival, strip updates and the once-per-sweep NB shape update for the tile
// (ti, tj) of block k of sweep w, tile edge T, NT threads, IB strip items in
// flight per thread. Must be called by every thread of every CTA of the launch
// (inactive CTAs included).
template <int T, int NT, int IB>
__device__ void tile_arrive_update(const StepArgs& a, int w, int k, int ti, int tj, const BlockGeo& g, int nTI,
                                   int nTJ, bool active, float s1, float s2, float alpha) {
    __shared__ int s_flag[3];
    __shared__ int s_visits[T];
    __shared__ float s_rc[T];
    __shared__ float red[NT / 32];
    const int tid = threadIdx.x;
    const float rhoc_blk = a.rhoc[w * a.per + k];
    const int64_t row0 = g.r0 + (int64_t)ti * T, col0 = g.c0 + (int64_t)tj * T;
    const int nr = active ? (int)min((int64_t)T, g.nI - (int64_t)ti * T) : 0;
    const int nc = active ? (int)min((int64_t)T, g.mJ - (int64_t)tj * T) : 0;

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

    if (s_flag[0]) {  // rows [row0, row0 + nr) of block k
        __threadfence();
        if (tid < nr) {
            const int v = a.cntR[row0 + tid] + 1;
            s_visits[tid] = v;
            s_rc[tid] = a.bias_corr ? rhoc_blk * bias_visit(a.a1, a.a2, v) : rhoc_blk;
        }
        __syncthreads();
        const float scale = (float)a.m / (float)g.mJ;
        strip_update<T, NT, IB>(a, a.partR + (size_t)((k * a.TI + ti) * a.TJ) * T * 2 * a.fr, (size_t)T * 2 * a.fr, nTJ,
                            nr, a.fr, row0, true, scale, s_rc);
        __syncthreads();
        if (tid < nr) a.cntR[row0 + tid] = s_visits[tid];
        if (tid == 0) a.ctrR[k * a.TI + ti] = 0u;
    }
    if (s_flag[1]) {  // columns [col0, col0 + nc) of block k
        __threadfence();
        __syncthreads();
        if (tid < nc) {
            const int v = a.cntC[col0 + tid] + 1;
            s_visits[tid] = v;
            s_rc[tid] = a.bias_corr ? rhoc_blk * bias_visit(a.a1, a.a2, v) : rhoc_blk;
        }
        __syncthreads();
        const float scale = (float)a.n / (float)g.nI;
        strip_update<T, NT, IB>(a, a.partC + (size_t)((k * a.TJ + tj) * a.TI) * T * 2 * a.fc, (size_t)T * 2 * a.fc, nTI,
                            nc, a.fc, col0, false, scale, s_rc);
        __syncthreads();
        if (tid < nc) a.cntC[col0 + tid] = s_visits[tid];
        if (tid == 0) a.ctrC[k * a.TJ + tj] = 0u;
    }

    // NB shape: moment sums pooled over the sweep, one update per sweep (App. B)
    if (a.family == GMF_NEGBIN && a.alpha_mode == 1) {
        const float S1 = block_sum_f<NT>(s1, red);
        const float S2 = block_sum_f<NT>(s2, red);
        const int cta = (k * a.TI + ti) * a.TJ + tj;
        if (tid == 0) {
            a.nbpart[2 * cta] = (double)S1;
            a.nbpart[2 * cta + 1] = (double)S2;
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            const unsigned total = (unsigned)(a.TJ * a.TI * a.per);  // CTAs of this model's sweep
            s_flag[2] = atomicAdd(a.ctrSweep, 1u) == total - 1;
        }
        __syncthreads();
        if (s_flag[2] && tid == 0) {
            __threadfence();
            const int total = a.TJ * a.TI * a.per;
            double T1 = 0.0, T2 = 0.0;
            for (int c = 0; c < total; c++) {
                T1 += __ldcg(a.nbpart + 2 * c);
                T2 += __ldcg(a.nbpart + 2 * c + 1);
            }
            if (T2 > 0.0) {
                float ahat = (float)(T1 / T2);
                if (ahat < a.eps) ahat = a.eps;
                const float rf = a.rho1[w];
                *a.alpha = (1.f - rf) * alpha + rf * ahat;
            }
            *a.ctrSweep = 0u;
        }
    }
}

}  // namespace gmfdev
