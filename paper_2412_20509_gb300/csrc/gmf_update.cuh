// Block geometry and the smoothed local update shared by the FP32 and
// tensor-core block-step kernels (eq. 12, eq. 14, App. B).
//
// A sweep is two launches. The tile kernel writes, per tile, its row partials
// (sum_j Ddot_ij R_jc, sum_j Dddot_ij R_jc^2 for the row-free columns c) and
// column partials to a per-tile slot (column-major: G(o, c) at slot[c*T + o],
// H(o, c) at slot[(nf + c)*T + o]) and the tile's NB moment sums. The update
// kernel then gives every 32-row slice of every row strip and column strip its
// own CTA: it sums the strip's slots in tile order and applies scale factor,
// penalty, damping, EMA and step to its rows (columns); its block 0 also
// updates the NB shape from the moment sums. Both kernels are launched with
// programmatic stream serialization and wait (griddepcontrol.wait) for the
// launch before them to complete before they touch what it writes: the tile
// kernel before it reads the parameters (its prologue and count-tile loads
// overlap the previous update), the update kernel before it reads the
// partials (its slice state is loaded before). A tile kernel lets its update
// launch start (griddepcontrol.launch_dependents) only after its own wait, so
// an update never starts while the previous update is still writing.
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

// The same block from its moving strip j (the row chunk, or the column chunk
// when the roles swap), which the caller already knows: no load of sigma.
__device__ __forceinline__ BlockGeo block_geo_strip(const StepArgs& a, int j, int k) {
    const int rc = a.swap ? k : j, cc = a.swap ? j : k;
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

// Half unit deviance D(y, mu) / 2w (Table S1; App. B for the negative
// binomial) in FP32 for a positive count, written so that no difference of
// two large logarithms appears: with r1 = (y - mu)/mu and r2 = (y - mu)/(mu +
// alpha), log(y/mu) = log1p(r1) and log((y + alpha)/(mu + alpha)) = log1p(r2)
// while |r| < 1/2, which keeps y log(y/mu) - (y - mu) accurate when y and mu
// are large and close. e = log mu (the clamped eta).
__device__ __forceinline__ float half_dev_ratio(bool nb, float y, float e, float mu, float alpha) {
    const float r1 = (y - mu) / mu;
    const float l1 = fabsf(r1) < 0.5f ? log1pf(r1) : logf(y) - e;
    if (!nb) return y * l1 - (y - mu);
    const float r2 = (y - mu) / (mu + alpha);
    const float lma = mu > alpha ? e + log1pf(alpha / mu) : logf(alpha) + log1pf(mu / alpha);
    const float l2 = fabsf(r2) < 0.5f ? log1pf(r2) : logf(y + alpha) - lma;
    return y * l1 - (y + alpha) * l2;
}

// Unit deviance / 2 without branches on y (every lane of a warp takes the same path):
//   Poisson  y (log y - eta) - (y - mu)
//   NB       y (log y - eta) - (y + a)(log(y + a) - log a - log1p(mu / a)),
// the y log y term zero at y = 0, so a zero count (most entries) is exactly a log1p(mu / a). log y and
// log(y + a) come from per-CTA tables for y < 256. Near mu = y the logarithms cancel: the rounding is
// ~6e-8 (y + a) log(y + a) per entry, ~1e-7 of a whole matrix's deviance. The form takes log mu = eta
// but mu itself from exp(eta), so an error in mu enters at first order (as mu times its relative error):
// mu comes from the accurate expf, whose error is a fraction of an ulp without a common sign. (The fast
// exponential scales eta by a rounded log2(e) and carries a relative bias of ~1e-8 |eta|, which at
// counts of a few hundred moved whole-matrix deviances by 4e-5.) Counts of 32 and more take the ratio
// form instead (half_dev_ratio: log1p of the relative residual), which keeps y log(y/mu) - (y - mu)
// accurate when y and mu are large and close; they are rare in count data, so the branch seldom
// splits a warp.
__device__ __forceinline__ float half_dev_tab(bool nb, float y, float e, float mu, float alpha, float la,
                                              const float* tlog, const float* tloga) {
    if (y >= 32.f) return half_dev_ratio(nb, y, e, mu, alpha);
    const int yi = (int)y;
    float ly, lya;
    if (yi < 256) {
        ly = tlog[yi];
        lya = tloga[yi];
    } else {
        ly = logf(y);
        lya = logf(y + alpha);
    }
    const float t1 = yi > 0 ? y * (ly - e) : 0.f;
    return nb ? t1 - (y + alpha) * ((lya - la) - log1pf(__fdividef(mu, alpha))) : t1 - (y - mu);
}

// ---- the other families of Table S1 (GMF_GAUSSIAN .. GMF_INVGAUSS): identity
// link (Gaussian), logit (Bernoulli), log (Gamma, inverse Gaussian); phi is
// the dispersion (1 for the Bernoulli).

// The family's scalar is estimated once per sweep: the NB shape by moments,
// the dispersion of the Gaussian, Gamma and inverse Gaussian by Pearson (App. B).
__host__ __device__ __forceinline__ bool scalar_estimated(int family, int alpha_mode) {
    return alpha_mode == 1 && (family == GMF_NEGBIN || family == GMF_GAUSSIAN || family == GMF_GAMMA ||
                               family == GMF_INVGAUSS);
}

// An unobserved entry (cfg.missing): the dtype's marker count, or NaN in float32 responses.
__device__ __forceinline__ bool y_missing(const StepArgs& a, float y) {
    return a.missing && (a.yf32 ? y != y : y == a.ymiss);
}

// Inverse link at the clamped linear predictor e.
__device__ __forceinline__ float glm_mean(int fam, float e) {
    if (fam == GMF_GAUSSIAN) return e;
    if (fam == GMF_BINOMIAL) return 1.f / (1.f + expf(-e));
    return expf(e);
}

// Variance function nu(mu).
__device__ __forceinline__ float glm_variance(int fam, float mu) {
    if (fam == GMF_GAUSSIAN) return 1.f;
    if (fam == GMF_BINOMIAL) return mu * (1.f - mu);
    return fam == GMF_GAMMA ? mu * mu : mu * mu * mu;
}

// Ddot / w = (y - mu) / (phi nu g') and Dddot / w = 1 / (phi nu g'^2) of Sec. 3 in closed form.
__device__ __forceinline__ void glm_derivs(int fam, float y, float mu, float phi, float& d1, float& d2) {
    if (fam == GMF_GAUSSIAN) {
        d1 = (y - mu) / phi;
        d2 = 1.f / phi;
    } else if (fam == GMF_BINOMIAL) {
        d1 = y - mu;
        d2 = mu * (1.f - mu);
    } else if (fam == GMF_GAMMA) {
        d1 = (y - mu) / (phi * mu);
        d2 = 1.f / phi;
    } else {
        d1 = (y - mu) / (phi * mu * mu);
        d2 = 1.f / (phi * mu);
    }
}

// r - log1p(r) without cancellation: its Taylor series for |r| < 1/4 (14 terms,
// truncation below 1e-8 relative), else the difference.
__device__ __forceinline__ float r_minus_log1p(float r) {
    if (fabsf(r) >= 0.25f) return r - log1pf(r);
    float s = 1.f / 14.f;
#pragma unroll
    for (int k = 13; k >= 2; k--) s = 1.f / (float)k - r * s;
    return r * r * s;
}

// log(1 + e^x) for any x.
__device__ __forceinline__ float softplus_f(float x) { return fmaxf(x, 0.f) + log1pf(expf(-fabsf(x))); }

// x log x, 0 at x = 0.
__device__ __forceinline__ float xlogx_f(float x) { return x > 0.f ? x * logf(x) : 0.f; }

// Unit deviance D(y, mu) / w of Table S1 (not divided by phi); e = the clamped eta.
__device__ __forceinline__ float glm_unit_dev(int fam, float y, float e, float mu) {
    if (fam == GMF_GAUSSIAN) return (y - mu) * (y - mu);
    if (fam == GMF_BINOMIAL)  // log mu = -softplus(-e), log(1 - mu) = -softplus(e)
        return 2.f * (xlogx_f(y) + xlogx_f(1.f - y) + y * softplus_f(-e) + (1.f - y) * softplus_f(e));
    if (fam == GMF_GAMMA) return 2.f * r_minus_log1p((y - mu) / mu);
    return (y - mu) * (y - mu) / (y * mu * mu);
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

// Programmatic dependent launch: wait for the preceding launch in the stream
// to complete and its writes to be visible (a no-op without one), and let the
// next launch start early.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Asynchronous 4-byte global -> shared copy (sm_80 cp.async).
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Moment sums of one tile for the NB shape update (App. B), written to the
// tile's slot of nbpart. Every thread of the CTA calls this.
template <int NT>
__device__ __forceinline__ void tile_moments(const StepArgs& a, int k, int ti, int tj, float s1, float s2) {
    __shared__ float red[NT / 32];
    if (scalar_estimated(a.family, a.alpha_mode)) {
        const float S1 = block_sum_f<NT>(s1, red);
        const float S2 = block_sum_f<NT>(s2, red);
        if (threadIdx.x == 0) {
            const int cta = (k * a.TI + ti) * a.TJ + tj;
            a.nbpart[2 * cta] = (double)S1;
            a.nbpart[2 * cta + 1] = (double)S2;
        }
    }
}

// Update of one slice: the rows [first, first + nr) of L (row side) or of R
// (column side), nf free values each, which are rows [o_begin, o_begin + nr)
// of their strip's tiles. The slice's parameter rows, smoothed derivatives and
// visit counts are contiguous in global memory: they are loaded (L2, coalesced)
// BEFORE griddepcontrol.wait, since the tile launch this update follows only
// reads them and the update launch before it has completed (the tile launch
// lets this launch start only after its own wait). The partial slots written
// by that tile launch are read after the wait and summed in slot order. The
// update runs in shared memory (stage); results go back with coalesced stores
// (whole parameter rows: the fixed columns are written back unchanged). Items
// (o, c) go to threads c-major so that the partial loads coalesce. Every
// thread of the CTA calls this.
template <int NT, int IB, int PF>
__device__ __forceinline__ void slice_update(const StepArgs& a, const float* __restrict__ part, size_t slot_stride,
                                             int nslots, int T, int o_begin, int nr, int nf, int64_t first,
                                             bool rowside, float scale, float rhoc_blk, float* stage) {
    const int tid = threadIdx.x;
    const int KP = a.KP, KS = a.KP + 1;  // staged row stride (odd: no bank conflicts)
    const int NS = nf | 1;               // staged derivative stride
    float* P = rowside ? a.L : a.R;
    float* Gb = rowside ? a.GbR : a.GbC;
    float* Hb = rowside ? a.HbR : a.HbC;
    int* cnt = rowside ? a.cntR : a.cntC;
    float* sP = stage;
    float* sG = sP + nr * KS;
    float* sH = sG + nr * NS;
    int* sC = (int*)(sH + nr * NS);
    // slice state -> registers (PF values of each array per thread, the rest later)
    const int nP = nr * KP, nG = nr * nf;
    float rp[PF], rg[PF], rh[PF];
    int rcn = 0;
#pragma unroll
    for (int u = 0; u < PF; u++) {
        const int e = tid + u * NT;
        rp[u] = e < nP ? __ldcg(P + first * KP + e) : 0.f;
        rg[u] = e < nG ? __ldcg(Gb + first * nf + e) : 0.f;
        rh[u] = e < nG ? __ldcg(Hb + first * nf + e) : 0.f;
    }
    if (tid < nr) rcn = __ldcg(cnt + first + tid);

    grid_dependency_wait();

    const int total = nr * nf;
    const int iters = (total + NT * IB - 1) / (NT * IB);  // the same for every thread
    for (int it = 0; it < iters; it++) {
        float sg[IB], sh[IB];
        int oo[IB], cc[IB];
        bool ok[IB];
#pragma unroll
        for (int b = 0; b < IB; b++) {
            const int e = it * NT * IB + b * NT + tid;
            ok[b] = e < total;
            cc[b] = ok[b] ? e / nr : 0;
            oo[b] = ok[b] ? e - cc[b] * nr : 0;
            sg[b] = sh[b] = 0.f;
        }
        for (int u0 = 0; u0 < nslots; u0 += 4) {
            float gv[IB][4], hv[IB][4];
#pragma unroll
            for (int b = 0; b < IB; b++)
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const bool l = ok[b] && u0 + u < nslots;
                    const float* src = part + (size_t)(u0 + u) * slot_stride + (size_t)cc[b] * T + o_begin + oo[b];
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
        if (it == 0) {
            // slice state: registers, then whatever did not fit, into shared memory
#pragma unroll
            for (int u = 0; u < PF; u++) {
                const int e = tid + u * NT;
                if (e < nP) sP[(e / KP) * KS + e % KP] = rp[u];
                if (e < nG) {
                    sG[(e / nf) * NS + e % nf] = rg[u];
                    sH[(e / nf) * NS + e % nf] = rh[u];
                }
            }
            for (int e = tid + PF * NT; e < nP; e += NT) sP[(e / KP) * KS + e % KP] = __ldcg(P + first * KP + e);
            for (int e = tid + PF * NT; e < nG; e += NT) {
                sG[(e / nf) * NS + e % nf] = __ldcg(Gb + first * nf + e);
                sH[(e / nf) * NS + e % nf] = __ldcg(Hb + first * nf + e);
            }
            if (tid < nr) sC[tid] = rcn;
            __syncthreads();
        }
#pragma unroll
        for (int b = 0; b < IB; b++) {
            if (ok[b]) {
                const int o = oo[b], c = cc[b];
                const int col = rowside ? 1 + a.p + c : (c < a.p ? 1 + c : 1 + a.q + c);
                const float lam = rowside ? (c < a.q ? a.lam[1] : a.lam[2]) : (c < a.p ? a.lam[0] : a.lam[3]);
                const float rc = a.bias_corr ? rhoc_blk * bias_visit(a.a1, a.a2, sC[o] + 1) : rhoc_blk;
                smoothed_step(sP[o * KS + col], sG[o * NS + c], sH[o * NS + c], sg[b], sh[b], scale, lam, a, rc);
            }
        }
    }
    __syncthreads();
    for (int e = tid; e < nP; e += NT) {
        const int r = e / KP;
        P[first * KP + e] = sP[r * KS + (e - r * KP)];
    }
    for (int e = tid; e < nG; e += NT) {
        const int r = e / nf;
        Gb[first * nf + e] = sG[r * NS + (e - r * nf)];
        Hb[first * nf + e] = sH[r * NS + (e - r * nf)];
    }
    for (int e = tid; e < nr; e += NT) cnt[first + e] = sC[e] + 1;
}

// Work units of the update kernel for one model: per block k of the sweep, the
// TI row strips and the TJ column strips of tile edge T, each in slices of SR
// rows (columns).
constexpr int UPD_NT = 128;  // threads per update CTA
constexpr int UPD_SR = 32;   // rows (columns) per slice

__host__ __device__ __forceinline__ int update_units(int per, int TI, int TJ, int T) {
    return per * (TI + TJ) * ((T + UPD_SR - 1) / UPD_SR);
}

// Floats of shared memory one update CTA stages: UPD_SR rows of the widest side.
__host__ __device__ __forceinline__ int update_stage_floats(int KP, int fr, int fc) {
    const int nf = fr > fc ? fr : fc;
    return UPD_SR * (KP + 1 + 2 * (nf | 1) + 1);
}

// One unit of the update launch. Everything before grid_dependency_wait()
// reads only data that the preceding tile launch does not write.
__device__ __forceinline__ void update_unit(const StepArgs& a, int w, int T, int unit, float* stage) {
    const int nsl = (T + UPD_SR - 1) / UPD_SR;
    const int per_block = (a.TI + a.TJ) * nsl;
    const int kz = unit / per_block;
    const int k = block_of_slot(a, kz);
    const int rem = unit - kz * per_block;
    const BlockGeo g = block_geo(a, w, k);
    const int nTI = (int)((g.nI + T - 1) / T), nTJ = (int)((g.mJ + T - 1) / T);
    const float rhoc_blk = a.rhoc[w * a.per + k];
    constexpr int PF = 4;  // prefetched values per thread and array (UPD_SR x 16 of P with 128 threads)
    if (rem < a.TI * nsl) {  // row strip ti of block k
        const int ti = rem / nsl, o_begin = (rem - ti * nsl) * UPD_SR;
        const int nstrip = ti < nTI ? (int)min((int64_t)T, g.nI - (int64_t)ti * T) : 0;
        if (o_begin >= nstrip) {
            grid_dependency_wait();
            return;
        }
        slice_update<UPD_NT, 4, PF>(a, a.partR + (size_t)((k * a.TI + ti) * a.TJ) * T * 2 * a.fr,
                                    (size_t)T * 2 * a.fr, nTJ, T, o_begin, min(UPD_SR, nstrip - o_begin), a.fr,
                                    g.r0 + (int64_t)ti * T + o_begin, true, (float)a.m / (float)g.mJ, rhoc_blk,
                                    stage);
    } else {  // column strip tj of block k
        const int r2 = rem - a.TI * nsl;
        const int tj = r2 / nsl, o_begin = (r2 - tj * nsl) * UPD_SR;
        const int nstrip = tj < nTJ ? (int)min((int64_t)T, g.mJ - (int64_t)tj * T) : 0;
        if (o_begin >= nstrip) {
            grid_dependency_wait();
            return;
        }
        slice_update<UPD_NT, 4, PF>(a, a.partC + (size_t)((k * a.TJ + tj) * a.TI) * T * 2 * a.fc,
                                    (size_t)T * 2 * a.fc, nTI, T, o_begin, min(UPD_SR, nstrip - o_begin), a.fc,
                                    g.c0 + (int64_t)tj * T + o_begin, false, (float)a.n / (float)g.nI, rhoc_blk,
                                    stage);
    }
}

// ---- the update launch of the tensor-core path. Its tile kernel writes each
// tile's partials column-major, slot[c * T + o] (G) and slot[(nf + c) * T + o]
// (H), as the FP32 path does. One CTA per 32-row slice of a strip: lane r of
// warp g owns row r of the slice and the free columns 2g, 2g+1 (a narrower
// block takes the column groups in passes), so every load of a slot is one
// coalesced row of 32 floats. Each thread loads its
// parameters and smoothed derivatives before griddepcontrol.wait, then adds
// the strip's slots in tile order (the same FP32 additions as slice_update, so
// both give the same bits) with the loads of four slots in flight.
constexpr int UTC_SR = 32;   // rows (columns) per slice

constexpr int UTC_CG = 2;    // free columns per thread
constexpr int UTC_SIF = 4;   // slots whose loads are in flight together
__host__ __device__ __forceinline__ int utc_groups(int fr, int fc) {
    return (fr > fc ? fr + UTC_CG - 1 : fc + UTC_CG - 1) / UTC_CG;
}
__host__ __device__ __forceinline__ int utc_units(int nk, int TI, int TJ, int T) {
    return nk * (TI + TJ) * ((T + UTC_SR - 1) / UTC_SR);
}

template <bool PASSES>
__device__ __forceinline__ void slice_update_tc(const StepArgs& a, const float* __restrict__ part, size_t slot_stride,
                                                int nslots, int T, int o_begin, int nr, int nf, int64_t first,
                                                bool rowside, float scale, float rhoc_blk, int* s_cnt) {
    const int r = threadIdx.x & 31, wq = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int G = (nf + UTC_CG - 1) / UTC_CG;  // column groups of this side
    const int npass = PASSES ? (G + nw - 1) / nw : 1;  // PASSES = false: a warp per group (the update launch)
    float* P = rowside ? a.L : a.R;
    float* Gb = rowside ? a.GbR : a.GbC;
    float* Hb = rowside ? a.HbR : a.HbC;
    int* cnt = rowside ? a.cntR : a.cntC;
    const int64_t row = first + r;
    if (wq == 0 && r < nr) s_cnt[r] = __ldcg(cnt + row);
    for (int pass = 0; pass < npass; pass++) {
        const int c0 = UTC_CG * (wq + pass * nw);
        const bool act = r < nr && c0 < nf;
        const int nc = act ? min(UTC_CG, nf - c0) : 0;
        int col[UTC_CG];
        float th[UTC_CG], gb[UTC_CG], hb[UTC_CG];
#pragma unroll
        for (int u = 0; u < UTC_CG; u++) {
            const int c = c0 + u;
            col[u] = rowside ? 1 + a.p + c : (c < a.p ? 1 + c : 1 + a.q + c);
            th[u] = gb[u] = hb[u] = 0.f;
            if (u < nc) {
                th[u] = __ldcg(P + row * a.KP + col[u]);
                gb[u] = __ldcg(Gb + row * nf + c);
                hb[u] = __ldcg(Hb + row * nf + c);
            }
        }
        if (pass == 0) grid_dependency_wait();

        float gs[UTC_CG] = {}, hs[UTC_CG] = {};
        if (act) {
            const float* base = part + o_begin + r;
            for (int t0 = 0; t0 < nslots; t0 += UTC_SIF) {
                float gv[UTC_SIF][UTC_CG], hv[UTC_SIF][UTC_CG];
#pragma unroll
                for (int v = 0; v < UTC_SIF; v++)
#pragma unroll
                    for (int u = 0; u < UTC_CG; u++) {
                        const bool l = t0 + v < nslots && u < nc;
                        const float* sp = base + (size_t)(t0 + v) * slot_stride + (size_t)(c0 + u) * T;
                        gv[v][u] = l ? __ldcg(sp) : 0.f;
                        hv[v][u] = l ? __ldcg(sp + (size_t)nf * T) : 0.f;
                    }
#pragma unroll
                for (int v = 0; v < UTC_SIF; v++)
                    if (t0 + v < nslots)
#pragma unroll
                        for (int u = 0; u < UTC_CG; u++) {
                            gs[u] += gv[v][u];
                            hs[u] += hv[v][u];
                        }
            }
        }
        if (pass == 0) __syncthreads();  // the slice's visit counts are in shared memory
#pragma unroll
        for (int u = 0; u < UTC_CG; u++) {
            if (u < nc) {
                const int c = c0 + u;
                const float lam = rowside ? (c < a.q ? a.lam[1] : a.lam[2]) : (c < a.p ? a.lam[0] : a.lam[3]);
                const float rc = a.bias_corr ? rhoc_blk * bias_visit(a.a1, a.a2, s_cnt[r] + 1) : rhoc_blk;
                smoothed_step(th[u], gb[u], hb[u], gs[u], hs[u], scale, lam, a, rc);
                P[row * a.KP + col[u]] = th[u];
                Gb[row * nf + c] = gb[u];
                Hb[row * nf + c] = hb[u];
            }
        }
    }
    if (wq == 0 && r < nr) cnt[row] = s_cnt[r] + 1;
}

// One unit of the tensor-core update launch (tile edge T = 128). strip >= 0:
// the block's moving strip, known to the caller. PASSES: the CTA may have
// fewer warps than the widest side has column groups (persistent kernels).
template <bool PASSES = false>
__device__ __forceinline__ void update_unit_tc(const StepArgs& a, int w, int T, int unit, int* s_cnt,
                                               int strip = -1) {
    const int nsl = (T + UTC_SR - 1) / UTC_SR;
    const int per_block = (a.TI + a.TJ) * nsl;
    const int kz = unit / per_block;
    const int k = block_of_slot(a, kz);
    const int rem = unit - kz * per_block;
    const BlockGeo g = strip >= 0 ? block_geo_strip(a, strip, k) : block_geo(a, w, k);
    const int nTI = (int)((g.nI + T - 1) / T), nTJ = (int)((g.mJ + T - 1) / T);
    const float rhoc_blk = a.rhoc[w * a.per + k];
    if (rem < a.TI * nsl) {  // row strip ti of block k
        const int ti = rem / nsl, o_begin = (rem - ti * nsl) * UTC_SR;
        const int nstrip = ti < nTI ? (int)min((int64_t)T, g.nI - (int64_t)ti * T) : 0;
        if (o_begin >= nstrip) {
            grid_dependency_wait();
            return;
        }
        const size_t ss = (size_t)T * 2 * a.fr;
        slice_update_tc<PASSES>(a, a.partR + (size_t)((k * a.TI + ti) * a.TJ) * ss, ss, nTJ, T, o_begin,
                        min(UTC_SR, nstrip - o_begin), a.fr, g.r0 + (int64_t)ti * T + o_begin, true,
                        (float)a.m / (float)g.mJ, rhoc_blk, s_cnt);
    } else {  // column strip tj of block k
        const int r2 = rem - a.TI * nsl;
        const int tj = r2 / nsl, o_begin = (r2 - tj * nsl) * UTC_SR;
        const int nstrip = tj < nTJ ? (int)min((int64_t)T, g.mJ - (int64_t)tj * T) : 0;
        if (o_begin >= nstrip) {
            grid_dependency_wait();
            return;
        }
        const size_t ss = (size_t)T * 2 * a.fc;
        slice_update_tc<PASSES>(a, a.partC + (size_t)((k * a.TJ + tj) * a.TI) * ss, ss, nTI, T, o_begin,
                        min(UTC_SR, nstrip - o_begin), a.fc, g.c0 + (int64_t)tj * T + o_begin, false,
                        (float)a.n / (float)g.nI, rhoc_blk, s_cnt);
    }
}

// NB shape or dispersion: moment (Pearson) sums of all tiles of the sweep, in
// tile order, then one smoothed update per sweep (App. B). One thread.
__device__ __forceinline__ void nb_shape_update(const StepArgs& a, int w) {
    if (!scalar_estimated(a.family, a.alpha_mode)) return;
    const int total = a.TJ * a.TI * a.per;
    double T1 = 0.0, T2 = 0.0;
    for (int c = 0; c < total; c++) {
        T1 += __ldcg(a.nbpart + 2 * c);
        T2 += __ldcg(a.nbpart + 2 * c + 1);
    }
    if (a.family != GMF_NEGBIN) {
        // Pearson sum and observed entries of the sweep, scaled to the whole
        // matrix over the residual degrees of freedom
        const double nm = (double)a.n * (double)a.m;
        const double dof = nm - (double)a.m * a.p - (double)a.n * a.q - (double)(a.n + a.m) * a.d - 1.0;
        if (T2 > 0.0 && dof > 0.0) {
            float phat = (float)((nm / T2) * T1 / dof);
            if (phat < a.eps) phat = a.eps;
            const float rf = a.rho1[w];
            *a.alpha = (1.f - rf) * (*a.alpha) + rf * phat;
        }
        return;
    }
    if (T2 > 0.0) {
        float ahat = (float)(T1 / T2);
        if (ahat < a.eps) ahat = a.eps;
        const float rf = a.rho1[w];
        *a.alpha = (1.f - rf) * (*a.alpha) + rf * ahat;
    }
}

}  // namespace gmfdev
