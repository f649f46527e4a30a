// Full deviance of mixed-precision handles on the tensor cores (Table S1; App.
// B for the negative binomial): gmf_deviance with eta from the block step's
// split-BF16 tcgen05 products.
#include <algorithm>

#include "gmf_tc_tile.cuh"

namespace {

using namespace gmfdev;
using namespace sm100;
using namespace gmftc;

// ---- full deviance on the tensor cores (Table S1; App. B). eta of every 128 x
// 128 tile of the whole (permuted) matrix comes from the block step's
// split-BF16 products (the same operands and MMAs), the unit deviances from
// TMEM in FP32. Persistent, 256 threads, two CTAs per SM, tiles c, c + G, ...
// for CTA c (a fixed assignment, so the sums are deterministic): while the
// epilogue of tile i runs, the counts of tile i + 1 are in flight (TMA into the
// second count buffer) and its eta MMAs run into the second TMEM accumulator;
// the operands of tile i + 1 are built once tile i's MMAs have completed. Per
// thread: one row of the tile and 64 columns, taken 8 at a time (a loop that is
// not unrolled: the unrolled 64-entry body did not fit the instruction cache),
// summed per 8 entries in FP32, the 8-entry sums with compensation per tile,
// the tiles in FP64; one FP64 value per CTA.

// log1p(t) for 0 <= t <= 1: the series log((1 + s)/(1 - s)) = 2 (s + s^3/3 +
// s^5/5 + ...) with s = t / (2 + t) <= 1/3 (Abramowitz and Stegun 4.1.27),
// truncated after s^15 (below 1e-8 relative): one reciprocal, eight FMAs.
__device__ __forceinline__ float log1p_01(float t) {
    const float s = __fdividef(t, 2.f + t), s2 = s * s;
    float p = 1.f / 15.f;
    p = fmaf(p, s2, 1.f / 13.f);
    p = fmaf(p, s2, 1.f / 11.f);
    p = fmaf(p, s2, 1.f / 9.f);
    p = fmaf(p, s2, 1.f / 7.f);
    p = fmaf(p, s2, 1.f / 5.f);
    p = fmaf(p, s2, 1.f / 3.f);
    return 2.f * fmaf(s * s2, p, s);
}

// log(1 + e^z) = max(z, 0) + log1p(e^-|z|), without a branch.
__device__ __forceinline__ float softplus_01(float z) { return fmaxf(z, 0.f) + log1p_01(expf(-fabsf(z))); }

// The ratio form for counts of 32 and more, out of line: rare, and large.
__device__ __noinline__ float half_dev_ratio_ool(bool nb, float y, float e, float alpha) {
    return half_dev_ratio(nb, y, e, expf(e), alpha);
}

// D / 2w of one entry for the scalar-shape NB and the Poisson. Below 32 the
// table holds (log y, log(y + alpha) - log alpha) (0 at y = 0), and with
// log1p(mu / alpha) = softplus(eta - log alpha) the NB form is
//   y (log y - eta) - (y + alpha)(log(y + alpha) - log alpha) + (y + alpha) softplus(eta - log alpha),
// exactly alpha log1p(mu / alpha) at y = 0; mu itself is not needed. Poisson:
// y (log y - eta) - (y - mu).
__device__ __forceinline__ float half_dev_tc(bool nb, float y, float e, float alpha, float la, const float2* tab) {
    if (y >= 32.f) return half_dev_ratio_ool(nb, y, e, alpha);
    const float2 t = tab[(int)y];
    const float t1 = y * (t.x - e);
    if (!nb) return t1 - y + expf(e);
    const float ya = y + alpha;
    return fmaf(ya, softplus_01(e - la), fmaf(-ya, t.y, t1));
}

constexpr int DTH = 256;

// Epilogue of one tile: the sum of 2 w D/2w over this thread's row i and its
// 64 columns (64 ch ..), from eta in TMEM at tacc and the counts at Ys; eight
// columns per step, summed in FP32, the 8-column sums with compensation.
template <bool Y16, bool GEN>
__device__ __forceinline__ float tile_deviance(const StepArgs& a, const uint8_t* Ys, uint32_t tacc, int q, int ch,
                                               int64_t row0, int64_t col0, int nr, int nc, bool nb, float alpha,
                                               float la, const float2* tab) {
    const int i = 32 * q + (threadIdx.x & 31);
    const bool row_ok = i < nr;
    const float* Wrow = (GEN && a.W) ? a.W + (row0 + i) * a.m + col0 : nullptr;
    float s = 0.f, comp = 0.f;
#pragma unroll 1
    for (int gq = 0; gq < 8; gq++) {
        const int j0 = 64 * ch + 8 * gq;
        uint32_t ev[8];
        tmem_ld8(tacc + ((uint32_t)(32 * q) << 16) + (uint32_t)j0, ev);
        float y[8];
        int yi[8];
        uint32_t big;  // nonzero when a count of the 8 is 32 or more
        if (Y16) {
            const uint4 u = *(const uint4*)(Ys + (j0 >> 6) * ATOM + sw128_off(i, (j0 & 63) * 2));
            const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int v = 0; v < 4; v++) {
                yi[2 * v] = (int)(uu[v] & 0xFFFFu);
                yi[2 * v + 1] = (int)(uu[v] >> 16);
            }
            big = (u.x | u.y | u.z | u.w) & 0xFFE0FFE0u;
        } else {
            const uint32_t byte = (uint32_t)(j0 & 31) * 4u;
            const int4 u0 = *(const int4*)(Ys + (j0 >> 5) * ATOM + sw128_off(i, byte));
            const int4 u1 = *(const int4*)(Ys + (j0 >> 5) * ATOM + sw128_off(i, byte + 16));
            yi[0] = u0.x; yi[1] = u0.y; yi[2] = u0.z; yi[3] = u0.w;
            yi[4] = u1.x; yi[5] = u1.y; yi[6] = u1.z; yi[7] = u1.w;
            big = (uint32_t)(u0.x | u0.y | u0.z | u0.w | u1.x | u1.y | u1.z | u1.w) & ~31u;
        }
#pragma unroll
        for (int v = 0; v < 8; v++) y[v] = (GEN && a.yf32) ? __int_as_float(yi[v]) : (float)yi[v];
        tmem_wait_ld();
        float g8 = 0.f;
        if (!GEN && big == 0u && row_ok && j0 + 8 <= nc) {
            // counts below 32 and every entry inside the tile (nearly all groups): no per-entry tests
#pragma unroll
            for (int v = 0; v < 8; v++) {
                const float e = fminf(fmaxf(__uint_as_float(ev[v]), -a.clamp), a.clamp);
                const float2 t = tab[yi[v]];
                const float t1 = y[v] * (t.x - e);
                if (nb) {
                    const float ya = y[v] + alpha;
                    g8 += fmaf(ya, softplus_01(e - la), fmaf(-ya, t.y, t1));
                } else {
                    g8 += t1 - y[v] + expf(e);
                }
            }
            g8 *= 2.f;
        } else {
#pragma unroll
        for (int v = 0; v < 8; v++) {
            const int j = j0 + v;
            const bool valid = row_ok && j < nc && !(GEN && y_missing(a, y[v]));
            const float e = fminf(fmaxf(__uint_as_float(ev[v]), -a.clamp), a.clamp);
            float hd;
            if (GEN && a.family >= GMF_GAUSSIAN) {
                hd = valid ? 0.5f * glm_unit_dev(a.family, y[v], e, glm_mean(a.family, e)) : 0.f;
            } else if (GEN && a.alpha_col) {
                const float aj = valid ? __ldg(a.alpha_col + col0 + j) : 1.f, mu = expf(e);
                hd = y[v] > 0.f ? half_dev_ratio_ool(nb, y[v], e, aj) : (nb ? aj * softplus_01(e - logf(aj)) : mu);
            } else {
                hd = half_dev_tc(nb, y[v], e, alpha, la, tab);
            }
            const float wv = (Wrow && valid) ? __ldg(Wrow + j) : 1.f;
            g8 += valid ? 2.f * wv * hd : 0.f;
        }
        }
        const float yk = g8 - comp;
        const float tk = s + yk;
        comp = (tk - s) - yk;
        s = tk;
    }
    return s;
}

// ST = 2: two count buffers and two TMEM accumulators (the next tile's counts
// and eta MMAs in flight during this tile's epilogue), two CTAs per SM. ST = 1:
// one of each and a serial tile loop, three CTAs per SM (16-bit counts and
// K <= 32), whose warps hide one another's waits.
template <bool Y16, bool GEN, int ST>
__global__ void __launch_bounds__(DTH, ST == 1 ? 3 : 2)
    deviance_tc(StepArgs a, TcLayout Lo, const __grid_constant__ CUtensorMap ymap, int ntj, int ntiles,
                double* part) {
    extern __shared__ __align__(1024) uint8_t smraw[];
    __shared__ uint64_t bars[3];  // counts of buffer 0 / 1, eta MMAs
    __shared__ uint32_t tmem_base;
    __shared__ float2 tab[256];  // (log v, log(v + alpha) - log alpha), v < 256
    __shared__ double red[DTH / 32];
    constexpr uint32_t TCOLS = ST == 1 ? 128u : 256u;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t* sm = smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u);
    const float alpha = *a.alpha;
    const float la = logf(alpha);
    tab[tid] = make_float2(tid > 0 ? logf((float)tid) : 0.f, tid > 0 ? logf((float)tid + alpha) - la : 0.f);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&bars[2], 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&tmem_base, TCOLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tb = tmem_base;
    const bool nb = a.family == GMF_NEGBIN;
    const int q = warp & 3, ch = warp >> 2;  // TMEM lanes 32q.., columns 64ch..64ch+63
    double total = 0.0;
    bool ok = true;
    // phases issued on / waited for at each mbarrier (at most one outstanding per
    // barrier): count buffers 0 and 1, eta MMAs
    int is0 = 0, is1 = 0, is2 = 0, wt0 = 0, wt1 = 0, wt2 = 0;
    const int G = gridDim.x;
    int t = blockIdx.x;
    auto tile_origin = [&](int tt, int64_t& row0, int64_t& col0, int& nr, int& nc) {
        const int ti = tt / ntj, tj = tt - ti * ntj;
        row0 = (int64_t)ti * TT;
        col0 = (int64_t)tj * TT;
        nr = (int)min((int64_t)TT, a.n - row0);
        nc = (int)min((int64_t)TT, a.m - col0);
    };
    if (ST == 1) {
        for (; t < ntiles; t += G) {
            int64_t row0, col0;
            int nr, nc;
            tile_origin(t, row0, col0, nr, nc);
            if (tid == 0) issue_counts(Lo, &ymap, sm, row0, col0, &bars[0]);
            is0++;
            build_operands<false>(a, Lo, sm, row0, col0, nr, nc);
            fence_proxy_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (tid == 0) issue_eta(Lo, sm, tb, &bars[2]);
            is2++;
            ok = cta_wait(&bars[2], (uint32_t)(wt2 & 1), a.err);
            wt2++;
            if (ok) {
                ok = cta_wait(&bars[0], (uint32_t)(wt0 & 1), a.err);
                wt0++;
            }
            if (!ok) break;
            tc_fence_after();
            total += (double)tile_deviance<Y16, GEN>(a, sm, tb, q, ch, row0, col0, nr, nc, nb, alpha, la, tab);
            // the counts, the operands and the accumulator are dead: the next tile may reuse them
            fence_proxy_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
        }
    } else {
        if (t < ntiles) {
            int64_t row0, col0;
            int nr, nc;
            tile_origin(t, row0, col0, nr, nc);
            if (tid == 0) issue_counts(Lo, &ymap, sm, row0, col0, &bars[0]);
            is0++;
            build_operands<false>(a, Lo, sm, row0, col0, nr, nc);
            fence_proxy_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (tid == 0) issue_eta(Lo, sm, tb, &bars[2]);
            is2++;
        }
        for (int it = 0; t < ntiles; it++, t += G) {
            const int b = it & 1;
            const int tn = t + G;
            int64_t row0, col0, rown = 0, coln = 0;
            int nr, nc, nrn = 0, ncn = 0;
            tile_origin(t, row0, col0, nr, nc);
            if (tn < ntiles) tile_origin(tn, rown, coln, nrn, ncn);
            if (tn < ntiles) {
                if (tid == 0) issue_counts(Lo, &ymap, sm + (b ^ 1) * Lo.y_bytes, rown, coln, &bars[b ^ 1]);
                if (b) is0++; else is1++;
            }
            // eta of tile t is complete: its operands may be overwritten
            ok = cta_wait(&bars[2], (uint32_t)(wt2 & 1), a.err);
            wt2++;
            if (!ok) break;
            tc_fence_after();
            if (tn < ntiles) {
                build_operands<false>(a, Lo, sm, rown, coln, nrn, ncn);
                fence_proxy_async_smem();
                tc_fence_before();
                __syncthreads();
                tc_fence_after();
                if (tid == 0) issue_eta(Lo, sm, tb + (uint32_t)(TT * (b ^ 1)), &bars[2]);
                is2++;
            }
            ok = cta_wait(&bars[b], (uint32_t)((b ? wt1 : wt0) & 1), a.err);
            if (b) wt1++; else wt0++;
            if (!ok) break;
            tc_fence_after();
            total += (double)tile_deviance<Y16, GEN>(a, sm + b * Lo.y_bytes, tb + (uint32_t)(TT * b), q, ch, row0,
                                                     col0, nr, nc, nb, alpha, la, tab);
            // tile t's counts and accumulator are dead: the loads and MMAs of tile t + 2 may reuse them
            fence_proxy_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
        }
    }
    if (!ok) {
        // a wait gave up: let this CTA's own copies and MMAs still in flight finish (bounded) before TMEM goes
        if (tid == 0) {
            if (is0 > wt0) mbar_wait(&bars[0], (uint32_t)(wt0 & 1), WAIT_POLLS);
            if (is1 > wt1) mbar_wait(&bars[1], (uint32_t)(wt1 & 1), WAIT_POLLS);
            if (is2 > wt2) mbar_wait(&bars[2], (uint32_t)(wt2 & 1), WAIT_POLLS);
            atomicOr(a.err, GMF_DEVERR_TIMEOUT);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tb, TCOLS);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
    if (lane == 0) red[warp] = total;
    __syncthreads();
    if (tid == 0) {
        double v = 0.0;
        for (int u = 0; u < DTH / 32; u++) v += red[u];
        part[blockIdx.x] = v;
    }
}

template <bool GEN, int ST>
const void* dev_tc_fn_gen(int y16) {
    return y16 ? (const void*)deviance_tc<true, GEN, ST> : (const void*)deviance_tc<false, GEN, ST>;
}
const void* dev_tc_fn(int y16, int gen, int st) {
    if (st == 1) return gen ? dev_tc_fn_gen<true, 1>(y16) : dev_tc_fn_gen<false, 1>(y16);
    return gen ? dev_tc_fn_gen<true, 2>(y16) : dev_tc_fn_gen<false, 2>(y16);
}

}  // namespace

namespace {

// Dynamic shared memory of the ST-stage variant: ST count buffers, one set of
// eta operands, alignment slack.
uint32_t dev_smem_of(const TcState* tc, int st) {
    return (uint32_t)st * tc->lay.y_bytes + 2u * (uint32_t)tc->lay.KA * ATOM + 1024u;
}
int dev_stages(const TcState* tc) { return tc->dev_smem == dev_smem_of(tc, 1) ? 1 : 2; }

// CTAs per SM of the ST-stage variant from registers, shared memory and TMEM
// (ST x 128 columns each; the occupancy query reports one CTA per SM for these
// kernels where the SM holds more); 0 where it cannot run.
int dev_ctas_per_sm(const gmf_model* h, const TcState* tc, int st, int gen) {
    const void* fn = dev_tc_fn(h->y16, gen, st);
    const uint32_t smem = dev_smem_of(tc, st);
    int dev = 0, smem_sm = 0, regs_sm = 0, resv = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        gmf_smem_limit(fn, smem) != cudaSuccess ||
        cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared) !=
            cudaSuccess ||
        cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const int regs_cta = ((fa.numRegs * 32 + 255) / 256) * 256 * (DTH / 32);
    const size_t smem_cta = (size_t)smem + fa.sharedSizeBytes + (size_t)resv;
    return std::min({regs_sm / std::max(regs_cta, 1), (int)((size_t)smem_sm / smem_cta), 4 / st});
}

}  // namespace

// The tensor-core deviance of a handle: the single-stage variant where three
// of its CTAs fit an SM (16-bit counts, K <= 32), else the double-buffered one
// at two per SM; the grid is what the device holds at once. With flags asking
// for the CUDA-core kernel, or where neither fits, dev_grid stays 0.
void gmf_tc_deviance_setup(gmf_model* h, TcState* tc) {
    tc->dev_grid = 0;
    if (h->cfg.flags & GMF_FLAG_SIMT_DEVIANCE) return;
    tc->dev_gen = (h->Wp || h->cfg.missing || h->cfg.alpha_mode == 2 || h->cfg.family > GMF_NEGBIN) ? 1 : 0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    int st = 1, per_sm = dev_ctas_per_sm(h, tc, 1, tc->dev_gen);
    if (per_sm < 3) {
        st = 2;
        per_sm = std::min(dev_ctas_per_sm(h, tc, 2, tc->dev_gen), 2);
    }
    if (per_sm < 1) return;
    tc->dev_smem = dev_smem_of(tc, st);
    const int64_t ntiles = ((h->n + TT - 1) / TT) * ((h->m + TT - 1) / TT);
    tc->dev_grid = (int)std::min<int64_t>((int64_t)per_sm * sms, std::max<int64_t>(ntiles, 1));
}

int gmf_tc_deviance_ok(const gmf_model* h) { return h->tc && ((const TcState*)h->tc)->dev_grid > 0; }

// Per-CTA FP64 sums of deviance_tc into h->devpart (at least as many slots as
// 64 x 64 tiles, so at least dev_grid), then their FP64 total at d_out.
cudaError_t gmf_tc_launch_deviance(gmf_model* h, double* d_out, cudaStream_t st) {
    const TcState* tc = (const TcState*)h->tc;
    const StepArgs a = gmf_make_args(h);
    const int stages = dev_stages(tc);
    TcLayout L = tc->lay;
    L.off_u = (uint32_t)stages * L.y_bytes;  // the count buffers, then the eta operands
    const int ntj = (int)((h->m + TT - 1) / TT);
    const int ntiles = (int)(((h->n + TT - 1) / TT) * ntj);
    const void* fn = dev_tc_fn(h->y16, tc->dev_gen, stages);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)tc->dev_grid);
    cfg.blockDim = dim3(DTH);
    cfg.dynamicSmemBytes = tc->dev_smem;
    cfg.stream = st;
    double* part = h->devpart;
    void* args[] = {(void*)&a, (void*)&L, (void*)&tc->ymap[h->ycur], (void*)&ntj, (void*)&ntiles, (void*)&part};
    const cudaError_t e = cudaLaunchKernelExC(&cfg, fn, args);
    if (e != cudaSuccess) return e;
    return gmf_launch_sum_parts(h->devpart, tc->dev_grid, d_out, st);
}
