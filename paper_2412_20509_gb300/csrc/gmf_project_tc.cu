// Per-cell projection of new cells (the row problem of Sec. 3 with the column
// side fixed, solved by the Fisher row step of Sec. 3.1) with the Fisher
// matrices on the tcgen05 tensor cores. Same passes, start and step control as
// project_kernel (gmf_project.cu); f = q + d <= 22 and uint16 counts.
//
// For 128 cells per CTA the genes stream in chunks of 64. Per chunk:
//   warp 16 (one thread): TMA of the counts (128 x 64, 128-byte swizzle), of R's rows (64 x KP,
//     FP32) and, in Fisher passes, of the chunk of the Khatri-Rao product
//     KR[pair][gene] = r_ga r_gb of [Z, V] (BF16, 128-byte swizzle, 256 pairs);
//   warps 0-15 (thread -> cell t % 128, genes 16 (t / 128) ..): eta, mu, the
//     unit deviances and the score sums sum_j Ddot_ij r_j in FP32, and the
//     Fisher weights Dddot_ij as BF16 into the swizzled A operand;
//   warp 17 (one thread): F_i += sum_j Dddot_ij KR_j (M = 128 cells, N = 256
//     pairs, K = 64 genes) into TMEM.
// BF16 rounding errors of the products are independent across the genes, so
// they average out in the sums (the Fisher matrix only sets the step; the
// score, which fixes the optimum, is exact FP32). After a pass the Fisher
// matrices go from TMEM to shared memory ([pair][cell], over the idle stage
// buffers) and one thread per cell applies the step control and solves by
// packed Cholesky. Every mbarrier wait is bounded; one that gives up sets the
// status word and the CTA stops at the next pass boundary.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>

#include <algorithm>
#include <string>

#include "gmf_internal.cuh"
#include "gmf_sm100.cuh"

using namespace sm100;

namespace {

constexpr int BM = 128;             // cells per CTA (MMA M)
constexpr int GC = 64;              // genes per chunk (MMA K)
constexpr int NCT = 512;            // compute threads (16 warps)
constexpr int NTH = NCT + 64;       // + the TMA warp and the MMA warp
constexpr int NPP = 256;            // pair columns (MMA N)
constexpr int FTC = 22;             // largest f: f (f + 1) / 2 <= 253
constexpr int PTC = 8;              // largest p
constexpr int FS = 23;              // stride of the per-cell vectors in shared memory (odd)
constexpr uint32_t A_BYTES = BM * 128, KR_BYTES = NPP * 128;
constexpr uint32_t WAIT_POLLS = 1u << 24;
constexpr float SLACK = 1e-5f;      // relative slack of the acceptance test

struct PArgs {
    int64_t n, m;
    int p, q, d, f, np, KP, nk, n_steps;
    uint32_t r_bytes, r_pad, y_bytes, stage, off_pers;   // r_pad: R rows rounded up to 1024 bytes
    const float* X;
    const float* off;
    const float* Ustart;
    const float* alpha;
    int nb;
    float clamp, lam_g, lam_u;
    float* Uout;
    float* Gout;
    float* dev;
    unsigned* err;
};

__device__ __forceinline__ int pidx(int i, int j) { return i * (i + 1) / 2 + j; }  // i >= j

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void bar_compute() { asm volatile("bar.sync 1, %0;" ::"n"(NCT) : "memory"); }
// Barrier of the compute threads that also ORs a flag over them (the same answer in every thread).
__device__ __forceinline__ int bar_compute_or(int flag) {
    int r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.s32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"(flag), "n"(NCT)
        : "memory");
    return r;
}

// Unit deviance / 2, branch-free (every lane of a warp takes the same path):
//   Poisson  y (log y - eta) - (y - mu),   NB  y (log y - eta) - (y + a)(log(y + a) - log(mu + a)),
// the y log y term zero at y = 0. log y and log(y + a) come from per-CTA tables for y < 256. Near
// mu = y the two logarithms of the NB term cancel: the rounding is ~1e-7 of (y + a) log(y + a) per
// entry, ~1e-6 of a cell's deviance over thousands of genes.
__device__ __forceinline__ float half_unit_dev(bool nb, float y, float ec, float mu, float alpha, const float* tlog,
                                               const float* tloga) {
    const int yi = (int)y;
    float ly, lya;
    if (yi < 256) {
        ly = tlog[yi];
        lya = tloga[yi];
    } else {
        ly = logf(y);
        lya = logf(y + alpha);
    }
    const float t1 = yi > 0 ? y * (ly - ec) : 0.f;
    return nb ? t1 - (y + alpha) * (lya - __logf(mu + alpha)) : t1 - (y - mu);
}

// 18 warps: five share one of the four SM sub-partitions, which caps registers at 96 per thread.
__global__ void __launch_bounds__(NTH, 1)
    project_tc(PArgs a, const __grid_constant__ CUtensorMap ymap, const __grid_constant__ CUtensorMap rmap,
               const __grid_constant__ CUtensorMap krmap) {
    extern __shared__ __align__(1024) uint8_t smraw[];
    __shared__ uint64_t full_tma[2], empty_cmp[2], full_a[2], empty_mma[2], mma_done, pass_gate;
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    __shared__ float tlog[256], tloga[256];  // log(v), log(v + alpha), v < 256

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t* sm = smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u);
    const int64_t cell0 = (int64_t)blockIdx.x * BM;
    const int f = a.f, np = a.np, KP = a.KP;
    // per-cell vectors that live across passes
    float* TH = (float*)(sm + a.off_pers);     // BM x FS: current point
    float* BEST = TH + BM * FS;                // best accepted point
    float* DEL = BEST + BM * FS;               // last step
    float* GRD = DEL + BM * FS;                // score sum over the 4 gene quarters
    float* FB = GRD + BM * FS;                 // BM: best objective
    float* DB = FB + BM;                       // BM: deviance at the best point
    float* DVQ = DB + BM;                      // 4 x BM: deviance partials
    float* S1Q = DVQ + 4 * BM;                 // 4 x BM: sum y (first pass)
    float* S2Q = S1Q + 4 * BM;                 // 4 x BM: sum exp(eta without gamma)
    float* F = (float*)sm;                     // np x BM Fisher matrices, over the stage buffers between passes

    if (tid == 0) {
        for (int s = 0; s < 2; s++) {
            mbar_init(&full_tma[s], 1);
            mbar_init(&empty_cmp[s], NCT / 32);
            mbar_init(&full_a[s], NCT / 32);
            mbar_init(&empty_mma[s], 1);
        }
        mbar_init(&mma_done, 1);
        mbar_init(&pass_gate, 1);
        fence_mbar_init();
        s_abort = 0;
    }
    for (int e = tid; e < BM * FS; e += NTH) {
        const int c = e / FS, k = e - c * FS;
        float v = 0.f;
        if (k >= a.q && k < f && a.Ustart && cell0 + c < a.n) v = a.Ustart[(cell0 + c) * a.d + (k - a.q)];
        TH[e] = v;
        BEST[e] = v;
        DEL[e] = 0.f;
    }
    if (tid < BM) FB[tid] = DB[tid] = 0.f;
    if (tid < 256) {
        const float al = *a.alpha;
        tlog[tid] = tid > 0 ? logf((float)tid) : 0.f;
        tloga[tid] = a.nb ? logf((float)tid + al) : 0.f;
    }
    if (warp == 17) tmem_alloc(&tmem_base, NPP);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tb = tmem_base;
    const int npass = a.n_steps + 2;  // 0: closed-form gamma; 1..n_steps: Fisher; n_steps + 1: evaluation

    if (warp == 16) {
        // ---------------------------------------------------------------- TMA producer
        if (lane == 0) {
            for (int P = 0; P < npass; P++) {
                if (P > 0 && !mbar_wait(&pass_gate, (uint32_t)(P - 1) & 1u, WAIT_POLLS)) {
                    atomicOr(a.err, GMF_DEVERR_TIMEOUT);
                    s_abort = 1;
                }
                if (s_abort) break;
                const bool fisher = P >= 1 && P <= a.n_steps;
                for (int kc = 0; kc < a.nk; kc++) {
                    const int s = kc & 1;
                    const int G = P * a.nk + kc;
                    bool ok = true;
                    if (G >= 2) {
                        ok = mbar_wait(&empty_cmp[s], (uint32_t)((G >> 1) - 1) & 1u, WAIT_POLLS);
                        const int prev = G - 2, Pp = prev / a.nk, kp = prev - Pp * a.nk;
                        if (ok && Pp >= 1 && Pp <= a.n_steps)
                            ok = mbar_wait(&empty_mma[s], (uint32_t)(((Pp - 1) * a.nk + kp) >> 1) & 1u, WAIT_POLLS);
                    }
                    if (!ok) {
                        atomicOr(a.err, GMF_DEVERR_TIMEOUT);
                        s_abort = 1;
                        break;
                    }
                    uint8_t* st = sm + (size_t)s * a.stage;
                    mbar_arrive_expect_tx(&full_tma[s], a.r_bytes + a.y_bytes + (fisher ? KR_BYTES : 0u));
                    tma_load_2d(st + A_BYTES + KR_BYTES, &rmap, 0, kc * GC, &full_tma[s]);
                    tma_load_2d(st + A_BYTES + KR_BYTES + a.r_pad, &ymap, kc * GC, (int)cell0, &full_tma[s]);
                    if (fisher) tma_load_2d(st + A_BYTES, &krmap, kc * GC, 0, &full_tma[s]);
                }
            }
        }
    } else if (warp == 17) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t id = idesc_bf16(BM, NPP, 0, 0);
            for (int P = 1; P <= a.n_steps && !s_abort; P++) {
                for (int kc = 0; kc < a.nk; kc++) {
                    const int s = kc & 1;
                    if (!mbar_wait(&full_a[s], (uint32_t)(((P - 1) * a.nk + kc) >> 1) & 1u, WAIT_POLLS)) {
                        atomicOr(a.err, GMF_DEVERR_TIMEOUT);
                        s_abort = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t abase = smem_u32(sm + (size_t)s * a.stage), bbase = abase + A_BYTES;
#pragma unroll
                    for (int ks = 0; ks < GC / 16; ks++)
                        umma_bf16(tb, sdesc(abase + 32u * ks, 16, 1024, SWIZZLE_128B),
                                  sdesc(bbase + 32u * ks, 16, 1024, SWIZZLE_128B), id, (kc > 0 || ks > 0) ? 1u : 0u);
                    umma_commit(&empty_mma[s]);
                }
                umma_commit(&mma_done);
            }
        }
    } else {
        // ---------------------------------------------------------------- compute threads
        const int cell = tid & (BM - 1), qg = tid >> 7;
        const int64_t gi = cell0 + cell;
        const bool cv = gi < a.n;
        const float alpha = *a.alpha;
        float xr[PTC];
#pragma unroll
        for (int k = 0; k < PTC; k++) xr[k] = (cv && k < a.p) ? a.X[gi * a.p + k] : 0.f;
        const float o = (cv && a.off) ? a.off[gi] : 0.f;
        float th[FTC];
        for (int P = 0; P < npass; P++) {
            const bool init = P == 0, fisher = P >= 1 && P <= a.n_steps;
#pragma unroll
            for (int k = 0; k < FTC; k++) th[k] = k < f ? TH[cell * FS + k] : 0.f;
            float g[FTC];
#pragma unroll
            for (int k = 0; k < FTC; k++) g[k] = 0.f;
            float dv = 0.f, s1 = 0.f, s2 = 0.f;
            for (int kc = 0; kc < a.nk; kc++) {
                const int s = kc & 1;
                const int G = P * a.nk + kc;
                const uint8_t* st = sm + (size_t)s * a.stage;
                if (!mbar_wait(&full_tma[s], (uint32_t)(G >> 1) & 1u, WAIT_POLLS)) {
                    atomicOr(a.err, GMF_DEVERR_TIMEOUT);
                    s_abort = 1;
                }
                const float* sR = (const float*)(st + A_BYTES + KR_BYTES);
                // the count tile has the 128-byte swizzle: a warp (32 cells, one gene) reads 8 banks, not 1
                const uint8_t* sY = st + A_BYTES + KR_BYTES + a.r_pad;
                uint32_t pk[8];
#pragma unroll
                for (int jj = 0; jj < 16; jj += 2) {  // fully unrolled: pk stays in registers
                    float wv[2];
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        const int j = qg * 16 + jj + h;
                        const float* rj = sR + j * KP;
                        const bool valid = cv && (int64_t)kc * GC + j < a.m;
                        const float y =
                            (float)*(const unsigned short*)(sY + sw128_off((uint32_t)cell, (uint32_t)(2 * j)));
                        // two interleaved partial sums: half the dependent chain
                        float eta = o, eta2 = 0.f;
#pragma unroll
                        for (int k = 0; k < PTC; k++)
                            if (k < a.p) eta = fmaf(xr[k], rj[1 + k], eta);
                        const float* rz = rj + 1 + a.p;
#pragma unroll
                        for (int k = 0; k < FTC; k += 2) {
                            if (k < f) eta2 = fmaf(th[k], rz[k], eta2);
                            if (k + 1 < f) eta = fmaf(th[k + 1], rz[k + 1], eta);
                        }
                        eta += eta2;
                        float ddd = 0.f;
                        if (init) {
                            const float rest = eta - th[0] * rz[0];
                            if (valid) {
                                s1 += y;
                                s2 += expf(fminf(fmaxf(rest, -a.clamp), a.clamp));
                            }
                        } else {
                            const float ec = fminf(fmaxf(eta, -a.clamp), a.clamp);
                            const float mu = __expf(ec);
                            if (valid) dv += half_unit_dev(a.nb, y, ec, mu, alpha, tlog, tloga);
                            if (fisher && valid) {
                                const float fct = a.nb ? __fdividef(alpha, alpha + mu) : 1.f;
                                const float dd = (y - mu) * fct;
                                ddd = mu * fct;
#pragma unroll
                                for (int k = 0; k < FTC; k++)
                                    if (k < f) g[k] = fmaf(dd, rz[k], g[k]);
                            }
                        }
                        wv[h] = ddd;
                    }
                    pk[jj >> 1] = pack_bf16x2(wv[0], wv[1]);
                }
                if (fisher) {
#pragma unroll
                    for (int q2 = 0; q2 < 2; q2++) {
                        const uint32_t off = sw128_off((uint32_t)cell, (uint32_t)(qg * 32 + q2 * 16));
                        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(smem_u32(st + off)),
                                     "r"(pk[4 * q2]), "r"(pk[4 * q2 + 1]), "r"(pk[4 * q2 + 2]), "r"(pk[4 * q2 + 3])
                                     : "memory");
                    }
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&full_a[s]);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty_cmp[s]);
            }
            // ---- pass end: partial sums over the four gene quarters, in quarter order
            DVQ[qg * BM + cell] = dv;
            S1Q[qg * BM + cell] = s1;
            S2Q[qg * BM + cell] = s2;
            for (int r = 0; r < 4; r++) {
                if (qg == r && fisher) {
#pragma unroll
                    for (int k = 0; k < FTC; k++)  // constant indices keep g in registers
                        if (k < f) GRD[cell * FS + k] = (r == 0 ? 0.f : GRD[cell * FS + k]) + g[k];
                }
                bar_compute();
            }
            if (fisher) {
                const bool ok = mbar_wait(&mma_done, (uint32_t)(P - 1) & 1u, WAIT_POLLS);
                if (!ok) {
                    atomicOr(a.err, GMF_DEVERR_TIMEOUT);
                    s_abort = 1;
                }
                tc_fence_after();
                // warp w: TMEM lanes 32 (w % 4) .., pair columns 64 (w / 4) .. + 63
                const int lg = warp & 3, cs = warp >> 2;
                const int c = 32 * lg + lane;
                if (ok)
                    for (int c0 = cs * 64; c0 < cs * 64 + 64; c0 += 32) {
                        uint32_t v[32];
                        tmem_ld32(tb + ((uint32_t)(32 * lg) << 16) + (uint32_t)c0, v);
                        tmem_wait_ld();
#pragma unroll
                        for (int u = 0; u < 32; u++)
                            if (c0 + u < np) F[(c0 + u) * BM + c] = __uint_as_float(v[u]);
                    }
                tc_fence_before();
            }
            bar_compute();
            if (qg == 0 && cv) {
                float* thc = TH + cell * FS;
                float* be = BEST + cell * FS;
                float* de = DEL + cell * FS;
                if (init) {
                    const float S1 = ((S1Q[cell] + S1Q[BM + cell]) + S1Q[2 * BM + cell]) + S1Q[3 * BM + cell];
                    const float S2 = ((S2Q[cell] + S2Q[BM + cell]) + S2Q[2 * BM + cell]) + S2Q[3 * BM + cell];
                    if (a.q > 0) thc[0] = logf(fmaxf(S1, 0.5f) / S2);
                } else {
                    const float D = 2.f * (((DVQ[cell] + DVQ[BM + cell]) + DVQ[2 * BM + cell]) + DVQ[3 * BM + cell]);
                    float pen = 0.f;
                    for (int k = 0; k < f; k++) pen += (k < a.q ? a.lam_g : a.lam_u) * thc[k] * thc[k];
                    const float obj = 0.5f * D + 0.5f * pen;
                    const float fb = FB[cell];
                    if (P == 1 || obj <= fb + SLACK * (1.f + fabsf(fb))) {
                        for (int k = 0; k < f; k++) be[k] = thc[k];
                        FB[cell] = obj;
                        DB[cell] = D;
                        if (fisher) {
                            // F + Lambda = L L' in place (packed, column `cell` of F); the right-hand side
                            // b = score - Lambda theta, then the solution, in place in this cell's GRD row
                            float* b = GRD + cell * FS;
                            for (int k = 0; k < f; k++) {
                                const float lam = k < a.q ? a.lam_g : a.lam_u;
                                F[pidx(k, k) * BM + cell] += lam;
                                b[k] -= lam * thc[k];
                            }
                            bool okc = true;
                            for (int j = 0; j < f && okc; j++) {
                                float sj = F[pidx(j, j) * BM + cell];
                                for (int k = 0; k < j; k++) sj -= F[pidx(j, k) * BM + cell] * F[pidx(j, k) * BM + cell];
                                if (!(sj > 0.f)) {
                                    okc = false;
                                    break;
                                }
                                const float ljj = sqrtf(sj);
                                F[pidx(j, j) * BM + cell] = ljj;
                                for (int i = j + 1; i < f; i++) {
                                    float t = F[pidx(i, j) * BM + cell];
                                    for (int k = 0; k < j; k++) t -= F[pidx(i, k) * BM + cell] * F[pidx(j, k) * BM + cell];
                                    F[pidx(i, j) * BM + cell] = t / ljj;
                                }
                            }
                            if (okc) {
                                for (int i = 0; i < f; i++) {  // L z = b
                                    float t = b[i];
                                    for (int k = 0; k < i; k++) t -= F[pidx(i, k) * BM + cell] * b[k];
                                    b[i] = t / F[pidx(i, i) * BM + cell];
                                }
                                for (int i = f - 1; i >= 0; i--) {  // L' x = z
                                    float t = b[i];
                                    for (int k = i + 1; k < f; k++) t -= F[pidx(k, i) * BM + cell] * b[k];
                                    b[i] = t / F[pidx(i, i) * BM + cell];
                                }
                            }
                            for (int k = 0; k < f; k++) {
                                de[k] = okc ? b[k] : 0.f;
                                thc[k] = be[k] + de[k];
                            }
                        }
                    } else {
                        for (int k = 0; k < f; k++) {
                            de[k] *= 0.5f;
                            thc[k] = be[k] + de[k];
                        }
                    }
                }
            }
            // the stage buffers (and F over them) go back to the TMA: order this pass's generic accesses first
            fence_proxy_async_smem();
            const int stop = bar_compute_or(s_abort);
            if (tid == 0) mbar_arrive(&pass_gate);
            if (stop) break;
        }
        // ---- outputs: the best point and its deviance
        for (int e = tid; e < BM * f; e += NCT) {
            const int c = e / f, k = e - c * f;
            if (cell0 + c >= a.n) continue;
            const float v = BEST[c * FS + k];
            if (k < a.q)
                a.Gout[(cell0 + c) * a.q + k] = v;
            else
                a.Uout[(cell0 + c) * a.d + (k - a.q)] = v;
        }
        if (tid < BM && cv && a.dev) a.dev[gi] = DB[tid];
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 17) tmem_dealloc(tb, NPP);
}

// KR[pair][gene] = r_ga r_gb (a >= b, packed pair index) of [Z, V] in BF16, zero padding.
__global__ void build_kr(const float* R, int64_t m, int KP, int p, int f, int np, int64_t mP, __nv_bfloat16* KR) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)NPP * mP;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int pr = (int)(e / mP);
        const int64_t j = e - (int64_t)pr * mP;
        float v = 0.f;
        if (pr < np && j < m) {
            int i = (int)((sqrtf(8.f * pr + 1.f) - 1.f) * 0.5f);
            while (i * (i + 1) / 2 > pr) i--;
            while ((i + 1) * (i + 2) / 2 <= pr) i++;
            const int k = pr - i * (i + 1) / 2;
            v = R[j * KP + 1 + p + i] * R[j * KP + 1 + p + k];
        }
        KR[e] = __float2bfloat16_rn(v);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &qr) ==
                cudaSuccess &&
            ptr)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
    }
    return fn;
}

struct ProjTcPlan {
    int nk;
    uint32_t r_bytes, r_pad, y_bytes, stage, off_pers;
    size_t smem;
};

bool plan(int64_t m, int p, int q, int d, int KP, ProjTcPlan* pl) {
    const int f = q + d;
    if (f > FTC || f < 1 || q < 1 || p > PTC || KP > 64) return false;
    pl->nk = (int)(((m + GC - 1) / GC + 1) / 2 * 2);
    pl->r_bytes = (uint32_t)(GC * KP * 4);
    pl->r_pad = (pl->r_bytes + 1023u) & ~1023u;
    pl->y_bytes = (uint32_t)(BM * GC * 2);
    pl->stage = (A_BYTES + KR_BYTES + pl->r_pad + pl->y_bytes + 1023u) & ~1023u;
    const uint32_t fisher_bytes = (uint32_t)(f * (f + 1) / 2) * BM * 4u;
    const uint32_t stages = std::max(2u * pl->stage, fisher_bytes);
    pl->off_pers = (stages + 15u) & ~15u;
    const uint32_t pers = 4u * (4u * BM * FS + 2u * BM + 12u * BM);
    pl->smem = (size_t)pl->off_pers + pers + 1024;
    int optin = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return pl->smem + 4096 <= (size_t)optin;  // static shared memory (barriers, log tables)
}

}  // namespace

// The tensor-core projection. Returns GMF_ERR_STATE, with nothing launched, only when
// the shapes are outside its range (the caller then uses the FP32 kernel).
int gmf_project_tc_run(const float* Rorig, int64_t m, int p, int q, int d, int KP, const void* Ynew, int y16,
                       int64_t n_new, const float* Xnew, const float* off, const float* Ustart, const float* alpha,
                       int nb, float clamp, float lam_g, float lam_u, int n_steps, float* Uout, float* Gout, float* dev,
                       unsigned* err_word, __nv_bfloat16** kr_buf, size_t* kr_elems, cudaStream_t st,
                       std::string* err) {
    ProjTcPlan pl;
    if (!y16 || ((uintptr_t)Ynew) % 16 != 0 || (m * 2) % 16 != 0 || !plan(m, p, q, d, KP, &pl)) return GMF_ERR_STATE;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) {
        *err = "cuTensorMapEncodeTiled is not available";
        return GMF_ERR_CUDA;
    }
    const int f = q + d, np = f * (f + 1) / 2;
    const int64_t mP = (int64_t)pl.nk * GC;
    const size_t need = (size_t)NPP * mP;
    if (*kr_elems < need) {
        if (*kr_buf) cudaFree(*kr_buf);
        *kr_buf = nullptr;
        *kr_elems = 0;
        if (cudaMalloc(kr_buf, sizeof(__nv_bfloat16) * need) != cudaSuccess) {
            *err = "device allocation failed";
            return GMF_ERR_OOM;
        }
        *kr_elems = need;
    }
    build_kr<<<(int)std::min<int64_t>(((int64_t)need + 255) / 256, 8192), 256, 0, st>>>(Rorig, m, KP, p, f, np, mP,
                                                                                        *kr_buf);
    CUtensorMap ymap, rmap, krmap;
    cuuint32_t one[2] = {1, 1};
    cuuint64_t yd[2] = {(cuuint64_t)m, (cuuint64_t)n_new}, ys[1] = {(cuuint64_t)m * 2};
    cuuint32_t yb[2] = {(cuuint32_t)GC, (cuuint32_t)BM};
    cuuint64_t rd[2] = {(cuuint64_t)KP, (cuuint64_t)m}, rs[1] = {(cuuint64_t)KP * 4};
    cuuint32_t rb[2] = {(cuuint32_t)KP, (cuuint32_t)GC};
    cuuint64_t kd[2] = {(cuuint64_t)mP, (cuuint64_t)NPP}, ks[1] = {(cuuint64_t)mP * 2};
    cuuint32_t kb[2] = {(cuuint32_t)GC, (cuuint32_t)NPP};
    CUresult cr = enc(&ymap, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, (void*)Ynew, yd, ys, yb, one,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr == CUDA_SUCCESS)
        cr = enc(&rmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)Rorig, rd, rs, rb, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                 CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr == CUDA_SUCCESS)
        cr = enc(&krmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)*kr_buf, kd, ks, kb, one,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) {
        *err = "cuTensorMapEncodeTiled failed for the projection's operands";
        return GMF_ERR_CUDA;
    }
    PArgs a{};
    a.n = n_new;
    a.m = m;
    a.p = p;
    a.q = q;
    a.d = d;
    a.f = f;
    a.np = np;
    a.KP = KP;
    a.nk = pl.nk;
    a.n_steps = n_steps;
    a.r_bytes = pl.r_bytes;
    a.r_pad = pl.r_pad;
    a.y_bytes = pl.y_bytes;
    a.stage = pl.stage;
    a.off_pers = pl.off_pers;
    a.X = Xnew;
    a.off = off;
    a.Ustart = Ustart;
    a.alpha = alpha;
    a.nb = nb;
    a.clamp = clamp;
    a.lam_g = lam_g;
    a.lam_u = lam_u;
    a.Uout = Uout;
    a.Gout = Gout;
    a.dev = dev;
    a.err = err_word;
    cudaError_t e = gmf_smem_limit((const void*)project_tc, pl.smem);
    if (e == cudaSuccess) {
        project_tc<<<(unsigned)((n_new + BM - 1) / BM), NTH, pl.smem, st>>>(a, ymap, rmap, krmap);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        *err = cudaGetErrorString(e);
        return GMF_ERR_CUDA;
    }
    return GMF_OK;
}
