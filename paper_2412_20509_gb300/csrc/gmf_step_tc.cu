// Tensor-core (tcgen05, sm_103a) path of the block step: Algorithm 1's per-block
// work (eq. 15 with App. B) with eta and the four gradient / curvature
// contractions on the 5th-generation tensor cores.
//
// One CTA per 128 x 128 tile, 16 warps:
//   1. thread 0 starts the TMA load of the tile's counts (128-byte swizzled
//      boxes) while all threads build the MMA operands in shared memory:
//        eta:  A = [L_hi | L_lo], B = [R_hi | R_lo] (BF16 split of the FP32
//              factors, K-concatenated); one accumulation runs the K chunks of
//              L_hi R_hi', then L_lo R_hi', then L_hi R_lo' (split-BF16, 3 products);
//        row side:    B = [Z, V]' and its square, K = tile columns;
//        column side: B = [X, U]' and its square, K = tile rows;
//   2. thread 0 issues the eta MMAs (FP32 accumulate in TMEM) and commits;
//   3. the 16 warps read eta from TMEM (warp w: lanes 32(w%4).., columns
//      32(w/4)..), compute mu = exp(eta), Ddot, Dddot (Sec. 3) in FP32 and
//      store them as BF16 into swizzled tiles: with 16-bit counts Ddot goes in
//      place over the count tile (same layout, each thread overwrites the
//      16 bytes it has just read) and Dddot over the dead eta operands, which
//      keeps a tile within half of an SM's shared memory (two CTAs per SM);
//      with 32-bit counts both go over the eta operands;
//   4. thread 0 issues the contractions: Ddot R_f and Dddot R_f^2 (A = the
//      tile, K-major) and Ddot' L_f and Dddot' L_f^2 (A = the same tile read
//      MN-major); warps 0-3 read the row sums, warps 4-7 the column sums, from
//      TMEM into the per-tile partial slots;
//   5. the shared strip update (gmf_update.cuh).
// Every mbarrier wait is bounded; on time-out the CTA flags GMF_DEVERR_TIMEOUT,
// waits once more (bounded) for its own in-flight copies and MMAs, frees TMEM
// and skips the update.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <string.h>

#include <algorithm>
#include <deque>
#include <vector>

#include <string>

#include "gmf_internal.cuh"
#include "gmf_sm100.cuh"
#include "gmf_update.cuh"
#include "gmf_tc_tile.cuh"

namespace {

using namespace gmfdev;
using namespace sm100;
using namespace gmftc;

// ---- cluster mode. The TI x TJ tiles of a block form one thread-block
// cluster. CTA (ti, tj) owns rows [tj*SRr, (tj+1)*SRr) of row strip ti and
// columns [ti*SCc, (ti+1)*SCc) of column strip tj. Each tile stores its row
// (column) partials straight from TMEM into the owners' shared memory, one
// slot per source tile (distributed shared memory stores, coalesced along the
// rows); after one cluster barrier each owner sums its slots in tile order
// (the order of the update launch, so both modes give the same bits) and
// applies the smoothed step. Nothing touches a peer's shared memory after that
// barrier, so no second barrier is needed before a CTA exits.

struct ClSlice {
    int nrs, ncs;              // rows / columns of this CTA's slices (0: none)
    int64_t first_r, first_c;  // their first global row of L / row of R
    int or0, oc0;              // their first index within the strip's tiles
};

__device__ __forceinline__ ClSlice cl_slice(const StepArgs& a, const TcLayout& Lo, const BlockGeo& g, int ti, int tj,
                                            int nTI, int nTJ) {
    ClSlice c;
    c.or0 = tj * Lo.SRr;
    c.oc0 = ti * Lo.SCc;
    const int nstr = ti < nTI ? (int)min((int64_t)TT, g.nI - (int64_t)ti * TT) : 0;
    const int nstc = tj < nTJ ? (int)min((int64_t)TT, g.mJ - (int64_t)tj * TT) : 0;
    c.nrs = max(0, min(Lo.SRr, nstr - c.or0));
    c.ncs = max(0, min(Lo.SCc, nstc - c.oc0));
    c.first_r = g.r0 + (int64_t)ti * TT + c.or0;
    c.first_c = g.c0 + (int64_t)tj * TT + c.oc0;
    return c;
}

// Shared-memory pieces of one side's slice (rows of P, Gb, Hb, counts).
struct ClStage {
    float *P, *G, *H;
    int* C;
};

__device__ __forceinline__ ClStage cl_stage_ptrs(float* base, int rows, int KS, int NS) {
    ClStage t;
    t.P = base;
    t.G = t.P + rows * KS;
    t.H = t.G + rows * NS;
    t.C = (int*)(t.H + rows * NS);
    return t;
}

// Start the copies of this CTA's slices with threads [t0, t0 + nt) (after the
// dependency wait: the previous sweep wrote these rows). Each thread waits for
// its own copies (cp.async.wait_all) before the cluster barrier. In the
// persistent kernel the copies are issued after the acquire that orders them
// behind their writer (the moving strip's count; the CTA's own fixed-strip
// slice has no other writer), and no stale line can serve them: a cluster
// visits each moving strip once per launch and reads operands through L2.
// stage_r / stage_c: copy that side (the persistent kernel keeps its fixed
// side's slice in shared memory from one block to the next).
__device__ __forceinline__ void cl_stage_issue(const StepArgs& a, const TcLayout& Lo, uint8_t* sm, const ClSlice& c,
                                               int t0, int nt, bool stage_r = true, bool stage_c = true) {
    const int KS = a.KP + 1;
    const int tid = (int)threadIdx.x - t0;
    if (tid < 0 || tid >= nt) return;
    const ClStage r = cl_stage_ptrs((float*)(sm + Lo.off_st), Lo.SRr, KS, a.fr | 1);
    const ClStage q = cl_stage_ptrs(r.P + (size_t)Lo.SRr * (KS + 2 * (a.fr | 1) + 1), Lo.SCc, KS, a.fc | 1);
    const int nrs = stage_r ? c.nrs : 0, ncs = stage_c ? c.ncs : 0;
    for (int e = tid; e < nrs * a.KP; e += nt)
        cp_async4(r.P + (e / a.KP) * KS + e % a.KP, a.L + c.first_r * a.KP + e);
    for (int e = tid; e < ncs * a.KP; e += nt)
        cp_async4(q.P + (e / a.KP) * KS + e % a.KP, a.R + c.first_c * a.KP + e);
    for (int e = tid; e < nrs * a.fr; e += nt) {
        cp_async4(r.G + (e / a.fr) * (a.fr | 1) + e % a.fr, a.GbR + c.first_r * a.fr + e);
        cp_async4(r.H + (e / a.fr) * (a.fr | 1) + e % a.fr, a.HbR + c.first_r * a.fr + e);
    }
    for (int e = tid; e < ncs * a.fc; e += nt) {
        cp_async4(q.G + (e / a.fc) * (a.fc | 1) + e % a.fc, a.GbC + c.first_c * a.fc + e);
        cp_async4(q.H + (e / a.fc) * (a.fc | 1) + e % a.fc, a.HbC + c.first_c * a.fc + e);
    }
    for (int e = tid; e < nrs; e += nt) cp_async4(r.C + e, a.cntR + c.first_r + e);
    for (int e = tid; e < ncs; e += nt) cp_async4(q.C + e, a.cntC + c.first_c + e);
}

// The strip updates of cluster mode. Every thread of every CTA of the cluster
// calls this (one cluster barrier). The parameter rows always go back to
// global memory; wb_r / wb_c: write back that side's smoothed derivatives and
// visit counts too (else only the staged counts advance: a side kept resident
// in shared memory by the persistent kernel).
__device__ __forceinline__ void cl_update(const StepArgs& a, const TcLayout& Lo, uint8_t* sm, const ClSlice& c,
                                          const BlockGeo& g, float rhoc_blk, int nTI, int nTJ, bool wb_r = true,
                                          bool wb_c = true) {
    const int KS = a.KP + 1, NSr = a.fr | 1, NSc = a.fc | 1;
    const ClStage r = cl_stage_ptrs((float*)(sm + Lo.off_st), Lo.SRr, KS, NSr);
    const ClStage q = cl_stage_ptrs(r.P + (size_t)Lo.SRr * (KS + 2 * NSr + 1), Lo.SCc, KS, NSc);
    cp_async_wait_all();
    cluster_sync();  // every tile's partials are in their owners' slots; the slices are staged
    const float* prow = (const float*)(sm + Lo.off_cp);
    const float* pcol = prow + (size_t)a.TJ * 2 * a.fr * Lo.SRr;
    const float scale_r = (float)a.m / (float)g.mJ, scale_c = (float)a.n / (float)g.nI;
    const int tot_r = c.nrs * a.fr, total = tot_r + c.ncs * a.fc;
    for (int e = threadIdx.x; e < total; e += NTH) {
        const bool rowside = e < tot_r;
        const int nf = rowside ? a.fr : a.fc;
        const int no = rowside ? c.nrs : c.ncs;
        const int SR = rowside ? Lo.SRr : Lo.SCc;
        const int e2 = rowside ? e : e - tot_r;
        const int cc = e2 / no, o = e2 - cc * no;
        const int nsl = rowside ? nTJ : nTI;
        const float* slot = (rowside ? prow : pcol) + (size_t)cc * SR + o;
        const size_t sstride = (size_t)2 * nf * SR, hofs = (size_t)nf * SR;
        float gs = 0.f, hs = 0.f;
        for (int t = 0; t < nsl; t++) {
            gs += slot[t * sstride];
            hs += slot[t * sstride + hofs];
        }
        const ClStage& st = rowside ? r : q;
        const int NS = rowside ? NSr : NSc;
        const int col = rowside ? 1 + a.p + cc : (cc < a.p ? 1 + cc : 1 + a.q + cc);
        const float lam = rowside ? (cc < a.q ? a.lam[1] : a.lam[2]) : (cc < a.p ? a.lam[0] : a.lam[3]);
        const float rc = a.bias_corr ? rhoc_blk * bias_visit(a.a1, a.a2, st.C[o] + 1) : rhoc_blk;
        smoothed_step(st.P[o * KS + col], st.G[o * NS + cc], st.H[o * NS + cc], gs, hs, rowside ? scale_r : scale_c,
                      lam, a, rc);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < c.nrs * a.KP; e += NTH) a.L[c.first_r * a.KP + e] = r.P[(e / a.KP) * KS + e % a.KP];
    for (int e = threadIdx.x; e < c.ncs * a.KP; e += NTH) a.R[c.first_c * a.KP + e] = q.P[(e / a.KP) * KS + e % a.KP];
    for (int e = threadIdx.x; e < (wb_r ? c.nrs * a.fr : 0); e += NTH) {
        a.GbR[c.first_r * a.fr + e] = r.G[(e / a.fr) * NSr + e % a.fr];
        a.HbR[c.first_r * a.fr + e] = r.H[(e / a.fr) * NSr + e % a.fr];
    }
    for (int e = threadIdx.x; e < (wb_c ? c.ncs * a.fc : 0); e += NTH) {
        a.GbC[c.first_c * a.fc + e] = q.G[(e / a.fc) * NSc + e % a.fc];
        a.HbC[c.first_c * a.fc + e] = q.H[(e / a.fc) * NSc + e % a.fc];
    }
    for (int e = threadIdx.x; e < c.nrs; e += NTH) {
        const int v = r.C[e] + 1;
        if (wb_r)
            a.cntR[c.first_r + e] = v;
        else
            r.C[e] = v;
    }
    for (int e = threadIdx.x; e < c.ncs; e += NTH) {
        const int v = q.C[e] + 1;
        if (wb_c)
            a.cntC[c.first_c + e] = v;
        else
            q.C[e] = v;
    }
}

// EPI: 0 = any model (weights, family and moment sums read at run time); EPI_NB / EPI_PO = negative binomial /
// Poisson without weights and without the NB moment sums, decided at compile time (fewer instructions per entry).
constexpr int EPI_ANY = 0, EPI_NB = 1, EPI_PO = 2;

// ---- the phases of one tile. COH: model state is read through L2 only (the
// persistent kernel, where other CTAs wrote it during the same launch).
// Epilogue: warp (q, cq) owns rows 32q.. and columns 32cq..32cq+31 of the tile;
// Ddot and Dddot go as BF16 into one swizzled tile over the dead eta operands.
template <bool Y16, int EPI>
__device__ __forceinline__ void epilogue(const StepArgs& a, const TcLayout& Lo, uint8_t* sm, uint32_t tb, int64_t row0,
                                         int64_t col0, int nr, int nc, float alpha, float& s1, float& s2) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool nb = EPI == EPI_ANY ? a.family == GMF_NEGBIN : EPI == EPI_NB;
    const bool glm = EPI == EPI_ANY && a.family >= GMF_GAUSSIAN;  // the other families of Table S1
    const bool moments = EPI == EPI_ANY && scalar_estimated(a.family, a.alpha_mode);
    const uint8_t* Ys = sm;
    uint8_t* Dd = sm + Lo.off_dd;
    uint8_t* DDd = sm + Lo.off_ddd;
    const int q = warp & 3, cq = warp >> 2;
    const int i = 32 * q + lane;
    const bool row_ok = i < nr;
    const float* Wrow = (EPI == EPI_ANY && a.W) ? a.W + (row0 + i) * a.m + col0 : nullptr;
    const int jc = 32 * cq;
    uint32_t ev[32];
    tmem_ld32(tb + ((uint32_t)(32 * q) << 16) + (uint32_t)jc, ev);
    tmem_wait_ld();
#pragma unroll
    for (int gq = 0; gq < 4; gq++) {
        const int j0 = jc + 8 * gq;
        float y[8];
        if (Y16) {
            const uint4 u = *(const uint4*)(Ys + (j0 >> 6) * ATOM + sw128_off(i, (j0 & 63) * 2));
            const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int t = 0; t < 4; t++) {
                y[2 * t] = (float)(uu[t] & 0xFFFFu);
                y[2 * t + 1] = (float)(uu[t] >> 16);
            }
        } else {
            const uint32_t byte = (uint32_t)(j0 & 31) * 4u;
            const int4 u0 = *(const int4*)(Ys + (j0 >> 5) * ATOM + sw128_off(i, byte));
            const int4 u1 = *(const int4*)(Ys + (j0 >> 5) * ATOM + sw128_off(i, byte + 16));
            if (EPI == EPI_ANY && a.yf32) {  // float32 responses: the same 4-byte tile
                y[0] = __int_as_float(u0.x); y[1] = __int_as_float(u0.y); y[2] = __int_as_float(u0.z);
                y[3] = __int_as_float(u0.w); y[4] = __int_as_float(u1.x); y[5] = __int_as_float(u1.y);
                y[6] = __int_as_float(u1.z); y[7] = __int_as_float(u1.w);
            } else {
                y[0] = (float)u0.x; y[1] = (float)u0.y; y[2] = (float)u0.z; y[3] = (float)u0.w;
                y[4] = (float)u1.x; y[5] = (float)u1.y; y[6] = (float)u1.z; y[7] = (float)u1.w;
            }
        }
        float dd[8], ddd[8];
#pragma unroll
        for (int t = 0; t < 8; t++) {
            if (glm) {
                const int j = j0 + t;
                const bool valid = row_ok && j < nc;
                const float wv = (Wrow && valid) ? __ldg(Wrow + j) : 1.f;
                const float e = fminf(fmaxf(__uint_as_float(ev[8 * gq + t]), -a.clamp), a.clamp);
                const float mu = glm_mean(a.family, e);
                const bool miss = y_missing(a, y[t]);
                const float yv = miss ? mu : y[t];
                float d1, d2;
                glm_derivs(a.family, yv, mu, alpha, d1, d2);
                const float wf = valid ? wv : 0.f;
                dd[t] = wf * d1;
                ddd[t] = wf * d2;
                if (moments && valid && !miss) {
                    s1 += wv * (yv - mu) * (yv - mu) / glm_variance(a.family, mu);
                    s2 += 1.f;
                }
                continue;
            }
            const int j = j0 + t;
            const bool valid = row_ok && j < nc;
            const float wv = (Wrow && valid) ? __ldg(Wrow + j) : 1.f;
            const float e = fminf(fmaxf(__uint_as_float(ev[8 * gq + t]), -a.clamp), a.clamp);
            const float mu = __expf(e);
            if (EPI == EPI_ANY && a.missing && y[t] == a.ymiss) y[t] = mu;  // imputation y <- mu (Sec. 3.2)
            const float aj = (EPI == EPI_ANY && a.alpha_col && valid) ? __ldg(a.alpha_col + col0 + j) : alpha;
            const float f = nb ? __fdividef(aj, aj + mu) : 1.f;
            const float wf = valid ? wv * f : 0.f;
            dd[t] = wf * (y[t] - mu);
            ddd[t] = wf * mu;
            if (moments && valid) {
                s1 = fmaf(wv * mu, mu, s1);
                s2 += wv * ((y[t] - mu) * (y[t] - mu) - mu);
            }
        }
        const uint32_t off = (uint32_t)(j0 >> 6) * ATOM + sw128_off(i, (j0 & 63) * 2);
        st_shared_v4(Dd + off, pack_bf16x2(dd[0], dd[1]), pack_bf16x2(dd[2], dd[3]), pack_bf16x2(dd[4], dd[5]),
                     pack_bf16x2(dd[6], dd[7]));
        st_shared_v4(DDd + off, pack_bf16x2(ddd[0], ddd[1]), pack_bf16x2(ddd[2], ddd[3]), pack_bf16x2(ddd[4], ddd[5]),
                     pack_bf16x2(ddd[6], ddd[7]));
    }
}

// Thread 0: Ddot R_f, Dddot R_f^2 (row side) and Ddot' L_f, Dddot' L_f^2 (column side).
__device__ __forceinline__ void issue_contractions(const TcLayout& Lo, uint8_t* sm, uint32_t tb, uint64_t* bar) {
    const uint8_t* Dd = sm + Lo.off_dd;
    const uint8_t* DDd = sm + Lo.off_ddd;
    const uint8_t* RF = sm + Lo.off_rf;
    const uint8_t* RF2 = sm + Lo.off_rf2;
    const uint8_t* LF = sm + Lo.off_lf;
    const uint8_t* LF2 = sm + Lo.off_lf2;
    const uint32_t idr = idesc_bf16(TT, Lo.NR, 0, 0);
    const uint32_t atr = (uint32_t)Lo.NR * 128u;
    for (int ks = 0; ks < TT / 16; ks++) {
        const uint32_t aoff = (uint32_t)(ks >> 2) * ATOM + (uint32_t)(ks & 3) * 32u;
        const uint32_t boff = (uint32_t)(ks >> 2) * atr + (uint32_t)(ks & 3) * 32u;
        umma_bf16(tb + Lo.t_row, sdesc(smem_u32(Dd) + aoff, 16, 1024, SWIZZLE_128B),
                  sdesc(smem_u32(RF) + boff, 16, 1024, SWIZZLE_128B), idr, ks > 0);
        umma_bf16(tb + Lo.t_row + Lo.NR, sdesc(smem_u32(DDd) + aoff, 16, 1024, SWIZZLE_128B),
                  sdesc(smem_u32(RF2) + boff, 16, 1024, SWIZZLE_128B), idr, ks > 0);
    }
    const uint32_t idc = idesc_bf16(TT, Lo.NC, 1, 0);
    const uint32_t atc = (uint32_t)Lo.NC * 128u;
    for (int ks = 0; ks < TT / 16; ks++) {
        const uint32_t aoff = (uint32_t)ks * 2048u;  // 16 tile rows = two 8-row groups
        const uint32_t boff = (uint32_t)(ks >> 2) * atc + (uint32_t)(ks & 3) * 32u;
        umma_bf16(tb + Lo.t_col, sdesc(smem_u32(Dd) + aoff, ATOM, 1024, SWIZZLE_128B),
                  sdesc(smem_u32(LF) + boff, 16, 1024, SWIZZLE_128B), idc, ks > 0);
        umma_bf16(tb + Lo.t_col + Lo.NC, sdesc(smem_u32(DDd) + aoff, ATOM, 1024, SWIZZLE_128B),
                  sdesc(smem_u32(LF2) + boff, 16, 1024, SWIZZLE_128B), idc, ks > 0);
    }
    umma_commit(bar);
}

// Warps 0-3 read the row sums, warps 4-7 the column sums, from TMEM into the
// per-tile partial slots (global memory), or in cluster mode into the owners'
// slots (distributed shared memory).
template <bool CL>
__device__ __forceinline__ void store_partials(const StepArgs& a, const TcLayout& Lo, uint8_t* sm, uint32_t tb, int k,
                                               int ti, int tj, int nr, int nc) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp >= 8) return;
    const int q = warp & 3;
    const uint32_t lanes = (uint32_t)(32 * q) << 16;
    const int o = 32 * q + lane;   // tile row (warps 0-3) or tile column (warps 4-7)
    const bool rowside = warp < 4;
    const int NF = rowside ? Lo.NR : Lo.NC;
    const int nf = rowside ? a.fr : a.fc;
    const uint32_t tg = tb + lanes + (rowside ? Lo.t_row : Lo.t_col);
    float* dst = rowside ? a.partR + (size_t)((k * a.TI + ti) * a.TJ + tj) * TT * 2 * a.fr
                         : a.partC + (size_t)((k * a.TJ + tj) * a.TI + ti) * TT * 2 * a.fc;
    // cluster mode: slot `src` of the owner of row (column) o, at index o - own * SR
    const int SR = rowside ? Lo.SRr : Lo.SCc;
    const int own = CL ? o / SR : 0, ol = o - own * SR, src = rowside ? tj : ti;
    const uint32_t slots = CL ? mapa_shared(smem_u32(sm + Lo.off_cp) +
                                                (rowside ? 0u : (uint32_t)(4 * a.TJ * 2 * a.fr * Lo.SRr)),
                                            rowside ? (uint32_t)(own + ti * a.TJ) : (uint32_t)(tj + own * a.TJ))
                              : 0u;
    const bool o_ok = o < (rowside ? nr : nc);
    for (int c0 = 0; c0 < NF; c0 += 16) {
        uint32_t rg[16], rh[16];
        tmem_ld16(tg + (uint32_t)c0, rg);
        tmem_ld16(tg + (uint32_t)(NF + c0), rh);
        tmem_wait_ld();
        if (o_ok) {
#pragma unroll
            for (int u = 0; u < 16; u++) {
                const int c = c0 + u;
                if (c < nf) {
                    if (CL) {
                        st_dsmem_f32(slots + 4u * (uint32_t)((src * 2 * nf + c) * SR + ol), __uint_as_float(rg[u]));
                        st_dsmem_f32(slots + 4u * (uint32_t)((src * 2 * nf + nf + c) * SR + ol),
                                     __uint_as_float(rh[u]));
                    } else {
                        dst[(size_t)c * TT + o] = __uint_as_float(rg[u]);
                        dst[(size_t)(nf + c) * TT + o] = __uint_as_float(rh[u]);
                    }
                }
            }
        }
    }
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void cluster_arrive_release() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}

// One thread: spin until *cnt >= target. Gives up, flagging a time-out, after
// limit_ns of the global timer (2 s unless gmf_set_wait_limit changed it) or as
// soon as another CTA has flagged one.
__device__ __forceinline__ void wait_count(const unsigned* cnt, unsigned target, unsigned* err, uint64_t limit_ns) {
    if (ld_acquire_u32(cnt) >= target) return;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (ld_acquire_u32(cnt) >= target) return;
        if (*(volatile unsigned*)err & GMF_DEVERR_TIMEOUT) return;
        if (global_ns() - t0 > limit_ns) {
            atomicOr(err, GMF_DEVERR_TIMEOUT);
            return;
        }
    }
}

// ---- the item queue of the dataflow epoch (sweep_tc_flow). One per CTA, in
// shared memory. A CTA holds the item it works on (buffer cur), the next one,
// decoded into buffer cur ^ 1 while the current one runs, and the ticket
// after that (next).
struct FlowQueue {
    unsigned* ctr;       // the launch's counters
    const int* gstart;   // [groups + 1]: first ticket of each group
    const int4* gent;    // [groups]: group entries
    int total;           // tickets of the launch
    int next;            // the ticket taken ahead
    int g;               // group of the last decoded ticket
    int4 item[2];        // {ticket, index in its group}
    int4 ent[2];         // the group entry
    int ready[2];        // 1: the item's prerequisites were already met when looked at ahead
};

// Prerequisite i (0-2) of an item with group entry e: the counter (nullptr:
// none) and the count it must reach (see sweep_tc_flow).
__device__ __forceinline__ const unsigned* flow_dep(const StepArgs& a, unsigned* ctr, int4 e, int i,
                                                    unsigned& target) {
    const int pi = e.x >> 1, wr = pi / a.per, k = pi - wr * a.per;
    if (e.x & 1) {  // update units: the block's tiles
        target = (unsigned)e.y;
        return i == 0 ? ctr + 3 + a.per + k : nullptr;
    }
    if (i == 0) {  // tiles: the previous update of the fixed strip (and of the block slot's partial slots)
        target = (unsigned)e.y;
        return e.y > 0 ? ctr + 3 + k : nullptr;
    }
    if (i == 1) {  // the last update of the moving strip
        target = (unsigned)e.w;
        return e.w > 0 ? ctr + 3 + 2 * a.per + e.z : nullptr;
    }
    target = (unsigned)wr;  // the NB shape after the previous sweep
    return (scalar_estimated(a.family, a.alpha_mode) && wr > 0) ? ctr + 1 : nullptr;
}

// One thread: decode the ticket taken ahead into buffer nb and take another.
__device__ __forceinline__ void flow_take(FlowQueue& q, int nb) {
    const int t = q.next;
    q.ready[nb] = 0;
    if (t < q.total) {
        int g = q.g;
        while (__ldg(q.gstart + g + 1) <= t) g++;
        q.g = g;
        q.ent[nb] = __ldg(q.gent + g);
        q.item[nb] = make_int4(t, t - __ldg(q.gstart + g), 0, 0);
        q.next = (int)atomicAdd(q.ctr, 1u);
    } else {
        q.item[nb] = make_int4(t, 0, 0, 0);
    }
}

// One warp, after its lane 0 decoded buffer nb: look once (lanes 0-2, acquire)
// at the item's prerequisites; if all are met its wait is skipped.
__device__ __forceinline__ void flow_look(FlowQueue& q, const StepArgs& a, int nb) {
    __syncwarp();
    const int lane = threadIdx.x & 31;
    bool ok = true;
    if (lane < 3 && q.item[nb].x < q.total) {
        unsigned target;
        const unsigned* c = flow_dep(a, q.ctr, q.ent[nb], lane, target);
        if (c) ok = ld_acquire_u32(c) >= target;
    }
    const unsigned all = __ballot_sync(0xffffffffu, ok);
    if (lane == 0) q.ready[nb] = all == 0xffffffffu;
}

// All threads: threads 0-2 wait for the prerequisites of the item in buffer
// cur unless they were met at the look ahead; with take_next thread 3 decodes
// the next item meanwhile.
__device__ __forceinline__ void flow_wait(FlowQueue& q, const StepArgs& a, int cur, bool take_next) {
    const int t = threadIdx.x;
    if (t < 3 && !q.ready[cur]) {
        unsigned target;
        const unsigned* c = flow_dep(a, q.ctr, q.ent[cur], t, target);
        if (c) wait_count(c, target, a.err, a.wait_ns);
    } else if (t == 3 && take_next) {
        flow_take(q, cur ^ 1);
    }
    __syncthreads();
}

// The CTA's three mbarriers (count tile, eta MMA, contraction MMAs) and its TMEM base.
struct TileSync {
    uint64_t bars[3];
    uint32_t tmem_base;
};

// One tile (ti, tj) of block k of sweep w for the model whose arguments are a
// / Lo. CL: cluster mode (the strip updates run here). The mbarriers are
// initialised here when init_bars, else they were initialised before and par
// is the parity of their next phase (a CTA that runs several tiles). With
// tmem_held the caller owns a TMEM allocation of at least Lo.tmem_cols columns
// at ts.tmem_base (a CTA may allocate only until it gives up its permit, so a
// CTA running several tiles allocates once); else the tile allocates and frees
// its own. COH: model state is read through L2 only (other CTAs of the same
// launch wrote it). fq: the dataflow queue whose item (buffer cur) this tile
// is -- it waits for the item's prerequisites where a per-sweep launch waits
// for the previous launch, and decodes and looks at the CTA's next item while
// warps 0-7 store the partial sums; nullptr elsewhere. Returns true when the
// tile was active (its mbarriers completed one phase).
template <bool Y16, bool CL, int EPI, bool COH = false>
__device__ __forceinline__ bool tc_tile(const StepArgs& a, const TcLayout& Lo, const CUtensorMap* ymap_p, int w,
                                        int k, int ti, int tj, uint8_t* smraw, TileSync& ts, uint32_t par,
                                        bool init_bars, bool tmem_held, FlowQueue* fq = nullptr, int cur = 0) {
    uint64_t* bars = ts.bars;
    const int tid = threadIdx.x, warp = tid >> 5;
    const BlockGeo g = fq ? block_geo_strip(a, fq->ent[cur].z, k) : block_geo(a, w, k);
    const int nTI = (int)((g.nI + TT - 1) / TT), nTJ = (int)((g.mJ + TT - 1) / TT);
    const bool active = ti < nTI && tj < nTJ;
    float s1 = 0.f, s2 = 0.f;

    uint8_t* sm = smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u);
    ClSlice cls{};
    float rhoc_blk = 0.f;  // the block's step factor, fixed for the epoch
    if (CL) {
        rhoc_blk = a.rhoc[w * a.per + k];
        cls = cl_slice(a, Lo, g, ti, tj, nTI, nTJ);
        cluster_arrive_relaxed();  // waited for before the first store into a peer (all peers have started)
    }
    if (active) {
        const int64_t row0 = g.r0 + (int64_t)ti * TT, col0 = g.c0 + (int64_t)tj * TT;
        const int nr = (int)min((int64_t)TT, g.nI - (int64_t)ti * TT);
        const int nc = (int)min((int64_t)TT, g.mJ - (int64_t)tj * TT);

        if (tid == 0 && init_bars) {
            mbar_init(&bars[0], 1);
            mbar_init(&bars[1], 1);
            mbar_init(&bars[2], 1);
            fence_mbar_init();
        }
        if (warp == 0 && !tmem_held) tmem_alloc(&ts.tmem_base, Lo.tmem_cols);
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        const uint32_t tb = ts.tmem_base;

        if (tid == 0) issue_counts(Lo, ymap_p, sm, row0, col0, &bars[0]);
        // the counts are read-only; everything below reads or writes model state
        // that the previous sweep's update launch may still be writing. The
        // next launch (this sweep's update) may start once every CTA is here,
        // i.e. once the previous update has completed.
        if (fq)
            flow_wait(*fq, a, cur, false);
        else
            grid_dependency_wait();
        grid_launch_dependents();
        const float alpha = COH ? __ldcg(a.alpha) : *a.alpha;

        build_operands<COH>(a, Lo, sm, row0, col0, nr, nc);
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();

        if (tid == 0) issue_eta(Lo, sm, tb, &bars[1]);
        bool ok = cta_wait(&bars[0], par, a.err);
        ok = cta_wait(&bars[1], par, a.err) && ok;
        tc_fence_after();

        if (ok) epilogue<Y16, EPI>(a, Lo, sm, tb, row0, col0, nr, nc, alpha, s1, s2);
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();

        if (ok && tid == 0) issue_contractions(Lo, sm, tb, &bars[2]);
        // warps 8-15 have no partials to read: they start the update slices' copies
        if (CL) cl_stage_issue(a, Lo, sm, cls, NTH / 2, NTH / 2);
        if (fq && tid == 256) flow_take(*fq, cur ^ 1);  // its ticket's round trip overlaps the MMAs
        if (ok) ok = cta_wait(&bars[2], par, a.err);
        tc_fence_after();
        if (CL) cluster_wait();

        if (fq && warp == 8) flow_look(*fq, a, cur ^ 1);  // beside the partial stores of warps 0-7
        if (ok) store_partials<CL>(a, Lo, sm, tb, k, ti, tj, nr, nc);
        if (!ok && tid == 0) atomicOr(a.err, GMF_DEVERR_TIMEOUT);
        if (tmem_held) fence_proxy_async_smem();  // a next tile of this CTA loads its counts over this one's operands
        tc_fence_before();
        __syncthreads();
        if (warp == 0 && !tmem_held) tmem_dealloc(tb, Lo.tmem_cols);
    } else {
        if (fq)  // before writing this sweep's moment slot
            flow_wait(*fq, a, cur, true);
        else
            grid_dependency_wait();
        grid_launch_dependents();
        if (CL) {
            cl_stage_issue(a, Lo, sm, cls, 0, NTH);
            cluster_wait();
        }
    }
    tile_moments<NTH>(a, k, ti, tj, s1, s2);
    if (CL) {
        cl_update(a, Lo, sm, cls, g, rhoc_blk, nTI, nTJ);
        // NB shape: the last CTA of the sweep pools the moment sums (App. B)
        if (scalar_estimated(a.family, a.alpha_mode)) {
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                const unsigned total = (unsigned)(a.TJ * a.TI * a.per);
                if (atomicAdd(a.nbctr, 1u) == total - 1) {
                    __threadfence();
                    nb_shape_update(a, w);
                    *a.nbctr = 0u;
                }
            }
        }
    }
    return active;
}

// ---- persistent epoch (cluster mode). One launch runs the sweeps [w0, w1);
// cluster k takes block k of every sweep. The block's fixed strip (column
// strip k; row strip k when the roles swap) belongs to cluster k alone: its
// slices' smoothed derivatives and visit counts stay in shared memory for the
// whole launch (written back after the last block), its parameter rows go
// back after every block for the peers' next operands, ordered by the cluster
// barrier. Only the moving strip passes between clusters. Every CTA adds one
// to the moving strip's completion count after its write-back (a release
// reduction; skipped after the launch's last block, which nothing later
// reads); block k of sweep w waits (acquire) until the count of its moving
// strip reaches need[w][k] -- the visits of that strip by the earlier sweeps
// of the launch -- times the cluster size. Every wait therefore points to an earlier sweep, and since all
// clusters are resident at once (checked with the occupancy query before this
// mode is chosen) they cannot wait in a cycle. An acquiring look one block
// ahead, while the contractions run, usually finds the next strip ready. State
// written during the launch is read through L2 only. The next block's count
// tile is loaded while the current block finishes. Results equal the
// per-sweep launches bit for bit (same phases, same sums in the same order).
// Block k of a sweep whose offset sigma[w] is sg (block_geo without the load).
__device__ __forceinline__ BlockGeo block_geo_sg(const StepArgs& a, int sg, int k) {
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

template <bool Y16, int EPI>
__global__ void __launch_bounds__(NTH, 1)
    sweep_tc_epoch(StepArgs a, TcLayout Lo, const __grid_constant__ CUtensorMap ymap, int w0, int w1) {
    extern __shared__ __align__(1024) uint8_t smraw[];
    __shared__ uint64_t bars[3];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int tj = blockIdx.x, ti = blockIdx.y, k = blockIdx.z;
    uint8_t* sm = smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u);
    const bool fix_r = a.swap != 0, fix_c = a.swap == 0;  // the side of the fixed strip

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&bars[2], 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&tmem_base, Lo.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tb = tmem_base;
    const float alpha = *a.alpha;  // the shape is not re-estimated inside this launch
    float s1 = 0.f, s2 = 0.f;      // (no moment sums in this mode)
    uint32_t ph = 0;               // parity of the mbarrier phases of the next active block
    bool dead = false;             // a bounded wait of this CTA timed out: no further copies or MMAs
    bool y_next = false;           // the count tile of the next block is already requested
    const unsigned ncta = (unsigned)(a.TI * a.TJ);
    __shared__ int s_ready;        // a block whose moving strip an early look found written back
    if (tid == 0) s_ready = -1;    // (ordered before its first read by the barrier at the top)
    // schedule of the current block; the next block's is loaded one block ahead
    int sg = a.sigma[w0];
    float rhoc_blk = a.rhoc[w0 * a.per + k];
    unsigned need = (unsigned)a.need[w0 * a.per + k];

    cluster_arrive_relaxed();  // matched by the wait at the top of the first sweep
    for (int w = w0; w < w1; w++) {
        const BlockGeo g = block_geo_sg(a, sg, k);
        const int nTI = (int)((g.nI + TT - 1) / TT), nTJ = (int)((g.mJ + TT - 1) / TT);
        const bool active = ti < nTI && tj < nTJ && !dead;
        const int64_t row0 = g.r0 + (int64_t)ti * TT, col0 = g.c0 + (int64_t)tj * TT;
        if (active && !y_next && tid == 0) issue_counts(Lo, &ymap, sm, row0, col0, &bars[0]);
        y_next = false;
        const ClSlice cls = cl_slice(a, Lo, g, ti, tj, nTI, nTJ);
        const int strip = a.swap ? (int)(g.c0 / a.nb_col) : (int)(g.r0 / a.nb_row);
        cluster_wait();  // the peers finished the previous block: fixed strip written, slots free
        if (tid == 0 && s_ready != w) wait_count(a.strip_done + strip, need * ncta, a.err, a.wait_ns);
        __syncthreads();
        tc_fence_after();
        const int wn = min(w + 1, w1 - 1);  // (the last block loads its own values again)
        const int sg_next = a.sigma[wn];
        const float rhoc_next = a.rhoc[wn * a.per + k];
        const unsigned need_next = (unsigned)a.need[wn * a.per + k];

        if (active) {
            const int nr = (int)min((int64_t)TT, g.nI - (int64_t)ti * TT);
            const int nc = (int)min((int64_t)TT, g.mJ - (int64_t)tj * TT);
            build_operands<true>(a, Lo, sm, row0, col0, nr, nc);
            fence_proxy_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();

            if (tid == 0) issue_eta(Lo, sm, tb, &bars[1]);
            bool ok = cta_wait(&bars[0], ph, a.err);
            ok = cta_wait(&bars[1], ph, a.err) && ok;
            tc_fence_after();

            if (ok) epilogue<Y16, EPI>(a, Lo, sm, tb, row0, col0, nr, nc, alpha, s1, s2);
            fence_proxy_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();

            if (ok && tid == 0) issue_contractions(Lo, sm, tb, &bars[2]);
            if (ok && w + 1 < w1) {  // the count tile is no longer read: request the next block's
                const BlockGeo gn = block_geo_sg(a, sg_next, k);
                if (ti * TT < gn.nI && tj * TT < gn.mJ) {
                    if (tid == 0)
                        issue_counts(Lo, &ymap, sm, gn.r0 + (int64_t)ti * TT, gn.c0 + (int64_t)tj * TT, &bars[0]);
                    y_next = true;
                }
            }
            cl_stage_issue(a, Lo, sm, cls, NTH / 2, NTH / 2, !fix_r || w == w0, !fix_c || w == w0);
            if (tid == 32 && w + 1 < w1) {
                // an early look (acquire) at the next block's moving strip by an idle warp
                // while the contractions run; when it is written back, the next block
                // does not poll (the barriers in between order the look before its reads)
                const BlockGeo gn = block_geo_sg(a, sg_next, k);
                const int sn = a.swap ? (int)(gn.c0 / a.nb_col) : (int)(gn.r0 / a.nb_row);
                if (ld_acquire_u32(a.strip_done + sn) >= need_next * ncta) s_ready = w + 1;
            }
            if (ok) ok = cta_wait(&bars[2], ph, a.err);
            tc_fence_after();
            if (ok) store_partials<true>(a, Lo, sm, tb, k, ti, tj, nr, nc);
            tc_fence_before();
            if (!ok) {
                if (tid == 0) atomicOr(a.err, GMF_DEVERR_TIMEOUT);
                // a requested count tile is drained (bounded) before the CTA stops copying
                if (y_next) mbar_wait(&bars[0], ph ^ 1u, WAIT_POLLS);
                y_next = false;
                dead = true;
            }
            ph ^= 1u;
        } else {
            cl_stage_issue(a, Lo, sm, cls, 0, NTH, !fix_r || w == w0, !fix_c || w == w0);
        }
        cl_update(a, Lo, sm, cls, g, rhoc_blk, nTI, nTJ, !fix_r || w == w1 - 1, !fix_c || w == w1 - 1);
        __syncthreads();
        // publish this CTA's rows of the moving strip (release, cumulative over the
        // CTA through the barrier above) while the cluster barrier's release drains
        if (tid == 32 && w + 1 < w1) red_release_add_u32(a.strip_done + strip, 1u);
        cluster_arrive_release();  // this CTA's slices are written back and its partial slots free
        sg = sg_next;
        rhoc_blk = rhoc_next;
        need = need_next;
    }
    cluster_wait();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tb, Lo.tmem_cols);
}

// With 16-bit counts and d up to ~27 a tile takes under half of an SM's shared
// memory and TMEM, so two CTAs share an SM (one's epilogue runs while the
// other builds operands or waits for its MMAs): registers are capped to fit.
template <bool Y16, int EPI>
__global__ void __launch_bounds__(NTH, Y16 ? 2 : 1)
    sweep_tc_kernel(StepArgs a, TcLayout Lo, const __grid_constant__ CUtensorMap ymap, int w) {
    extern __shared__ __align__(1024) uint8_t smraw[];
    __shared__ TileSync ts;
    tc_tile<Y16, false, EPI>(a, Lo, &ymap, w, block_of_slot(a, blockIdx.z), blockIdx.y, blockIdx.x, smraw, ts, 0u,
                             true, false);
}

// Cluster mode: launched with cluster dimensions (TJ, TI, 1), one cluster per block.
template <bool Y16, int EPI>
__global__ void __launch_bounds__(NTH, 1)
    sweep_tc_cluster(StepArgs a, TcLayout Lo, const __grid_constant__ CUtensorMap ymap, int w) {
    extern __shared__ __align__(1024) uint8_t smraw[];
    __shared__ TileSync ts;
    tc_tile<Y16, true, EPI>(a, Lo, &ymap, w, block_of_slot(a, blockIdx.z), blockIdx.y, blockIdx.x, smraw, ts, 0u,
                            true, false);
}

// The kernel of a handle: counts type, cluster mode and epilogue variant.
template <int EPI>
const void* tc_fn_epi(int y16, int cl) {
    if (cl) return y16 ? (const void*)sweep_tc_cluster<true, EPI> : (const void*)sweep_tc_cluster<false, EPI>;
    return y16 ? (const void*)sweep_tc_kernel<true, EPI> : (const void*)sweep_tc_kernel<false, EPI>;
}
const void* tc_fn(int y16, int cl, int epi) {
    return epi == EPI_NB ? tc_fn_epi<EPI_NB>(y16, cl) : epi == EPI_PO ? tc_fn_epi<EPI_PO>(y16, cl)
                                                                      : tc_fn_epi<EPI_ANY>(y16, cl);
}
template <int EPI>
const void* tc_epoch_fn_epi(int y16) {
    return y16 ? (const void*)sweep_tc_epoch<true, EPI> : (const void*)sweep_tc_epoch<false, EPI>;
}
const void* tc_epoch_fn(int y16, int epi) {
    return epi == EPI_NB ? tc_epoch_fn_epi<EPI_NB>(y16) : epi == EPI_PO ? tc_epoch_fn_epi<EPI_PO>(y16)
                                                                        : tc_epoch_fn_epi<EPI_ANY>(y16);
}

// Several models (ranks) sharing the count matrix, the partitions and the
// settings (so one epilogue variant serves all): blockIdx.z = slot * per + k,
// slot -> model through `order` (heaviest models first).
template <bool Y16, int EPI>
__global__ void __launch_bounds__(NTH, Y16 ? 2 : 1) sweep_tc_multi(const StepArgs* __restrict__ av, const TcLayout* __restrict__ lv,
                                                         const int* __restrict__ order, int per,
                                                         const __grid_constant__ CUtensorMap ymap, int w) {
    extern __shared__ __align__(1024) uint8_t smraw[];
    __shared__ StepArgs s_a;
    __shared__ TcLayout s_l;
    if (threadIdx.x == 0) {
        const int model = order[blockIdx.z / per];
        s_a = av[model];
        s_l = lv[model];
    }
    __syncthreads();
    __shared__ TileSync ts;
    tc_tile<Y16, false, EPI>(s_a, s_l, &ymap, w, blockIdx.z % per, blockIdx.y, blockIdx.x, smraw, ts, 0u, true, false);
}

// One sweep of several models as one persistent launch (cooperative, so every
// CTA is resident): the CTAs first take the tiles of every model's blocks,
// heaviest model first (slot order), one after another; then, past a grid
// barrier, the strip updates of every model (the update launch's units); then
// each model's NB shape. The same tile and update functions as the tile and
// update launches, in the same order of additions, so the results are equal
// bit for bit. The grid barrier is a counter raised by every CTA; each CTA
// waits (thread 0, bounded by the global timer: past wait_ns it flags
// GMF_DEVERR_TIMEOUT and goes on, so the launch ends) until the counter reaches
// the next multiple of the grid size. The counter is cleared before each epoch.
__device__ __forceinline__ void grid_barrier(unsigned* ctr, uint64_t wait_ns, unsigned* err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();  // this CTA's partial sums and moment sums, before its arrival
        const unsigned old = atomicAdd(ctr, 1u);
        const unsigned target = (old / gridDim.x + 1u) * gridDim.x;
        if (ld_acquire_u32(ctr) < target) {
            const uint64_t t0 = global_ns();
            while (ld_acquire_u32(ctr) < target) {
                if (*(volatile unsigned*)err & GMF_DEVERR_TIMEOUT) break;
                if (global_ns() - t0 > wait_ns) {
                    atomicOr(err, GMF_DEVERR_TIMEOUT);
                    break;
                }
            }
        }
    }
    __syncthreads();
}

// The CTA holds one TMEM allocation of tmem_cols columns (the widest model's)
// for all its tiles; the host keeps (CTAs per SM) x tmem_cols within the SM's
// 512 columns, so no allocation waits for a CTA that is itself waiting at the
// grid barrier.
template <bool Y16, int EPI>
__global__ void __launch_bounds__(NTH, Y16 ? 2 : 1)
    sweep_tc_multi_persist(const StepArgs* __restrict__ av, const TcLayout* __restrict__ lv,
                           const int* __restrict__ order, int nmod, int per, const __grid_constant__ CUtensorMap ymap,
                           int w, unsigned* gctr, unsigned long long wait_ns, unsigned* err, uint32_t tmem_cols) {
    extern __shared__ __align__(1024) uint8_t smraw[];
    __shared__ StepArgs s_a;
    __shared__ TcLayout s_l;
    __shared__ TileSync ts;
    __shared__ int s_cnt[UTC_SR];
    const int TI = av[0].TI, TJ = av[0].TJ;  // the same partitions for every model
    const int tiles = per * TI * TJ;
    uint32_t par = 0;
    bool init = true;
    if ((int)blockIdx.x < nmod * tiles && (threadIdx.x >> 5) == 0) tmem_alloc(&ts.tmem_base, tmem_cols);
    for (int it = blockIdx.x; it < nmod * tiles; it += gridDim.x) {
        const int slot = it / tiles, rem = it - slot * tiles;
        const int k = rem / (TI * TJ), r2 = rem - k * (TI * TJ);
        const int ti = r2 / TJ, tj = r2 - ti * TJ;
        __syncthreads();  // the previous tile no longer reads the shared arguments
        if (threadIdx.x == 0) {
            s_a = av[order[slot]];
            s_l = lv[order[slot]];
        }
        __syncthreads();
        if (tc_tile<Y16, false, EPI>(s_a, s_l, &ymap, w, k, ti, tj, smraw, ts, par, init, true)) {
            par ^= 1u;
            init = false;
        }
    }
    if ((int)blockIdx.x < nmod * tiles) {
        tc_fence_before();
        __syncthreads();
        if ((threadIdx.x >> 5) == 0) tmem_dealloc(ts.tmem_base, tmem_cols);
    }
    grid_barrier(gctr, wait_ns, err);
    const int units = utc_units(per, TI, TJ, TT);
    for (int it = blockIdx.x; it < nmod * units; it += gridDim.x) {
        const int slot = it / units;
        __syncthreads();
        if (threadIdx.x == 0) s_a = av[order[slot]];
        __syncthreads();
        update_unit_tc<true>(s_a, w, TT, it - slot * units, s_cnt);
    }
    if (threadIdx.x == 0)
        for (int mm = blockIdx.x; mm < nmod; mm += gridDim.x) nb_shape_update(av[mm], w);
}

// ---- dataflow epoch (tiles and updates of a sweep range in one persistent
// launch, for blocks too large for cluster mode). The work items are the
// tiles of block (w, k) -- group T(p), p = (w - w0) * per + k -- and that
// block's update units -- group U(p). Every CTA takes items in ticket order
// from a global counter. The host lays the groups out so that each item's
// prerequisites come earlier: T(p) before U(p), and before T(p) the update of
// the previous visit of each strip it reads (U(p - per) for the fixed strip,
// the last earlier visit of the moving strip). A CTA takes a ticket only when
// it runs, and holds at most the item it works on, the next one (decoded)
// and the ticket after it; so the smallest unfinished item is always held by
// a running CTA whose prerequisites are done, and the launch ends without any
// CTA having to be resident at the same time as another (no cooperative
// launch). The waits are bounded by the global timer all the same. A block's
// updates trail its tiles by a few groups, so the tiles of the next sweep fill
// the SMs that the last wave of a sweep leaves idle.
// Counters, cumulative over the launch and zeroed before it:
//   ctr[0]              tickets handed out
//   ctr[1]              NB shape updates done (alpha_mode 1)
//   ctr[2]              tiles done, all blocks (alpha_mode 1: the CTA finishing a sweep's last tile updates the shape)
//   ctr[3 + k]          update units done of block slot k (its fixed strip and its partial slots)
//   ctr[3 + per + k]    tiles done of block slot k
//   ctr[3 + 2 per + j]  moving-side update units done of moving strip j
// Group g (host-made, int4): tiles {2p, update units of slot k needed, moving
// strip j, moving-side units of j needed}; updates {2p + 1, tiles of slot k
// needed, j, 0}. Same tile and update functions, same sums in the same order
// as the per-sweep launches: the results are equal bit for bit.
template <bool Y16, int EPI>
__global__ void __launch_bounds__(NTH, Y16 ? 2 : 1)
    sweep_tc_flow(StepArgs a, TcLayout Lo, const __grid_constant__ CUtensorMap ymap, int w0,
                  const int4* __restrict__ gent, const int* __restrict__ gstart, int ngroups, unsigned* ctr,
                  uint32_t tmem_cols) {
    extern __shared__ __align__(1024) uint8_t smraw[];
    __shared__ TileSync ts;
    __shared__ int s_cnt[UTC_SR];
    __shared__ FlowQueue fq;
    const int tid = threadIdx.x, warp = tid >> 5;
    constexpr int nsl = TT / UTC_SR;
    if (warp == 0) tmem_alloc(&ts.tmem_base, tmem_cols);
    if (tid == 3) {
        fq.ctr = ctr;
        fq.gstart = gstart;
        fq.gent = gent;
        fq.total = gstart[ngroups];
        fq.g = 0;
        fq.next = (int)atomicAdd(ctr, 1u);
        flow_take(fq, 0);
    }
    __syncthreads();
    uint32_t par = 0;
    bool init = true;
    for (int buf = 0;; buf ^= 1) {
        const int4 it = fq.item[buf];
        if (it.x >= fq.total) break;
        const int4 e = fq.ent[buf];
        const int pi = e.x >> 1, idx = it.y;
        const int wr = pi / a.per, k = pi - wr * a.per, w = w0 + wr;
        if ((e.x & 1) == 0) {  // tile idx of block (w, k)
            if (tc_tile<Y16, false, EPI, true>(a, Lo, &ymap, w, k, idx / a.TJ, idx % a.TJ, smraw, ts, par, init, true,
                                               &fq, buf)) {
                par ^= 1u;
                init = false;
            }
            __syncthreads();
            if (tid == 32) {
                // the tile's partial (and moment) sums, before its count: a release by a thread that the
                // CTA barrier ordered after every other thread's stores
                red_release_add_u32(ctr + 3 + a.per + k, 1u);
                if (scalar_estimated(a.family, a.alpha_mode)) {
                    __threadfence();
                    if (atomicAdd(ctr + 2, 1u) + 1u == (unsigned)((wr + 1) * a.per * a.TI * a.TJ)) {
                        __threadfence();
                        nb_shape_update(a, w);
                        red_release_add_u32(ctr + 1, 1u);
                    }
                }
            }
        } else {  // update unit idx of block (w, k)
            flow_wait(fq, a, buf, false);
            // the widest side's column groups take warps 0 .. G-1; the last warp decodes and looks at the
            // next item meanwhile (it only waits at the update's barriers)
            if (warp == NTH / 32 - 1) {
                if ((tid & 31) == 0) flow_take(fq, buf ^ 1);
                flow_look(fq, a, buf ^ 1);
            }
            update_unit_tc<true>(a, w, TT, k * (a.TI + a.TJ) * nsl + idx, s_cnt, e.z);
            __syncthreads();
            if (tid == 32) {  // the slice's parameters and smoothed derivatives, before its counts
                red_release_add_u32(ctr + 3 + k, 1u);
                const bool rowside = idx < a.TI * nsl;
                if (rowside != (a.swap != 0)) red_release_add_u32(ctr + 3 + 2 * a.per + e.z, 1u);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(ts.tmem_base, tmem_cols);
}

template <int EPI>
const void* tc_flow_fn_epi(int y16) {
    return y16 ? (const void*)sweep_tc_flow<true, EPI> : (const void*)sweep_tc_flow<false, EPI>;
}
const void* tc_flow_fn(int y16, int epi) {
    return epi == EPI_NB ? tc_flow_fn_epi<EPI_NB>(y16) : epi == EPI_PO ? tc_flow_fn_epi<EPI_PO>(y16)
                                                                       : tc_flow_fn_epi<EPI_ANY>(y16);
}

template <int EPI>
const void* tc_persist_fn_epi(int y16) {
    return y16 ? (const void*)sweep_tc_multi_persist<true, EPI> : (const void*)sweep_tc_multi_persist<false, EPI>;
}
const void* tc_persist_fn(int y16, int epi) {
    return epi == EPI_NB ? tc_persist_fn_epi<EPI_NB>(y16) : epi == EPI_PO ? tc_persist_fn_epi<EPI_PO>(y16)
                                                                          : tc_persist_fn_epi<EPI_ANY>(y16);
}

template <int EPI>
const void* tc_multi_fn_epi(int y16) {
    return y16 ? (const void*)sweep_tc_multi<true, EPI> : (const void*)sweep_tc_multi<false, EPI>;
}
const void* tc_multi_fn(int y16, int epi) {
    return epi == EPI_NB ? tc_multi_fn_epi<EPI_NB>(y16) : epi == EPI_PO ? tc_multi_fn_epi<EPI_PO>(y16)
                                                                        : tc_multi_fn_epi<EPI_ANY>(y16);
}

int tc_cluster_layout(gmf_model* h, TcState* tc);
int tc_persist_check(gmf_model* h, TcState* tc);
int tc_flow_setup(gmf_model* h, TcState* tc);
void gmf_tc_release(TcState* tc);

int fail_str(std::string* err, const char* msg) {
    if (err) *err = msg;
    return GMF_ERR_ARG;
}

}  // namespace

// TMA descriptor of an n x m count matrix at Y: 128-byte boxes of TT rows, 128-byte swizzle.
static int tc_encode_y(const gmf_model* h, CUtensorMap* map, const void* Y) {
    const int es = h->y16 ? 2 : 4;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr) != cudaSuccess ||
        !fn)
        return GMF_ERR_CUDA;
    cuuint64_t dims[2] = {(cuuint64_t)h->m, (cuuint64_t)h->n};
    cuuint64_t strides[1] = {(cuuint64_t)h->m * es};
    cuuint32_t box[2] = {(cuuint32_t)(128 / es), (cuuint32_t)TT};
    cuuint32_t estr[2] = {1, 1};
    const CUresult cr = ((PFN_cuTensorMapEncodeTiled_v12000)fn)(
        map, h->y16 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_INT32, 2, (void*)Y, dims, strides, box,
        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return cr == CUDA_SUCCESS ? GMF_OK : GMF_ERR_CUDA;
}

// The tensor map of the handle's second count buffer (gmf_update_y_async).
int gmf_tc_set_ybuf(gmf_model* h, int idx, const void* Y) {
    if (!h->tc) return GMF_OK;
    return tc_encode_y(h, &((TcState*)h->tc)->ymap[idx], Y);
}

// Set up the tensor-core path of a handle: layout, TMA descriptor, attributes.
int gmf_tc_prepare_checked(gmf_model* h, std::string* err) {
    const int es = h->y16 ? 2 : 4;
    if ((h->m * es) % 16 != 0) return fail_str(err, "mixed precision needs m * sizeof(count) to be a multiple of 16 bytes");
    if (((int64_t)h->cfg.nb_col * es) % 16 != 0)
        return fail_str(err, "mixed precision needs nb_col * sizeof(count) to be a multiple of 16 bytes");
    TcState* tc = new TcState();
    memset(tc, 0, sizeof *tc);
    TcLayout& L = tc->lay;
    L.KP16 = (h->K + 15) & ~15;
    if (L.KP16 > 64) {
        delete tc;
        return fail_str(err, "mixed precision supports 1+p+q+d <= 64");
    }
    L.KA = (2 * L.KP16 + 63) / 64;
    L.NR = (std::max(h->fr, 1) + 15) & ~15;
    L.NC = (std::max(h->fc, 1) + 15) & ~15;
    L.JB = 128 / es;
    L.y_bytes = (uint32_t)(TT / L.JB) * ATOM;
    L.off_u = L.y_bytes;
    // Ddot in place over 16-bit counts; not where the persistent cluster epoch
    // may run, which loads the next block's counts while the contractions still
    // read Ddot
    {
        const int64_t ti = (std::min<int64_t>(h->cfg.nb_row, h->n) + TT - 1) / TT;
        const int64_t tj = (std::min<int64_t>(h->cfg.nb_col, h->m) + TT - 1) / TT;
        const bool cl_epoch = (h->cfg.flags & GMF_FLAG_PERSIST) && !(h->cfg.flags & GMF_FLAG_NO_CLUSTER) && ti * tj <= 16;
        L.dd_in_y = (h->y16 && !cl_epoch) ? 1 : 0;
    }
    L.off_dd = L.dd_in_y ? 0u : L.off_u;
    L.off_ddd = L.dd_in_y ? L.off_u : L.off_u + 2u * ATOM;
    const uint32_t size_u = std::max<uint32_t>(2u * L.KA * ATOM, (L.dd_in_y ? 2u : 4u) * ATOM);
    L.off_rf = L.off_u + size_u;
    L.off_rf2 = L.off_rf + (uint32_t)L.NR * 256u;
    L.off_lf = L.off_rf2 + (uint32_t)L.NR * 256u;
    L.off_lf2 = L.off_lf + (uint32_t)L.NC * 256u;
    L.smem = L.off_lf2 + (uint32_t)L.NC * 256u + 1024u;
    L.t_row = TT;
    L.t_col = TT + 2u * L.NR;
    const uint32_t need = L.t_col + 2u * L.NC;
    L.tmem_cols = need <= 256 ? 256 : 512;
    {
        int optin = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa;
        const cudaError_t fe = cudaFuncGetAttributes(&fa, tc_fn(h->y16, 0, EPI_ANY));
        if (fe != cudaSuccess || (size_t)L.smem + fa.sharedSizeBytes > (size_t)optin) {
            delete tc;
            return fail_str(err, "mixed precision: the tile does not fit in shared memory (reduce d or use uint16 counts)");
        }
    }
    if (tc_encode_y(h, &tc->ymap[0], h->Yp) != GMF_OK) {
        delete tc;
        if (err) *err = "cuTensorMapEncodeTiled failed for the count matrix";
        return GMF_ERR_CUDA;
    }
    tc->epi = (h->Wp || h->cfg.missing || h->cfg.alpha_mode == 2 || h->cfg.family > GMF_NEGBIN) ? EPI_ANY
              : h->cfg.family == GMF_NEGBIN ? (h->cfg.alpha_mode == 1 ? EPI_ANY : EPI_NB)
                                            : EPI_PO;
    cudaError_t e = gmf_smem_limit(tc_fn(h->y16, 0, tc->epi), L.smem);
    // all of the unified L1 / shared array as shared memory: room for two tiles per SM
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_fn(h->y16, 0, tc->epi), cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) {
        delete tc;
        if (err) *err = cudaGetErrorString(e);
        return GMF_ERR_CUDA;
    }
    tc->TI = (int)((std::min<int64_t>(h->cfg.nb_row, h->n) + TT - 1) / TT);
    tc->TJ = (int)((std::min<int64_t>(h->cfg.nb_col, h->m) + TT - 1) / TT);
    tc->cluster = 0;
    tc->persist = 0;
    if (!(h->cfg.flags & GMF_FLAG_NO_CLUSTER) && tc->TI * tc->TJ <= 16) tc->cluster = tc_cluster_layout(h, tc);
    if (tc->cluster && (h->cfg.flags & GMF_FLAG_PERSIST)) tc->persist = tc_persist_check(h, tc);
    if (!tc->cluster && (h->cfg.flags & GMF_FLAG_PERSIST)) {
        const int rc = tc_flow_setup(h, tc);
        if (rc != GMF_OK) {
            gmf_tc_release(tc);
            if (err) *err = "device allocation for the dataflow epoch failed";
            return rc;
        }
    }
    gmf_tc_deviance_setup(h, tc);
    h->tc = tc;
    return GMF_OK;
}

namespace {

// Shared-memory and cluster-size attributes of a cluster kernel, and whether
// all clusters of one sweep can be resident at once.
int cluster_fits(gmf_model* h, TcState* tc, const void* fn, uint32_t smem) {
    const int TI = tc->TI, TJ = tc->TJ;
    if (gmf_smem_limit(fn, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (TI * TJ > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(TJ, TI, h->per);
    cfg.blockDim = dim3(NTH);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = TJ;
    at[0].val.clusterDim.y = TI;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nclusters >= h->per ? 1 : 0;
}

// Cluster mode needs the partials and the update slices in shared memory next
// to the tile, cluster dimensions (TJ, TI) within the device's limit, and room
// for all clusters of a sweep at once (else the sweep would run in waves).
int tc_cluster_layout(gmf_model* h, TcState* tc) {
    TcLayout& L = tc->lay;
    const int TI = tc->TI, TJ = tc->TJ;
    L.SRr = (TT + TJ - 1) / TJ;
    L.SCc = (TT + TI - 1) / TI;
    L.off_cp = (L.off_lf2 + (uint32_t)L.NC * 256u + 15u) & ~15u;
    L.off_st = L.off_cp + 4u * (uint32_t)(TJ * 2 * h->fr * L.SRr + TI * 2 * h->fc * L.SCc);
    const uint32_t st_bytes = 4u * (uint32_t)(L.SRr * (h->KP + 1 + 2 * (h->fr | 1) + 1) +
                                              L.SCc * (h->KP + 1 + 2 * (h->fc | 1) + 1));
    L.smem_cl = L.off_st + st_bytes + 1024u;
    return cluster_fits(h, tc, tc_fn(h->y16, 1, tc->epi), L.smem_cl);
}

// The persistent epoch needs every cluster of a sweep resident at once (the
// same occupancy test) and a fixed NB shape: the per-sweep shape estimate of
// alpha_mode 1 pools all clusters of a sweep, which this launch never joins.
// The dataflow epoch's grid: as many CTAs as fit on the device at once by
// registers, shared memory, threads and TMEM (each CTA holds its tile's TMEM
// for the whole launch), computed from the kernel's attributes (the launch
// needs no co-residency, so an estimate that is too high only queues CTAs).
// Returns GMF_OK with tc->flow = 0 where it cannot run (the per-sweep launches
// stay), an error only when an allocation fails.
int tc_flow_setup(gmf_model* h, TcState* tc) {
    const void* fn = tc_flow_fn(h->y16, tc->epi);
    int dev = 0, sms = 0, smem_sm = 0, regs_sm = 0, thr_sm = 0, resv = 0;
    cudaFuncAttributes fa;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        gmf_smem_limit(fn, tc->lay.smem) != cudaSuccess ||
        cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared) !=
            cudaSuccess ||
        cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
        cudaGetLastError();
        return GMF_OK;
    }
    const int regs_cta = ((fa.numRegs * 32 + 255) / 256) * 256 * (NTH / 32);  // allocated per warp, 256 at a time
    const size_t smem_cta = (size_t)tc->lay.smem + fa.sharedSizeBytes + (size_t)resv;
    int per_sm = std::min({regs_sm / std::max(regs_cta, 1), (int)((size_t)smem_sm / smem_cta), thr_sm / NTH,
                           (int)(512u / tc->lay.tmem_cols)});
    if (per_sm < 1) return GMF_OK;
    const size_t groups = (size_t)2 * h->nsw * h->per;
    const size_t nctr = 3 + 2 * (size_t)h->per + (size_t)std::max(h->r, h->s);
    if (cudaMalloc(&tc->fent, sizeof(int4) * groups) != cudaSuccess ||
        cudaMalloc(&tc->fstart, sizeof(int) * (groups + 1)) != cudaSuccess ||
        cudaMalloc(&tc->fctr, sizeof(unsigned) * nctr) != cudaSuccess) {
        cudaGetLastError();
        return GMF_ERR_OOM;
    }
    tc->flow_grid = per_sm * sms;
    tc->flow = 1;
    return GMF_OK;
}

void gmf_tc_release(TcState* tc) {
    if (tc->fent) cudaFree(tc->fent);
    if (tc->fstart) cudaFree(tc->fstart);
    if (tc->fctr) cudaFree(tc->fctr);
    delete tc;
}

int tc_persist_check(gmf_model* h, TcState* tc) {
    if (scalar_estimated(h->cfg.family, h->cfg.alpha_mode)) return 0;
    if (tc->lay.dd_in_y) return 0;  // the next block's count tile would overwrite Ddot
    return cluster_fits(h, tc, tc_epoch_fn(h->y16, tc->epi), tc->lay.smem_cl);
}

}  // namespace

cudaError_t gmf_tc_launch(gmf_model* h, const StepArgs& base, int w, cudaStream_t st) {
    TcState* tc = (TcState*)h->tc;
    StepArgs a = base;
    a.TI = tc->TI;
    a.TJ = tc->TJ;
    dim3 grid(tc->TJ, tc->TI, a.nk);
    if (tc->cluster) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = dim3(NTH);
        cfg.dynamicSmemBytes = tc->lay.smem_cl;
        cfg.stream = st;
        cudaLaunchAttribute at[2];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = tc->TJ;
        at[0].val.clusterDim.y = tc->TI;
        at[0].val.clusterDim.z = 1;
        at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 2;
        void* args[] = {&a, (void*)&tc->lay, (void*)&tc->ymap[h->ycur], &w};
        return cudaLaunchKernelExC(&cfg, tc_fn(h->y16, 1, tc->epi), args);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(NTH);
    cfg.dynamicSmemBytes = tc->lay.smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    void* args[] = {&a, (void*)&tc->lay, (void*)&tc->ymap[h->ycur], &w};
    return cudaLaunchKernelExC(&cfg, tc_fn(h->y16, 0, tc->epi), args);
}

cudaError_t gmf_tc_launch_update(gmf_model* h, const StepArgs& base, int w, cudaStream_t st) {
    const TcState* tc = (const TcState*)h->tc;
    if (tc->cluster) return cudaSuccess;  // the tile launch did the updates
    StepArgs a = base;
    a.TI = tc->TI;
    a.TJ = tc->TJ;
    return gmf_launch_update_tc(a, w, TT, st);
}

// The sweeps [w0, w1) as one persistent launch (sweep_tc_epoch): the strip
// completion counts start from zero.
static cudaError_t tc_launch_flow(gmf_model* h, int w0, int w1, cudaStream_t st);

cudaError_t gmf_tc_launch_epoch(gmf_model* h, int w0, int w1, cudaStream_t st) {
    TcState* tc = (TcState*)h->tc;
    if (tc->flow) return tc_launch_flow(h, w0, w1, st);
    cudaError_t e = cudaMemsetAsync(h->strip_done, 0, sizeof(unsigned) * (size_t)std::max(h->r, h->s), st);
    if (e != cudaSuccess) return e;
    StepArgs a = gmf_make_args(h);
    a.TI = tc->TI;
    a.TJ = tc->TJ;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(tc->TJ, tc->TI, h->per);
    cfg.blockDim = dim3(NTH);
    cfg.dynamicSmemBytes = tc->lay.smem_cl;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = tc->TJ;
    at[0].val.clusterDim.y = tc->TI;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    void* args[] = {&a, (void*)&tc->lay, (void*)&tc->ymap[h->ycur], &w0, &w1};
    return cudaLaunchKernelExC(&cfg, tc_epoch_fn(h->y16, tc->epi), args);
}

int gmf_tc_persistent(const gmf_model* h) {
    return h->tc && (((const TcState*)h->tc)->persist || ((const TcState*)h->tc)->flow);
}
int gmf_tc_flow(const gmf_model* h) { return h->tc && ((const TcState*)h->tc)->flow; }

// The group order of the dataflow launch over sweeps [w0, w1) (see
// sweep_tc_flow): T(p) in block order; U(p) once `lag` later tile groups are
// out, or earlier where a tile group reads what U(p) writes. Each entry holds
// the counts its items wait for. Staged with the epoch's schedule.
int gmf_tc_stage_flow(gmf_model* h, const int32_t* sigma, int w0, int w1, cudaStream_t st) {
    TcState* tc = (TcState*)h->tc;
    const int per = h->per, swap = h->swap, mod = swap ? h->s : h->r;
    const int P = (w1 - w0) * per;
    const int tij = tc->TI * tc->TJ, nsl = TT / UTC_SR, ub = (tc->TI + tc->TJ) * nsl;
    const int mu = (swap ? tc->TJ : tc->TI) * nsl;  // moving-side units of a block
    const int lag = std::max(0, h->flow_lag);
    std::vector<int4> ent;
    std::vector<int> start;
    ent.reserve((size_t)2 * P);
    start.reserve((size_t)2 * P + 1);
    std::vector<int> last((size_t)mod, -1), visits((size_t)mod, 0);
    std::deque<int> pending;  // tile groups whose update group is not out yet, in order
    int ticket = 0;
    auto strip = [&](int p) { return (sigma[w0 + p / per] + p % per) % mod; };
    auto updates_through = [&](int q) {
        while (!pending.empty() && pending.front() <= q) {
            const int u = pending.front();
            pending.pop_front();
            start.push_back(ticket);
            ent.push_back(make_int4(2 * u + 1, (u / per + 1) * tij, strip(u), 0));
            ticket += ub;
        }
    };
    for (int p = 0; p < P; p++) {
        const int wr = p / per;
        const int j = strip(p);
        if (wr > 0) updates_through(p - per);
        if (last[(size_t)j] >= 0) updates_through(last[(size_t)j]);
        const int nd = visits[(size_t)j] + h->need_extra;  // earlier visits of the moving strip in this launch
        start.push_back(ticket);
        ent.push_back(make_int4(2 * p, wr * ub, j, nd * mu));
        ticket += tij;
        pending.push_back(p);
        last[(size_t)j] = p;
        visits[(size_t)j]++;
        while ((int)pending.size() > lag) updates_through(pending.front());
    }
    updates_through(P);
    start.push_back(ticket);
    tc->flow_groups = (int)ent.size();
    if (ent.empty()) return GMF_OK;
    if (cudaMemcpyAsync(tc->fent, ent.data(), sizeof(int4) * ent.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(tc->fstart, start.data(), sizeof(int) * start.size(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
        return GMF_ERR_CUDA;
    return GMF_OK;
}

static cudaError_t tc_launch_flow(gmf_model* h, int w0, int w1, cudaStream_t st) {
    TcState* tc = (TcState*)h->tc;
    const size_t nctr = 3 + 2 * (size_t)h->per + (size_t)std::max(h->r, h->s);
    cudaError_t e = cudaMemsetAsync(tc->fctr, 0, sizeof(unsigned) * nctr, st);
    if (e != cudaSuccess) return e;
    StepArgs a = gmf_make_args(h);
    a.TI = tc->TI;
    a.TJ = tc->TJ;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(tc->flow_grid);
    cfg.blockDim = dim3(NTH);
    cfg.dynamicSmemBytes = tc->lay.smem;
    cfg.stream = st;
    uint32_t cols = tc->lay.tmem_cols;
    int ng = tc->flow_groups;
    void* args[] = {&a, (void*)&tc->lay, (void*)&tc->ymap[h->ycur], &w0, (void*)&tc->fent, (void*)&tc->fstart, &ng,
                    (void*)&tc->fctr, &cols};
    (void)w1;
    return cudaLaunchKernelExC(&cfg, tc_flow_fn(h->y16, tc->epi), args);
}

size_t gmf_tc_layout_size() { return sizeof(TcLayout); }
const void* gmf_tc_layout(const gmf_model* h) { return &((const TcState*)h->tc)->lay; }
uint32_t gmf_tc_smem(const gmf_model* h) { return ((const TcState*)h->tc)->lay.smem; }
uint32_t gmf_tc_tmem_cols(const gmf_model* h) { return ((const TcState*)h->tc)->lay.tmem_cols; }
void gmf_tc_grid(const gmf_model* h, int* TI, int* TJ) {
    *TI = ((const TcState*)h->tc)->TI;
    *TJ = ((const TcState*)h->tc)->TJ;
}

cudaError_t gmf_tc_multi_attr(const gmf_model* h0, uint32_t smem) {
    const void* fn = tc_multi_fn(h0->y16, ((const TcState*)h0->tc)->epi);
    cudaError_t e = gmf_smem_limit(fn, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    return e;
}

// One sweep of nmodels models: grid (TJ, TI, nmodels * per), with programmatic
// stream serialization like the single-model tile launch.
cudaError_t gmf_tc_launch_multi(const gmf_model* h0, const StepArgs* d_args, const void* d_lays, const int* d_order,
                                int nmodels, uint32_t smem, int w, cudaStream_t st) {
    const TcState* tc = (const TcState*)h0->tc;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(tc->TJ, tc->TI, h0->per * nmodels);
    cfg.blockDim = dim3(NTH);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const TcLayout* lays = (const TcLayout*)d_lays;
    int per = h0->per;
    void* args[] = {(void*)&d_args, (void*)&lays, (void*)&d_order, &per, (void*)&tc->ymap[h0->ycur], &w};
    return cudaLaunchKernelExC(&cfg, tc_multi_fn(h0->y16, tc->epi), args);
}

// One sweep of nmodels models as one cooperative persistent launch: as many CTAs
// as can be resident at once (at most one per tile); returns the grid size in *grid.
cudaError_t gmf_tc_launch_multi_persist(const gmf_model* h0, const StepArgs* d_args, const void* d_lays,
                                        const int* d_order, int nmodels, uint32_t smem, uint32_t tmem_cols, int w,
                                        unsigned* gctr, unsigned* err, cudaStream_t st) {
    const TcState* tc = (const TcState*)h0->tc;
    const void* fn = tc_persist_fn(h0->y16, tc->epi);
    cudaError_t e = gmf_smem_limit(fn, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NTH, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    if (tmem_cols < 32 || tmem_cols > 512) return cudaErrorInvalidValue;
    per_sm = std::min(per_sm, (int)(512u / tmem_cols));  // every resident CTA holds its TMEM for the tile phase
    const int tiles = h0->per * tc->TI * tc->TJ * nmodels;
    const int grid = std::max(1, std::min(per_sm * sms, tiles));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(NTH);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const TcLayout* lays = (const TcLayout*)d_lays;
    int per = h0->per;
    unsigned long long wait_ns = h0->wait_ns > 0 ? (unsigned long long)h0->wait_ns : 2000000000ull;
    void* args[] = {(void*)&d_args, (void*)&lays, (void*)&d_order, &nmodels, &per, (void*)&tc->ymap[h0->ycur], &w,
                    &gctr, &wait_ns, &err, &tmem_cols};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

int gmf_tc_cluster(const gmf_model* h) { return h->tc && ((const TcState*)h->tc)->cluster; }

void gmf_tc_free(gmf_model* h) {
    if (h->tc) gmf_tc_release((TcState*)h->tc);
    h->tc = nullptr;
}
