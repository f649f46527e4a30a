// Tensor-core (tcgen05, sm_103a) path of the block step: Algorithm 1's per-block
// work (eq. 15 with App. B) with eta and the four gradient / curvature
// contractions on the 5th-generation tensor cores.
//
// One CTA per 128 x 128 tile, 16 warps:
//   1. thread 0 starts the TMA load of the tile's counts (128-byte swizzled
//      boxes) while all threads build the MMA operands in shared memory:
//        eta:  A = [L_hi | L_lo | L_hi], B = [R_hi | R_hi | R_lo] (BF16 split of
//              the FP32 factors, K-concatenated), so one accumulation gives
//              L_hi R_hi' + L_lo R_hi' + L_hi R_lo' (split-BF16, 3 products);
//        row side:    B = [Z, V]' and its square, K = tile columns;
//        column side: B = [X, U]' and its square, K = tile rows;
//   2. thread 0 issues the eta MMAs (FP32 accumulate in TMEM) and commits;
//   3. the 16 warps read eta from TMEM (warp w: lanes 32(w%4).., columns
//      32(w/4)..), compute mu = exp(eta), Ddot, Dddot (Sec. 3) in FP32 and
//      store them as BF16 into one swizzled tile (over the dead eta operands);
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

#include <string>

#include "gmf_internal.cuh"
#include "gmf_sm100.cuh"
#include "gmf_update.cuh"

namespace {

using namespace gmfdev;
using namespace sm100;

constexpr int TT = 128;            // tile edge (rows and columns)
constexpr int NTH = 512;           // threads per CTA (16 warps)
constexpr uint32_t ATOM = 16384;   // 128 rows x 128 bytes, 128-byte swizzle
constexpr uint32_t WAIT_POLLS = 1u << 26;

struct TcLayout {
    int KP16;              // K rounded up to 16
    int KA;                // 128-byte atoms per eta operand row (3*KP16 bf16)
    int NR, NC;            // contraction widths (q+d, p+d rounded up to 16)
    int JB;                // count columns per TMA box (128 bytes)
    uint32_t y_bytes;      // bytes of the count tile
    uint32_t off_u;        // union: eta operands, then the Ddot / Dddot tile
    uint32_t off_rf, off_rf2, off_lf, off_lf2;
    uint32_t smem;         // dynamic shared memory including alignment slack
    uint32_t tmem_cols, t_row, t_col;
};

struct TcState {
    TcLayout lay;
    CUtensorMap ymap;
    int TI, TJ;
};

__device__ __forceinline__ void st_shared_v4(void* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(smem_u32(p)), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

__device__ __forceinline__ uint32_t bf16_bits(float x) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// Bounded wait shared by the CTA: returns true when every thread saw the phase.
__device__ __forceinline__ bool cta_wait(uint64_t* bar, uint32_t parity, unsigned* err) {
    bool ok = mbar_wait(bar, parity, WAIT_POLLS);
    if (!ok) {
        atomicOr(err, GMF_DEVERR_TIMEOUT);
        ok = mbar_wait(bar, parity, WAIT_POLLS);  // drain this CTA's own copies / MMAs
    }
    return __syncthreads_and(ok) != 0;
}

// One tile (blockIdx.x, blockIdx.y) of block k of sweep w for the model whose
// arguments are a / Lo.
template <bool Y16>
__device__ __forceinline__ void tc_tile(const StepArgs& a, const TcLayout& Lo, const CUtensorMap* ymap_p, int w,
                                        int k, uint8_t* smraw) {
    __shared__ uint64_t bars[3];
    __shared__ uint32_t tmem_base;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tj = blockIdx.x, ti = blockIdx.y;
    const BlockGeo g = block_geo(a, w, k);
    const int nTI = (int)((g.nI + TT - 1) / TT), nTJ = (int)((g.mJ + TT - 1) / TT);
    const bool active = ti < nTI && tj < nTJ;
    const bool nb = a.family == GMF_NEGBIN;
    const bool moments = nb && a.alpha_mode == 1;
    float alpha = 0.f;
    float s1 = 0.f, s2 = 0.f;

    uint8_t* sm = smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u);
    if (active) {
        uint8_t* Ys = sm;
        uint8_t* Aop = sm + Lo.off_u;
        uint8_t* Bop = Aop + Lo.KA * ATOM;
        uint8_t* Dd = sm + Lo.off_u;   // overlays the eta operands once the eta MMA has completed
        uint8_t* DDd = Dd + 2 * ATOM;
        uint8_t* RF = sm + Lo.off_rf;
        uint8_t* RF2 = sm + Lo.off_rf2;
        uint8_t* LF = sm + Lo.off_lf;
        uint8_t* LF2 = sm + Lo.off_lf2;
        const int64_t row0 = g.r0 + (int64_t)ti * TT, col0 = g.c0 + (int64_t)tj * TT;
        const int nr = (int)min((int64_t)TT, g.nI - (int64_t)ti * TT);
        const int nc = (int)min((int64_t)TT, g.mJ - (int64_t)tj * TT);

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

        if (tid == 0) {
            mbar_arrive_expect_tx(&bars[0], Lo.y_bytes);
            const int nbox = TT / Lo.JB;
            for (int b = 0; b < nbox; b++)
                tma_load_2d(Ys + b * ATOM, ymap_p, (int)(col0 + (int64_t)b * Lo.JB), (int)row0, &bars[0]);
        }
        // the counts are read-only; everything below reads or writes model state
        // that the previous sweep's update launch may still be writing. The
        // next launch (this sweep's update) may start once every CTA is here,
        // i.e. once the previous update has completed.
        grid_dependency_wait();
        grid_launch_dependents();
        alpha = *a.alpha;

        // ---- operands. Thread groups of 128: L rows -> eta A; R rows -> eta B;
        //      L rows -> column-side B ([X, U] and squares); R rows -> row-side B ([Z, V] and squares).
        {
            const int grp = tid >> 7, r = tid & (TT - 1);
            const bool isL = (grp & 1) == 0;
            const bool ok = isL ? r < nr : r < nc;
            const float* src = isL ? a.L + (row0 + r) * a.KP : a.R + (col0 + r) * a.KP;
            if (grp < 2) {
                uint8_t* op = isL ? Aop : Bop;
                for (int kb = 0; kb < Lo.KP16; kb += 32) {
                    float v[32];
#pragma unroll
                    for (int u = 0; u < 8; u++) {
                        const int kk = kb + 4 * u;
                        const float4 x = (ok && kk < a.KP) ? __ldg((const float4*)(src + kk))
                                                           : make_float4(0.f, 0.f, 0.f, 0.f);
                        v[4 * u] = x.x;
                        v[4 * u + 1] = x.y;
                        v[4 * u + 2] = x.z;
                        v[4 * u + 3] = x.w;
                    }
#pragma unroll
                    for (int h8 = 0; h8 < 4; h8++) {
                        const int kk0 = kb + 8 * h8;
                        if (kk0 < Lo.KP16) {
                            uint32_t hi[4], lo[4];
#pragma unroll
                            for (int t = 0; t < 4; t++) {
                                const float x0 = v[8 * h8 + 2 * t], x1 = v[8 * h8 + 2 * t + 1];
                                hi[t] = pack_bf16x2(x0, x1);
                                const float r0 = x0 - __uint_as_float(hi[t] << 16);
                                const float r1 = x1 - __uint_as_float(hi[t] & 0xFFFF0000u);
                                lo[t] = pack_bf16x2(r0, r1);
                            }
#pragma unroll
                            for (int seg = 0; seg < 3; seg++) {
                                // A segments: hi, lo, hi;  B segments: hi, hi, lo
                                const bool use_lo = isL ? seg == 1 : seg == 2;
                                const int kc = seg * Lo.KP16 + kk0;
                                uint8_t* dst = op + (kc >> 6) * ATOM + sw128_off(r, (kc & 63) * 2);
                                if (use_lo)
                                    st_shared_v4(dst, lo[0], lo[1], lo[2], lo[3]);
                                else
                                    st_shared_v4(dst, hi[0], hi[1], hi[2], hi[3]);
                            }
                        }
                    }
                }
            } else {
                // value and square of each multiplier column; K index of the contraction = r
                const int NF = isL ? Lo.NC : Lo.NR;
                const int nf = isL ? a.fc : a.fr;
                uint8_t* o1 = isL ? LF : RF;
                uint8_t* o2 = isL ? LF2 : RF2;
                const uint32_t atom = (uint32_t)NF * 128u;
                for (int c0 = 0; c0 < NF; c0 += 16) {
                    float v[16];
#pragma unroll
                    for (int u = 0; u < 16; u++) {
                        const int c = c0 + u;
                        const int col = isL ? (c < a.p ? 1 + c : 1 + a.q + c) : 1 + a.p + c;
                        v[u] = (ok && c < nf) ? __ldg(src + col) : 0.f;
                    }
#pragma unroll
                    for (int u = 0; u < 16; u++) {
                        const uint32_t off = (r >> 6) * atom + sw128_off(c0 + u, (r & 63) * 2);
                        *(__nv_bfloat16*)(o1 + off) = __float2bfloat16_rn(v[u]);
                        *(__nv_bfloat16*)(o2 + off) = __float2bfloat16_rn(v[u] * v[u]);
                    }
                }
            }
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();

        if (tid == 0) {
            const uint32_t id = idesc_bf16(TT, TT, 0, 0);
            const int nks = 3 * Lo.KP16 / 16;
            for (int ks = 0; ks < nks; ks++) {
                const uint32_t off = (uint32_t)(ks >> 2) * ATOM + (uint32_t)(ks & 3) * 32u;
                umma_bf16(tb, sdesc(smem_u32(Aop) + off, 16, 1024, SWIZZLE_128B),
                          sdesc(smem_u32(Bop) + off, 16, 1024, SWIZZLE_128B), id, ks > 0);
            }
            umma_commit(&bars[1]);
        }
        bool ok = cta_wait(&bars[0], 0, a.err);
        ok = cta_wait(&bars[1], 0, a.err) && ok;
        tc_fence_after();

        if (ok) {
            // ---- epilogue: warp (q, cq) owns rows 32q.. and columns 32cq..32cq+31
            const int q = warp & 3, cq = warp >> 2;
            const int i = 32 * q + lane;
            const bool row_ok = i < nr;
            const float* Wrow = a.W ? a.W + (row0 + i) * a.m + col0 : nullptr;
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
                    y[0] = (float)u0.x; y[1] = (float)u0.y; y[2] = (float)u0.z; y[3] = (float)u0.w;
                    y[4] = (float)u1.x; y[5] = (float)u1.y; y[6] = (float)u1.z; y[7] = (float)u1.w;
                }
                float dd[8], ddd[8];
#pragma unroll
                for (int t = 0; t < 8; t++) {
                    const int j = j0 + t;
                    const bool valid = row_ok && j < nc;
                    const float wv = (Wrow && valid) ? __ldg(Wrow + j) : 1.f;
                    const float e = fminf(fmaxf(__uint_as_float(ev[8 * gq + t]), -a.clamp), a.clamp);
                    const float mu = __expf(e);
                    const float f = nb ? __fdividef(alpha, alpha + mu) : 1.f;
                    const float wf = valid ? wv * f : 0.f;
                    dd[t] = wf * (y[t] - mu);
                    ddd[t] = wf * mu;
                    if (moments && valid) {
                        s1 = fmaf(wv * mu, mu, s1);
                        s2 += wv * ((y[t] - mu) * (y[t] - mu) - mu);
                    }
                }
                const uint32_t off = (uint32_t)(j0 >> 6) * ATOM + sw128_off(i, (j0 & 63) * 2);
                st_shared_v4(Dd + off, pack_bf16x2(dd[0], dd[1]), pack_bf16x2(dd[2], dd[3]),
                             pack_bf16x2(dd[4], dd[5]), pack_bf16x2(dd[6], dd[7]));
                st_shared_v4(DDd + off, pack_bf16x2(ddd[0], ddd[1]), pack_bf16x2(ddd[2], ddd[3]),
                             pack_bf16x2(ddd[4], ddd[5]), pack_bf16x2(ddd[6], ddd[7]));
            }
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();

        if (ok && tid == 0) {
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
            umma_commit(&bars[2]);
        }
        if (ok) ok = cta_wait(&bars[2], 0, a.err);
        tc_fence_after();

        if (ok && warp < 8) {
            const int q = warp & 3;
            const uint32_t lanes = (uint32_t)(32 * q) << 16;
            const int o = 32 * q + lane;   // tile row (warps 0-3) or tile column (warps 4-7)
            const bool rowside = warp < 4;
            const int NF = rowside ? Lo.NR : Lo.NC;
            const int nf = rowside ? a.fr : a.fc;
            const uint32_t tg = tb + lanes + (rowside ? Lo.t_row : Lo.t_col);
            float* dst = rowside ? a.partR + (size_t)((k * a.TI + ti) * a.TJ + tj) * TT * 2 * a.fr
                                 : a.partC + (size_t)((k * a.TJ + tj) * a.TI + ti) * TT * 2 * a.fc;
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
                            dst[(size_t)c * TT + o] = __uint_as_float(rg[u]);
                            dst[(size_t)(nf + c) * TT + o] = __uint_as_float(rh[u]);
                        }
                    }
                }
            }
        }
        if (!ok && tid == 0) atomicOr(a.err, GMF_DEVERR_TIMEOUT);
        tc_fence_before();
        __syncthreads();
        if (warp == 0) tmem_dealloc(tb, Lo.tmem_cols);
    } else {
        grid_dependency_wait();  // before writing this sweep's moment slot
        grid_launch_dependents();
    }
    tile_moments<NTH>(a, k, ti, tj, s1, s2);
}

template <bool Y16>
__global__ void __launch_bounds__(NTH, 1)
    sweep_tc_kernel(StepArgs a, TcLayout Lo, const __grid_constant__ CUtensorMap ymap, int w) {
    extern __shared__ __align__(1024) uint8_t smraw[];
    tc_tile<Y16>(a, Lo, &ymap, w, blockIdx.z, smraw);
}

// Several models (ranks) sharing the count matrix and the partitions: blockIdx.z
// = slot * per + k, slot -> model through `order` (heaviest models first).
template <bool Y16>
__global__ void __launch_bounds__(NTH, 1) sweep_tc_multi(const StepArgs* __restrict__ av, const TcLayout* __restrict__ lv,
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
    tc_tile<Y16>(s_a, s_l, &ymap, w, blockIdx.z % per, smraw);
}

int fail_str(std::string* err, const char* msg) {
    if (err) *err = msg;
    return GMF_ERR_ARG;
}

}  // namespace

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
    L.KA = (3 * L.KP16 + 63) / 64;
    L.NR = (std::max(h->fr, 1) + 15) & ~15;
    L.NC = (std::max(h->fc, 1) + 15) & ~15;
    L.JB = 128 / es;
    L.y_bytes = (uint32_t)(TT / L.JB) * ATOM;
    L.off_u = L.y_bytes;
    const uint32_t size_u = std::max<uint32_t>(2u * L.KA * ATOM, 4u * ATOM);
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
        const cudaError_t fe = h->y16 ? cudaFuncGetAttributes(&fa, sweep_tc_kernel<true>)
                                      : cudaFuncGetAttributes(&fa, sweep_tc_kernel<false>);
        if (fe != cudaSuccess || (size_t)L.smem + fa.sharedSizeBytes > (size_t)optin) {
            delete tc;
            return fail_str(err, "mixed precision: the tile does not fit in shared memory (reduce d or use uint16 counts)");
        }
    }
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr) != cudaSuccess ||
        !fn) {
        delete tc;
        if (err) *err = "cuTensorMapEncodeTiled is not available";
        return GMF_ERR_CUDA;
    }
    cuuint64_t dims[2] = {(cuuint64_t)h->m, (cuuint64_t)h->n};
    cuuint64_t strides[1] = {(cuuint64_t)h->m * es};
    cuuint32_t box[2] = {(cuuint32_t)L.JB, (cuuint32_t)TT};
    cuuint32_t estr[2] = {1, 1};
    CUresult cr = ((PFN_cuTensorMapEncodeTiled_v12000)fn)(
        &tc->ymap, h->y16 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_INT32, 2, h->Yp, dims, strides,
        box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) {
        delete tc;
        if (err) *err = "cuTensorMapEncodeTiled failed for the count matrix";
        return GMF_ERR_CUDA;
    }
    cudaError_t e = h->y16 ? cudaFuncSetAttribute(sweep_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)L.smem)
                           : cudaFuncSetAttribute(sweep_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)L.smem);
    if (e != cudaSuccess) {
        delete tc;
        if (err) *err = cudaGetErrorString(e);
        return GMF_ERR_CUDA;
    }
    tc->TI = (int)((std::min<int64_t>(h->cfg.nb_row, h->n) + TT - 1) / TT);
    tc->TJ = (int)((std::min<int64_t>(h->cfg.nb_col, h->m) + TT - 1) / TT);
    h->tc = tc;
    return GMF_OK;
}

cudaError_t gmf_tc_launch(gmf_model* h, int w, cudaStream_t st) {
    TcState* tc = (TcState*)h->tc;
    StepArgs a = gmf_make_args(h);
    a.TI = tc->TI;
    a.TJ = tc->TJ;
    dim3 grid(tc->TJ, tc->TI, h->per);
    const cudaError_t e =
        h->y16 ? gmf_launch_pdl(sweep_tc_kernel<true>, grid, dim3(NTH), tc->lay.smem, st, a, tc->lay, tc->ymap, w)
               : gmf_launch_pdl(sweep_tc_kernel<false>, grid, dim3(NTH), tc->lay.smem, st, a, tc->lay, tc->ymap, w);
    return e;
}

cudaError_t gmf_tc_launch_update(gmf_model* h, int w, cudaStream_t st) {
    const TcState* tc = (const TcState*)h->tc;
    StepArgs a = gmf_make_args(h);
    a.TI = tc->TI;
    a.TJ = tc->TJ;
    return gmf_launch_update(a, w, TT, st);
}

size_t gmf_tc_layout_size() { return sizeof(TcLayout); }
const void* gmf_tc_layout(const gmf_model* h) { return &((const TcState*)h->tc)->lay; }
uint32_t gmf_tc_smem(const gmf_model* h) { return ((const TcState*)h->tc)->lay.smem; }
void gmf_tc_grid(const gmf_model* h, int* TI, int* TJ) {
    *TI = ((const TcState*)h->tc)->TI;
    *TJ = ((const TcState*)h->tc)->TJ;
}

cudaError_t gmf_tc_multi_attr(int y16, uint32_t smem) {
    return y16 ? cudaFuncSetAttribute(sweep_tc_multi<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
               : cudaFuncSetAttribute(sweep_tc_multi<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// One sweep of nmodels models: grid (TJ, TI, nmodels * per).
cudaError_t gmf_tc_launch_multi(const gmf_model* h0, const StepArgs* d_args, const void* d_lays, const int* d_order,
                                int nmodels, uint32_t smem, int w, cudaStream_t st) {
    const TcState* tc = (const TcState*)h0->tc;
    dim3 grid(tc->TJ, tc->TI, h0->per * nmodels);
    const TcLayout* lays = (const TcLayout*)d_lays;
    return h0->y16 ? gmf_launch_pdl(sweep_tc_multi<true>, grid, dim3(NTH), smem, st, d_args, lays, d_order, h0->per,
                                    tc->ymap, w)
                   : gmf_launch_pdl(sweep_tc_multi<false>, grid, dim3(NTH), smem, st, d_args, lays, d_order, h0->per,
                                    tc->ymap, w);
}

void gmf_tc_free(gmf_model* h) {
    delete (TcState*)h->tc;
    h->tc = nullptr;
}
