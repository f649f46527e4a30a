// Tile pieces shared by the tensor-core kernels (tcgen05, sm_103a): the
// layout of a 128 x 128 tile in shared memory, the handle's tensor-core state,
// the bounded CTA-wide mbarrier wait, the TMA load of a count tile, the
// split-BF16 eta operands (Algorithm 1's linear predictor, eq. 3) and the
// eta MMAs. The block step (gmf_step_tc.cu) and the full deviance
// (gmf_deviance_tc.cu) build on them.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "gmf_internal.cuh"
#include "gmf_sm100.cuh"
#include "gmf_update.cuh"

namespace gmftc {

using namespace gmfdev;
using namespace sm100;

constexpr int TT = 128;            // tile edge (rows and columns)
constexpr int NTH = 512;           // threads per CTA (16 warps)
constexpr uint32_t ATOM = 16384;   // 128 rows x 128 bytes, 128-byte swizzle
constexpr uint32_t WAIT_POLLS = 1u << 26;

struct TcLayout {
    int KP16;              // K rounded up to 16
    int KA;                // 128-byte atoms per eta operand row ([hi | lo]: 2*KP16 bf16)
    int NR, NC;            // contraction widths (q+d, p+d rounded up to 16)
    int JB;                // count columns per TMA box (128 bytes)
    uint32_t y_bytes;      // bytes of the count tile
    uint32_t off_u;        // union: eta operands, then the Dddot tile (and Ddot unless it is in the count tile)
    uint32_t off_dd, off_ddd;  // Ddot and Dddot tiles (2 atoms each)
    int dd_in_y;           // 1: Ddot overwrites the 16-bit count tile
    uint32_t off_rf, off_rf2, off_lf, off_lf2;
    uint32_t smem;         // dynamic shared memory including alignment slack
    uint32_t tmem_cols, t_row, t_col;
    // cluster mode (one thread-block cluster per block of the sweep)
    int SRr, SCc;          // rows of a row strip / columns of a column strip each CTA updates
    uint32_t off_cp;       // slots of this CTA's slices: row partials [TJ][2 fr][SRr], column [TI][2 fc][SCc]
    uint32_t off_st;       // the CTA's update slices: parameter rows, smoothed derivatives, visit counts
    uint32_t smem_cl;      // dynamic shared memory of the cluster kernels
};

struct TcState {
    TcLayout lay;
    CUtensorMap ymap[2];   // the count matrix in each of the handle's count buffers (ymap[1] once allocated)
    int TI, TJ;
    int cluster;           // 1: the strip updates run inside the tile launch (cluster mode)
    int persist;           // 1: a sweep range runs as one persistent launch (sweep_tc_epoch)
    int epi;               // epilogue variant (EPI_*)
    int flow;              // 1: a sweep range runs as one dataflow launch (sweep_tc_flow)
    int flow_grid;         // its CTAs
    int flow_groups;       // item groups staged for the next launch
    int4* fent;            // [2 nsw per]: group entries in launch order (see sweep_tc_flow)
    int* fstart;           // [2 nsw per + 1]: first ticket of each group
    unsigned* fctr;        // [3 + 2 per + max(r, s)]: the launch's counters
    int dev_grid;          // CTAs of the tensor-core deviance launch (0: the CUDA-core kernel runs)
    uint32_t dev_smem;     // its dynamic shared memory
    int dev_gen;           // 1: its variant with weights, missing entries or per-gene shapes
};

__device__ __forceinline__ void st_shared_v4(void* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(smem_u32(p)), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

__device__ __forceinline__ uint32_t bf16_bits(float x) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// Bounded wait shared by the CTA: thread 0 polls the mbarrier while the other
// threads wait at the CTA barrier, which takes no issue slots (with two tiles on
// an SM, 16 polling warps would steal them from the other tile's epilogue). The
// phase's completion, observed by thread 0, reaches the other threads through
// the barrier (its writes by TMA or by the tensor cores are visible to them
// after it; tcgen05 reads still follow a tcgen05 fence). True when the phase
// completed.
__device__ __forceinline__ bool cta_wait(uint64_t* bar, uint32_t parity, unsigned* err) {
    int ok = 1;
    if (threadIdx.x == 0) {
        ok = mbar_wait(bar, parity, WAIT_POLLS);
        if (!ok) {
            atomicOr(err, GMF_DEVERR_TIMEOUT);
            ok = mbar_wait(bar, parity, WAIT_POLLS);  // drain this CTA's own copies / MMAs
        }
    }
    return __syncthreads_and(ok) != 0;
}

template <bool COH>
__device__ __forceinline__ float4 ld_state4(const float* p) {
    return COH ? __ldcg((const float4*)p) : __ldg((const float4*)p);
}
template <bool COH>
__device__ __forceinline__ float ld_state(const float* p) {
    return COH ? __ldcg(p) : __ldg(p);
}

// Thread 0: the TMA load of the count tile at (row0, col0) into Ys.
__device__ __forceinline__ void issue_counts(const TcLayout& Lo, const CUtensorMap* ymap_p, uint8_t* Ys, int64_t row0,
                                             int64_t col0, uint64_t* bar) {
    mbar_arrive_expect_tx(bar, Lo.y_bytes);
    const int nbox = TT / Lo.JB;
    for (int b = 0; b < nbox; b++)
        tma_load_2d(Ys + b * ATOM, ymap_p, (int)(col0 + (int64_t)b * Lo.JB), (int)row0, bar);
}

// Operands. Thread groups of 128: L rows -> eta A; R rows -> eta B; L rows ->
// column-side B ([X, U] and squares); R rows -> row-side B ([Z, V] and squares).
template <bool COH>
__device__ __forceinline__ void build_operands(const StepArgs& a, const TcLayout& Lo, uint8_t* sm, int64_t row0,
                                               int64_t col0, int nr, int nc) {
    const int tid = threadIdx.x;
    uint8_t* Aop = sm + Lo.off_u;
    uint8_t* Bop = Aop + Lo.KA * ATOM;
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
                const float4 x = (ok && kk < a.KP) ? ld_state4<COH>(src + kk) : make_float4(0.f, 0.f, 0.f, 0.f);
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
                    for (int seg = 0; seg < 2; seg++) {
                        // segments of A and of B: hi, lo
                        const bool use_lo = seg == 1;
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
        // value and square of each multiplier column; K index of the contraction = the tile's row
        // (L side) or column (R side). Warp-wide: lane c reads column c of 8 consecutive rows (one
        // coalesced load per row) and writes those rows' BF16 values, 16 bytes, with one store.
        const int NF = isL ? Lo.NC : Lo.NR;
        const int nf = isL ? a.fc : a.fr;
        const int nvalid = isL ? nr : nc;
        const float* base = isL ? a.L + row0 * a.KP : a.R + col0 * a.KP;
        uint8_t* o1 = sm + (isL ? Lo.off_lf : Lo.off_rf);
        uint8_t* o2 = sm + (isL ? Lo.off_lf2 : Lo.off_rf2);
        const uint32_t atom = (uint32_t)NF * 128u;
        const int wq = (tid >> 5) & 3, lane = tid & 31;
        for (int c0 = 0; c0 < NF; c0 += 32) {
            const int c = c0 + lane;
            const bool cok = c < nf;
            const int col = cok ? (isL ? (c < a.p ? 1 + c : 1 + a.q + c) : 1 + a.p + c) : 0;
            // the warp's four 8-row groups rg = wq + 4 it: all 32 loads in flight before the first store
            float v[4][8];
#pragma unroll
            for (int it = 0; it < 4; it++)
#pragma unroll
                for (int u = 0; u < 8; u++) {
                    const int rr = 8 * (wq + 4 * it) + u;
                    v[it][u] = (cok && rr < nvalid) ? ld_state<COH>(base + (int64_t)rr * a.KP + col) : 0.f;
                }
            if (c < NF) {
#pragma unroll
                for (int it = 0; it < 4; it++) {
                    const int rg = wq + 4 * it;
                    const float* x = v[it];
                    const uint32_t off = (uint32_t)(rg >> 3) * atom + sw128_off(c, (8 * rg & 63) * 2);
                    st_shared_v4(o1 + off, pack_bf16x2(x[0], x[1]), pack_bf16x2(x[2], x[3]), pack_bf16x2(x[4], x[5]),
                                 pack_bf16x2(x[6], x[7]));
                    st_shared_v4(o2 + off, pack_bf16x2(x[0] * x[0], x[1] * x[1]), pack_bf16x2(x[2] * x[2], x[3] * x[3]),
                                 pack_bf16x2(x[4] * x[4], x[5] * x[5]), pack_bf16x2(x[6] * x[6], x[7] * x[7]));
                }
            }
        }
    }
}

// Thread 0: eta = L_hi R_hi' + L_lo R_hi' + L_hi R_lo' into TMEM columns [0,
// 128), from A = [L_hi | L_lo] and B = [R_hi | R_lo] (K chunks of 16 in that order).
__device__ __forceinline__ uint32_t kchunk_off(int k) {  // element k of a K-major row -> byte offset of its chunk
    return (uint32_t)(k >> 6) * ATOM + (uint32_t)((k & 63) >> 4) * 32u;
}
__device__ __forceinline__ void issue_eta(const TcLayout& Lo, uint8_t* sm, uint32_t tb, uint64_t* bar) {
    const uint8_t* Aop = sm + Lo.off_u;
    const uint8_t* Bop = Aop + Lo.KA * ATOM;
    const uint32_t id = idesc_bf16(TT, TT, 0, 0);
    const int nkc = Lo.KP16 / 16;
    for (int pr = 0; pr < 3; pr++) {
        const int sa = pr == 1 ? Lo.KP16 : 0, sb = pr == 2 ? Lo.KP16 : 0;  // (hi, hi), (lo, hi), (hi, lo)
        for (int kc = 0; kc < nkc; kc++) {
            umma_bf16(tb, sdesc(smem_u32(Aop) + kchunk_off(sa + 16 * kc), 16, 1024, SWIZZLE_128B),
                      sdesc(smem_u32(Bop) + kchunk_off(sb + 16 * kc), 16, 1024, SWIZZLE_128B), id, pr + kc > 0);
        }
    }
    umma_commit(bar);
}

}  // namespace gmftc

// Tensor-core deviance set-up of a handle (gmf_deviance_tc.cu), called once
// the tile layout and the count tensor map exist.
void gmf_tc_deviance_setup(gmf_model* h, gmftc::TcState* tc);
