// C ABI of the GB300 GMF library: handles, validation, permuted storage and
// the launch sequence of each entry point. The kernels live in
// gmf_step_simt.cu (FP32 path), gmf_step_tc.cu (tensor-core path),
// gmf_orth.cu (Algorithm 2) and gmf_project.cu (per-cell Fisher scoring).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <string>
#include <vector>

#include "gmf_internal.cuh"

static thread_local std::string g_err;

static int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CUDA_TRY(expr)                                                                             \
    do {                                                                                           \
        cudaError_t e_ = (expr);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(e_ == cudaErrorMemoryAllocation ? GMF_ERR_OOM : GMF_ERR_CUDA, "%s: %s (%s:%d)", \
                        #expr, cudaGetErrorString(e_), __FILE__, __LINE__);                        \
    } while (0)

extern "C" const char* gmf_last_error(void) { return g_err.c_str(); }

// Error reporting for gmf_noalloc.cu (same thread-local message as the ABI).
int gmf_noalloc_fail(int code, const char* msg) { return fail(code, "%s", msg); }
extern "C" const char* gmf_version(void) { return "gmf-gb300 0.1 (sm_103a)"; }

// tensor-core path hooks (gmf_step_tc.cu)
int gmf_tc_prepare_checked(gmf_model* h, std::string* err);
cudaError_t gmf_tc_launch(gmf_model* h, const StepArgs& a, int w, cudaStream_t st);
cudaError_t gmf_tc_launch_update(gmf_model* h, const StepArgs& a, int w, cudaStream_t st);
int gmf_tc_cluster(const gmf_model* h);
int gmf_tc_persistent(const gmf_model* h);
int gmf_tc_flow(const gmf_model* h);
int gmf_tc_stage_flow(gmf_model* h, const int32_t* sigma, int w0, int w1, cudaStream_t st);
cudaError_t gmf_tc_launch_epoch(gmf_model* h, int w0, int w1, cudaStream_t st);
int gmf_tc_set_ybuf(gmf_model* h, int idx, const void* Y);
void gmf_tc_free(gmf_model* h);

// One sweep launch of the configured path.
// A sweep is a tile launch and an update launch; t0/t1 (or null) are recorded
// around the tile launch.
static cudaError_t launch_sweep(gmf_model* h, const StepArgs& a, int w, cudaStream_t st, cudaEvent_t t0 = nullptr,
                                cudaEvent_t t1 = nullptr) {
    const bool mixed = h->cfg.precision == GMF_PREC_MIXED;
    cudaError_t e = t0 ? cudaEventRecord(t0, st) : cudaSuccess;
    if (e == cudaSuccess) e = mixed ? gmf_tc_launch(h, a, w, st) : gmf_launch_sweep_simt(h, a, w, st);
    if (e == cudaSuccess && t1) e = cudaEventRecord(t1, st);
    if (e == cudaSuccess) e = mixed ? gmf_tc_launch_update(h, a, w, st) : gmf_launch_update(a, w, GMF_TILE, st);
    return e;
}
// Algorithm 2 (gmf_orth.cu), per-cell projection (gmf_project.cu)
int gmf_orth_run(gmf_model* h, int mode, cudaStream_t st, std::string* err);
int gmf_project_run(gmf_model* h, const void* Ynew, int y16, int64_t n_new, const float* Xnew,
                    const float* off, const float* Ustart, int n_steps, float* Uout, float* Gout, float* dev,
                    cudaStream_t st, std::string* err);

extern "C" void gmf_config_default(gmf_config* c, int64_t n, int64_t m, int32_t p, int32_t q, int32_t d,
                                   int32_t family, int32_t nb_row, int32_t nb_col) {
    if (!c) return;
    memset(c, 0, sizeof *c);
    c->n = n;
    c->m = m;
    c->p = p;
    c->q = q;
    c->d = d;
    c->family = family;
    c->nb_row = nb_row;
    c->nb_col = nb_col;
    c->lambda[0] = 0.0;
    c->lambda[1] = 0.0;
    c->lambda[2] = 1.0;
    c->lambda[3] = 0.0;
    c->a1 = 0.1;
    c->a2 = 0.01;
    c->k0 = 0.01;
    c->k1 = 1e-3;
    c->tau = 0.75;
    c->damping = 1e-3;
    c->eps = 1e-8;
    c->eta_clamp = 30.0;
    c->precision = GMF_PREC_FP32;
}

static bool is_perm(const int32_t* p, int64_t n) {
    std::vector<char> seen((size_t)n, 0);
    for (int64_t i = 0; i < n; i++) {
        if (p[i] < 0 || p[i] >= n || seen[(size_t)p[i]]) return false;
        seen[(size_t)p[i]] = 1;
    }
    return true;
}

template <typename T>
static cudaError_t dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void**)p, count * sizeof(T));
}

static void trace_destroy(gmf_model* h) {
    if (!h->trace_ev) return;
    for (int i = 0; i < 2 * GMF_TRACE_POOL; i++) cudaEventDestroy(h->trace_ev[i]);
    delete[] h->trace_ev;
    h->trace_ev = nullptr;
}

static void release(gmf_model* h) {
    if (!h) return;
    trace_destroy(h);
    for (int i = 0; i < 2; i++)
        if (h->epoch_graph[i]) cudaGraphExecDestroy(h->epoch_graph[i]);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    if (h->tc) gmf_tc_free(h);
    if (h->ybuf[1]) {  // the second count buffer: wait for its last gather, free both buffers below
        if (h->copy_stream) cudaStreamSynchronize(h->copy_stream);
        cudaEventDestroy(h->y_ready);
        for (int i = 0; i < 2; i++) cudaEventDestroy(h->y_free[i]);
        cudaFree(h->ybuf[h->ycur ^ 1]);
        h->Yp = h->ybuf[h->ycur];
    }
    if (h->y_shared) {  // owned by another handle
        h->Yp = nullptr;
        h->Wp = nullptr;
        h->ystage = nullptr;
    }
    if (h->copy_stream) {
        cudaStreamSynchronize(h->copy_stream);
        cudaStreamDestroy(h->copy_stream);
    }
    if (h->up_init) {
        for (int i = 0; i < 2; i++) {
            cudaEventDestroy(h->up_copied[i]);
            cudaEventDestroy(h->up_free[i]);
        }
    }
    void* ptrs[] = {h->Yp, h->Wp, h->ystage2, h->L, h->R, h->GbR, h->HbR, h->GbC, h->HbC, h->cntR, h->cntC, h->alpha,
                    h->rperm, h->cperm, h->ystage, h->Rorig, h->kr_buf, h->partR, h->partC, h->nbpart, h->nbctr,
                    h->sigma, h->rhoc, h->rho1, h->need, h->kmap, h->strip_done, h->err, h->devpart, h->devtot,
                    h->alpha_col};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete[] h->h_rperm;
    delete[] h->h_cperm;
    delete h;
}

extern "C" void gmf_free(gmf_model* h) { release(h); }

// Host: build the permuted augmented factors L = [o|X|Gamma|U], R = [1|B|Z|V] as float32.
static void build_factors(const gmf_model* h, const double* X, const double* Z, const double* off,
                          const double* B, const double* G, const double* U, const double* V,
                          std::vector<float>& L, std::vector<float>& R) {
    const int K = h->KP, p = h->p, q = h->q, d = h->d;
    L.assign((size_t)h->n * K, 0.f);
    R.assign((size_t)h->m * K, 0.f);
    for (int64_t ip = 0; ip < h->n; ip++) {
        const int64_t i = h->h_rperm[ip];
        float* l = &L[(size_t)ip * K];
        l[0] = off ? (float)off[i] : 0.f;
        for (int a = 0; a < p; a++) l[1 + a] = (float)X[i * p + a];
        for (int b = 0; b < q; b++) l[1 + p + b] = (float)G[i * q + b];
        for (int c = 0; c < d; c++) l[1 + p + q + c] = (float)U[i * d + c];
    }
    for (int64_t jp = 0; jp < h->m; jp++) {
        const int64_t j = h->h_cperm[jp];
        float* r = &R[(size_t)jp * K];
        r[0] = 1.f;
        for (int a = 0; a < p; a++) r[1 + a] = (float)B[j * p + a];
        for (int b = 0; b < q; b++) r[1 + p + b] = (float)Z[j * q + b];
        for (int c = 0; c < d; c++) r[1 + p + q + c] = (float)V[j * d + c];
    }
}

// The device address of host counts the device can read with the gather
// kernel (16-byte aligned, rows of a multiple of 16 bytes), or null.
static const void* host_gather_src(const gmf_model* h, const void* Y) {
    void* d = nullptr;
    if (!gmf_gather_host_ok(h->y16, h->m) || ((uintptr_t)Y & 15u) != 0) return nullptr;
    if (cudaHostGetDevicePointer(&d, (void*)Y, 0) != cudaSuccess) {
        cudaGetLastError();  // (not page-locked)
        return nullptr;
    }
    return d;
}

static int upload_y(gmf_model* h, const void* Y, int on_device, cudaStream_t st) {
    const size_t bytes = (size_t)h->n * h->m * (h->y16 ? 2 : 4);
    const void* src = Y;
    const void* dsrc = on_device ? nullptr : host_gather_src(h, Y);
    if (dsrc) {  // one permuting gather over the host link, ordered on st
        CUDA_TRY(gmf_launch_gather_host(dsrc, h->Yp, h->y16, h->n, h->m, h->rperm, h->cperm, st));
        return GMF_OK;
    }
    if (!on_device) {
        if (!h->ystage) CUDA_TRY(cudaMalloc(&h->ystage, bytes));
        CUDA_TRY(cudaMemcpyAsync(h->ystage, Y, bytes, cudaMemcpyHostToDevice, st));
        src = h->ystage;
    }
    CUDA_TRY(gmf_launch_permute_y(src, h->Yp, h->y16, h->n, h->m, h->rperm, h->cperm, st));
    return GMF_OK;
}

// gmf_init, or (share != nullptr) a handle that reads the count matrix, the
// weights and the partitions of `share` instead of owning copies.
static int init_impl(gmf_model** out, const gmf_config* cfg, const void* Y, int32_t y_dtype, int32_t y_on_device,
                     const float* W, const double* X, const double* Z, const double* offset,
                     const int32_t* row_perm, const int32_t* col_perm, const double* B0, const double* G0,
                     const double* U0, const double* V0, double alpha0, void* stream, const gmf_model* share) {
    if (share) {
        Y = share->Yp;
        y_dtype = share->yf32 ? GMF_Y_FLOAT32 : share->y16 ? GMF_Y_UINT16 : GMF_Y_INT32;
        y_on_device = 1;
        W = share->Wp;
        row_perm = share->h_rperm;
        col_perm = share->h_cperm;
        if (cfg && (cfg->n != share->n || cfg->m != share->m || cfg->nb_row != share->cfg.nb_row ||
                    cfg->nb_col != share->cfg.nb_col))
            return fail(GMF_ERR_ARG, "gmf_init: a shared count matrix needs the same n, m and minibatch sizes");
    }
    if (!out) return fail(GMF_ERR_ARG, "gmf_init: out is NULL");
    *out = nullptr;
    if (!cfg) return fail(GMF_ERR_ARG, "gmf_init: cfg is NULL");
    const gmf_config& c = *cfg;
    if (c.n <= 0 || c.m <= 0) return fail(GMF_ERR_ARG, "gmf_init: n and m must be positive");
    if (c.n > (int64_t)INT32_MAX || c.m > (int64_t)INT32_MAX)
        return fail(GMF_ERR_ARG, "gmf_init: n and m must fit in int32");
    if (c.p < 0 || c.q < 0 || c.d < 0) return fail(GMF_ERR_ARG, "gmf_init: p, q, d must be >= 0");
    const int K = 1 + c.p + c.q + c.d;
    if (K > GMF_KMAX || c.q + c.d > GMF_FREE_MAX || c.p + c.d > GMF_FREE_MAX)
        return fail(GMF_ERR_ARG, "gmf_init: 1+p+q+d must be <= %d", GMF_KMAX);
    if (c.family < GMF_POISSON || c.family > GMF_INVGAUSS) return fail(GMF_ERR_ARG, "gmf_init: unknown family");
    if (c.nb_row <= 0 || c.nb_col <= 0) return fail(GMF_ERR_ARG, "gmf_init: minibatch sizes must be positive");
    if (c.bias_corr != 0 && c.bias_corr != 1) return fail(GMF_ERR_ARG, "gmf_init: bias_corr must be 0 or 1");
    if (c.alpha_mode < 0 || c.alpha_mode > 2) return fail(GMF_ERR_ARG, "gmf_init: alpha_mode must be 0, 1 or 2");
    if (c.precision != GMF_PREC_FP32 && c.precision != GMF_PREC_MIXED)
        return fail(GMF_ERR_ARG, "gmf_init: unknown precision");
    if (c.flags & ~(GMF_FLAG_NO_CLUSTER | GMF_FLAG_PERSIST | GMF_FLAG_SIMT_DEVIANCE | GMF_FLAG_STAGED_UPLOAD)) return fail(GMF_ERR_ARG, "gmf_init: unknown bits in flags");
    if (c.missing != 0 && c.missing != 1) return fail(GMF_ERR_ARG, "gmf_init: missing must be 0 or 1");
    if (!(c.a1 > 0 && c.a1 <= 1 && c.a2 > 0 && c.a2 <= 1)) return fail(GMF_ERR_ARG, "gmf_init: a1, a2 in (0, 1]");
    if (!(c.k0 > 0) || c.k1 < 0 || !(c.tau > 0)) return fail(GMF_ERR_ARG, "gmf_init: bad learning-rate schedule");
    if (c.damping < 0 || !(c.eta_clamp > 0)) return fail(GMF_ERR_ARG, "gmf_init: bad damping or eta_clamp");
    if (y_dtype != GMF_Y_INT32 && y_dtype != GMF_Y_UINT16 && y_dtype != GMF_Y_FLOAT32)
        return fail(GMF_ERR_ARG, "gmf_init: bad y_dtype");
    if (c.family <= GMF_NEGBIN && y_dtype == GMF_Y_FLOAT32)
        return fail(GMF_ERR_ARG, "gmf_init: the Poisson and NB families take int32 or uint16 counts");
    if ((c.family == GMF_GAUSSIAN || c.family == GMF_GAMMA || c.family == GMF_INVGAUSS) && y_dtype != GMF_Y_FLOAT32)
        return fail(GMF_ERR_ARG, "gmf_init: the Gaussian, Gamma and inverse Gaussian families take float32 responses");
    if (c.alpha_mode == 2 && c.family != GMF_NEGBIN)
        return fail(GMF_ERR_ARG, "gmf_init: alpha_mode 2 (per-gene shapes) is for the negative binomial");
    if (!Y || !X || !Z || !row_perm || !col_perm || !B0 || !G0 || !U0 || !V0)
        return fail(GMF_ERR_ARG, "gmf_init: a required pointer is NULL");
    if ((c.p > 0 && !X) || !(alpha0 > 0) ) return fail(GMF_ERR_ARG, "gmf_init: alpha0 must be > 0");
    if (!is_perm(row_perm, c.n)) return fail(GMF_ERR_ARG, "gmf_init: row_perm is not a permutation of 0..n-1");
    if (!is_perm(col_perm, c.m)) return fail(GMF_ERR_ARG, "gmf_init: col_perm is not a permutation of 0..m-1");

    gmf_model* h = new gmf_model();
    memset(h, 0, sizeof *h);
    h->cfg = c;
    h->flow_lag = 2;
    cudaGetDevice(&h->device);
    h->n = c.n;
    h->m = c.m;
    h->p = c.p;
    h->q = c.q;
    h->d = c.d;
    h->K = K;
    h->KP = (K + 3) & ~3;
    h->fr = c.q + c.d;
    h->fc = c.p + c.d;
    h->r = (int)((c.n + c.nb_row - 1) / c.nb_row);
    h->s = (int)((c.m + c.nb_col - 1) / c.nb_col);
    h->swap = h->r < h->s;
    h->nsw = h->swap ? h->s : h->r;
    h->per = h->swap ? h->r : h->s;
    h->TI = (int)((std::min<int64_t>(c.nb_row, c.n) + GMF_TILE - 1) / GMF_TILE);
    h->TJ = (int)((std::min<int64_t>(c.nb_col, c.m) + GMF_TILE - 1) / GMF_TILE);
    h->y16 = y_dtype == GMF_Y_UINT16;
    h->yf32 = y_dtype == GMF_Y_FLOAT32;
    h->h_rperm = new int32_t[c.n];
    h->h_cperm = new int32_t[c.m];
    memcpy(h->h_rperm, row_perm, sizeof(int32_t) * c.n);
    memcpy(h->h_cperm, col_perm, sizeof(int32_t) * c.m);
    cudaStream_t st = (cudaStream_t)stream;

#define INIT_TRY(expr)                   \
    do {                                 \
        int rc_ = (expr);                \
        if (rc_ != GMF_OK) {             \
            std::string keep = g_err;    \
            release(h);                  \
            g_err = keep;                \
            return rc_;                  \
        }                                \
    } while (0)
#define INIT_CUDA(expr) INIT_TRY(([&]() -> int { CUDA_TRY(expr); return GMF_OK; })())

    const size_t nm = (size_t)c.n * c.m;
    if (share) {
        h->Yp = share->Yp;
        h->Wp = share->Wp;
        h->y_shared = 1;
    } else {
        INIT_CUDA(cudaMalloc(&h->Yp, nm * (h->y16 ? 2 : 4)));
        if (W) INIT_CUDA(dalloc(&h->Wp, nm));
    }
    h->ybuf[0] = h->Yp;
    INIT_CUDA(dalloc(&h->L, (size_t)c.n * h->KP));
    INIT_CUDA(dalloc(&h->R, (size_t)c.m * h->KP));
    INIT_CUDA(dalloc(&h->GbR, (size_t)c.n * h->fr));
    INIT_CUDA(dalloc(&h->HbR, (size_t)c.n * h->fr));
    INIT_CUDA(dalloc(&h->GbC, (size_t)c.m * h->fc));
    INIT_CUDA(dalloc(&h->HbC, (size_t)c.m * h->fc));
    INIT_CUDA(dalloc(&h->cntR, (size_t)c.n));
    INIT_CUDA(dalloc(&h->cntC, (size_t)c.m));
    INIT_CUDA(dalloc(&h->alpha, 1));
    if (c.alpha_mode == 2) INIT_CUDA(dalloc(&h->alpha_col, (size_t)c.m));
    INIT_CUDA(dalloc(&h->rperm, (size_t)c.n));
    INIT_CUDA(dalloc(&h->cperm, (size_t)c.m));
    {
        // partial slots of the FP32 path's 64 x 64 tiles or the tensor-core path's 128 x 128 tiles
        const size_t TI2 = (size_t)((std::min<int64_t>(c.nb_row, c.n) + 127) / 128);
        const size_t TJ2 = (size_t)((std::min<int64_t>(c.nb_col, c.m) + 127) / 128);
        const size_t tiles = std::max((size_t)h->TI * h->TJ * GMF_TILE, TI2 * TJ2 * 128);
        INIT_CUDA(dalloc(&h->partR, (size_t)h->per * tiles * 2 * std::max(h->fr, 1)));
        INIT_CUDA(dalloc(&h->partC, (size_t)h->per * tiles * 2 * std::max(h->fc, 1)));
    }
    INIT_CUDA(dalloc(&h->nbpart, (size_t)2 * h->per * h->TI * h->TJ));
    INIT_CUDA(dalloc(&h->nbctr, 1));
    INIT_CUDA(dalloc(&h->sigma, (size_t)h->nsw));
    INIT_CUDA(dalloc(&h->rhoc, (size_t)h->nsw * h->per));
    INIT_CUDA(dalloc(&h->rho1, (size_t)h->nsw));
    INIT_CUDA(dalloc(&h->need, (size_t)h->nsw * h->per));
    INIT_CUDA(dalloc(&h->kmap, (size_t)h->per));
    INIT_CUDA(dalloc(&h->strip_done, (size_t)std::max(h->r, h->s)));
    INIT_CUDA(dalloc(&h->err, 1));
    h->devparts = (int)(((c.n + GMF_TILE - 1) / GMF_TILE) * ((c.m + GMF_TILE - 1) / GMF_TILE));
    INIT_CUDA(dalloc(&h->devpart, (size_t)h->devparts));
    INIT_CUDA(dalloc(&h->devtot, 1));

    INIT_CUDA(cudaMemcpyAsync(h->rperm, row_perm, sizeof(int32_t) * c.n, cudaMemcpyHostToDevice, st));
    INIT_CUDA(cudaMemcpyAsync(h->cperm, col_perm, sizeof(int32_t) * c.m, cudaMemcpyHostToDevice, st));
    INIT_CUDA(cudaMemsetAsync(h->GbR, 0, sizeof(float) * c.n * h->fr, st));
    INIT_CUDA(cudaMemsetAsync(h->HbR, 0, sizeof(float) * c.n * h->fr, st));
    INIT_CUDA(cudaMemsetAsync(h->GbC, 0, sizeof(float) * c.m * h->fc, st));
    INIT_CUDA(cudaMemsetAsync(h->HbC, 0, sizeof(float) * c.m * h->fc, st));
    INIT_CUDA(cudaMemsetAsync(h->cntR, 0, sizeof(int) * c.n, st));
    INIT_CUDA(cudaMemsetAsync(h->cntC, 0, sizeof(int) * c.m, st));
    INIT_CUDA(cudaMemsetAsync(h->err, 0, sizeof(unsigned), st));
    INIT_CUDA(cudaMemsetAsync(h->nbctr, 0, sizeof(unsigned), st));
    float a0 = (float)alpha0;
    INIT_CUDA(cudaMemcpyAsync(h->alpha, &a0, sizeof(float), cudaMemcpyHostToDevice, st));
    if (h->alpha_col) {   // every gene starts from alpha0
        const std::vector<float> ac((size_t)c.m, a0);
        INIT_CUDA(cudaMemcpyAsync(h->alpha_col, ac.data(), sizeof(float) * c.m, cudaMemcpyHostToDevice, st));
    }
    {
        std::vector<float> L, R;
        build_factors(h, X, Z, offset, B0, G0, U0, V0, L, R);
        INIT_CUDA(cudaMemcpyAsync(h->L, L.data(), sizeof(float) * L.size(), cudaMemcpyHostToDevice, st));
        INIT_CUDA(cudaMemcpyAsync(h->R, R.data(), sizeof(float) * R.size(), cudaMemcpyHostToDevice, st));
        INIT_CUDA(cudaStreamSynchronize(st));
    }
    if (!share) INIT_TRY(upload_y(h, Y, y_on_device, st));
    if (W && !share) {
        float* wsrc = (float*)W;
        float* wtmp = nullptr;
        if (!y_on_device) {
            INIT_CUDA(dalloc(&wtmp, nm));
            INIT_CUDA(cudaMemcpyAsync(wtmp, W, nm * sizeof(float), cudaMemcpyHostToDevice, st));
            wsrc = wtmp;
        }
        INIT_CUDA(gmf_launch_permute_w(wsrc, h->Wp, c.n, c.m, h->rperm, h->cperm, st));
        INIT_CUDA(cudaStreamSynchronize(st));
        if (wtmp) cudaFree(wtmp);
    }
    INIT_CUDA(gmf_sweep_simt_attr(h));
    if (c.precision == GMF_PREC_MIXED) {
        std::string err;
        const int rc = gmf_tc_prepare_checked(h, &err);
        if (rc != GMF_OK) {
            release(h);
            return fail(rc, "gmf_init: %s", err.c_str());
        }
    }
    INIT_CUDA(cudaStreamSynchronize(st));
    *out = h;
    return GMF_OK;
}

extern "C" int gmf_init(gmf_model** out, const gmf_config* cfg, const void* Y, int32_t y_dtype, int32_t y_on_device,
                        const float* W, const double* X, const double* Z, const double* offset,
                        const int32_t* row_perm, const int32_t* col_perm, const double* B0, const double* G0,
                        const double* U0, const double* V0, double alpha0, void* stream) {
    return init_impl(out, cfg, Y, y_dtype, y_on_device, W, X, Z, offset, row_perm, col_perm, B0, G0, U0, V0, alpha0,
                     stream, nullptr);
}

int gmf_init_shared(gmf_model** out, const gmf_config* cfg, const gmf_model* owner, const double* X, const double* Z,
                    const double* offset, const double* B0, const double* G0, const double* U0, const double* V0,
                    double alpha0, void* stream) {
    return init_impl(out, cfg, nullptr, 0, 1, nullptr, X, Z, offset, nullptr, nullptr, B0, G0, U0, V0, alpha0, stream,
                     owner);
}

int gmf_fail(int code, const char* msg) { return fail(code, "%s", msg); }

extern "C" int gmf_update_y(gmf_model* h, const void* Y, int32_t y_on_device, void* stream) {
    if (!h || !Y) return fail(GMF_ERR_ARG, "gmf_update_y: NULL argument");
    if (h->y_shared) return fail(GMF_ERR_STATE, "gmf_update_y: this handle reads another handle's counts");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = upload_y(h, Y, y_on_device, st);
    if (rc) return rc;
    if (!y_on_device) CUDA_TRY(cudaStreamSynchronize(st));
    return GMF_OK;
}

extern "C" int gmf_update_y_async(gmf_model* h, const void* Y, void* stream) {
    if (!h || !Y) return fail(GMF_ERR_ARG, "gmf_update_y_async: NULL argument");
    if (h->y_shared) return fail(GMF_ERR_STATE, "gmf_update_y_async: this handle reads another handle's counts");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)h->n * h->m * (h->y16 ? 2 : 4);
    if (!h->copy_stream) CUDA_TRY(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    // Direct path: page-locked, mapped host memory is read by one gather kernel on
    // the copy stream into the count buffer that is not current; the handle then
    // switches buffers, so work already enqueued on `st` keeps its counts.
    const void* dsrc = (h->y_fixed || (h->cfg.flags & GMF_FLAG_STAGED_UPLOAD)) ? nullptr : host_gather_src(h, Y);
    if (dsrc) {
        if (!h->ybuf[1]) {  // the second buffer, its events and its TMA descriptor, all or nothing
            void* buf = nullptr;
            cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
            bool okb = cudaMalloc(&buf, bytes) == cudaSuccess;
            for (int i = 0; i < 3 && okb; i++) okb = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) == cudaSuccess;
            okb = okb && gmf_tc_set_ybuf(h, 1, buf) == GMF_OK;
            if (!okb) {
                for (int i = 0; i < 3; i++)
                    if (ev[i]) cudaEventDestroy(ev[i]);
                if (buf) cudaFree(buf);
                cudaGetLastError();
                return fail(GMF_ERR_CUDA, "gmf_update_y_async: cannot set up the second count buffer");
            }
            h->ybuf[1] = buf;
            h->y_ready = ev[0];
            h->y_free[0] = ev[1];
            h->y_free[1] = ev[2];
        }
        const int nb = h->ycur ^ 1;
        CUDA_TRY(cudaEventRecord(h->y_free[h->ycur], st));          // the current buffer's readers so far
        CUDA_TRY(cudaStreamWaitEvent(h->copy_stream, h->y_free[nb], 0));  // nb's last readers (none at first)
        CUDA_TRY(gmf_launch_gather_host(dsrc, h->ybuf[nb], h->y16, h->n, h->m, h->rperm, h->cperm, h->copy_stream));
        CUDA_TRY(cudaEventRecord(h->y_ready, h->copy_stream));
        CUDA_TRY(cudaStreamWaitEvent(st, h->y_ready, 0));
        h->ycur = nb;
        h->Yp = h->ybuf[nb];
        return GMF_OK;
    }
    if (!h->up_init) {
        if (!h->ystage) CUDA_TRY(cudaMalloc(&h->ystage, bytes));
        CUDA_TRY(cudaMalloc(&h->ystage2, bytes));
        for (int i = 0; i < 2; i++) {
            CUDA_TRY(cudaEventCreateWithFlags(&h->up_copied[i], cudaEventDisableTiming));
            CUDA_TRY(cudaEventCreateWithFlags(&h->up_free[i], cudaEventDisableTiming));
        }
        h->up_init = 1;
    }
    const int i = h->up_idx;
    h->up_idx ^= 1;
    void* buf = i ? h->ystage2 : h->ystage;
    // the copy into buf waits for the permutation that last read buf (no wait before its first use)
    CUDA_TRY(cudaStreamWaitEvent(h->copy_stream, h->up_free[i], 0));
    CUDA_TRY(cudaMemcpyAsync(buf, Y, bytes, cudaMemcpyHostToDevice, h->copy_stream));
    CUDA_TRY(cudaEventRecord(h->up_copied[i], h->copy_stream));
    CUDA_TRY(cudaStreamWaitEvent(st, h->up_copied[i], 0));
    CUDA_TRY(gmf_launch_permute_y(buf, h->Yp, h->y16, h->n, h->m, h->rperm, h->cperm, st));
    CUDA_TRY(cudaEventRecord(h->up_free[i], st));
    return GMF_OK;
}

extern "C" int32_t gmf_num_sweeps(const gmf_model* h) { return h ? h->nsw : -1; }

extern "C" int32_t gmf_count_buffers(const gmf_model* h) {
    if (!h) return -1;
    return h->ybuf[1] ? 2 : 1;
}

extern "C" int32_t gmf_epoch_mode(const gmf_model* h) {
    if (!h) return -1;
    if (h->cfg.precision != GMF_PREC_MIXED) return GMF_EPOCH_SEPARATE;
    if (gmf_tc_persistent(h)) return GMF_EPOCH_PERSISTENT;
    return gmf_tc_cluster(h) ? GMF_EPOCH_CLUSTER : GMF_EPOCH_SEPARATE;
}

extern "C" int32_t gmf_launches_per_sweep(const gmf_model* h) {
    if (!h) return -1;
    const int mode = gmf_epoch_mode(h);
    return mode == GMF_EPOCH_PERSISTENT ? 0 : mode == GMF_EPOCH_CLUSTER ? 1 : 2;
}

// Visits of each block's moving strip by the earlier sweeps of [w_begin, w_end)
// (the blocks of one sweep move along disjoint strips).
static void strip_need(int r, int s, const int32_t* sigma, int w_begin, int w_end, int32_t* need) {
    const int swap = r < s, per = std::min(r, s), mod = swap ? s : r;
    std::vector<int32_t> visits((size_t)mod, 0);
    for (int w = w_begin; w < w_end; w++) {
        for (int k = 0; k < per; k++) need[(size_t)(w - w_begin) * per + k] = visits[(size_t)((sigma[w] + k) % mod)];
        for (int k = 0; k < per; k++) visits[(size_t)((sigma[w] + k) % mod)]++;
    }
}

extern "C" int gmf_strip_schedule(int32_t r, int32_t s, const int32_t* sigma, int32_t w_begin, int32_t w_end,
                                  int32_t* need_out) {
    if (!sigma || !need_out) return fail(GMF_ERR_ARG, "gmf_strip_schedule: NULL argument");
    if (r < 1 || s < 1) return fail(GMF_ERR_ARG, "gmf_strip_schedule: r = %d, s = %d", r, s);
    const int S = std::max(r, s);
    if (w_begin < 0 || w_end > S || w_begin > w_end)
        return fail(GMF_ERR_ARG, "gmf_strip_schedule: sweep range [%d, %d) outside [0, %d)", w_begin, w_end, S);
    for (int w = 0; w < S; w++)
        if (sigma[w] < 0 || sigma[w] >= S) return fail(GMF_ERR_ARG, "gmf_strip_schedule: sigma[%d] = %d", w, sigma[w]);
    strip_need(r, s, sigma, w_begin, w_end, need_out);
    return GMF_OK;
}

// Wait for the recorded event pairs and add their durations to the running total.
static int trace_collect(gmf_model* h, cudaStream_t st) {
    if (!h->trace_ev || h->trace_used == 0) return GMF_OK;
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int i = 0; i < h->trace_used; i++) {
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, h->trace_ev[2 * i], h->trace_ev[2 * i + 1]));
        h->trace_ms += ms;
    }
    h->trace_launches += h->trace_used;
    h->trace_used = 0;
    return GMF_OK;
}

// Copy the epoch's sweep offsets and the step factors of every block of the
// range [w_begin, w_end) to the device, in FP64 on the host: block k of sweep w
// has t = t_now + (w - w_begin) * per + k + 1.
int gmf_stage_schedule(gmf_model* h, const int32_t* sigma, int w_begin, int w_end, cudaStream_t st) {
    const gmf_config& c = h->cfg;
    std::vector<float> rc((size_t)h->nsw * h->per, 0.f), r1((size_t)h->nsw, 0.f);
    for (int w = w_begin; w < w_end; w++) {
        for (int k = 0; k < h->per; k++) {
            const double t = (double)(h->t + (int64_t)(w - w_begin) * h->per + k + 1);
            const double rho = c.k0 / pow(1.0 + c.k0 * c.k1 * t, c.tau);
            const double ct = c.bias_corr == 0 ? (1.0 - pow(c.a2, t)) / (1.0 - pow(c.a1, t)) : 1.0;
            rc[(size_t)w * h->per + k] = (float)(rho * ct);
            if (k == 0) r1[w] = (float)rho;
        }
    }
    CUDA_TRY(cudaMemcpyAsync(h->rhoc, rc.data(), sizeof(float) * rc.size(), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(h->rho1, r1.data(), sizeof(float) * r1.size(), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(h->sigma, sigma, sizeof(int32_t) * h->nsw, cudaMemcpyHostToDevice, st));
    if (gmf_tc_persistent(h)) {
        std::vector<int32_t> need((size_t)h->nsw * h->per, 0);
        strip_need(h->r, h->s, sigma, w_begin, w_end, need.data() + (size_t)w_begin * h->per);
        if (h->need_extra > 0)
            for (size_t i = (size_t)w_begin * h->per; i < (size_t)w_end * h->per; i++) need[i] += h->need_extra;
        CUDA_TRY(cudaMemcpyAsync(h->need, need.data(), sizeof(int32_t) * need.size(), cudaMemcpyHostToDevice, st));
        if (gmf_tc_flow(h)) {
            const int rc = gmf_tc_stage_flow(h, sigma, w_begin, w_end, st);
            if (rc) return fail(rc, "staging the dataflow epoch's item order failed");
        }
    }
    return GMF_OK;
}

extern "C" int gmf_sgd_sweeps(gmf_model* h, const int32_t* sigma, int32_t w_begin, int32_t w_end, void* stream) {
    if (!h || !sigma) return fail(GMF_ERR_ARG, "gmf_sgd_sweeps: NULL argument");
    if (w_begin < 0 || w_end > h->nsw || w_begin > w_end)
        return fail(GMF_ERR_ARG, "gmf_sgd_sweeps: sweep range [%d, %d) outside [0, %d)", w_begin, w_end, h->nsw);
    if (!is_perm(sigma, h->nsw)) return fail(GMF_ERR_ARG, "gmf_sgd_sweeps: sigma is not a permutation of 0..%d", h->nsw - 1);
    cudaStream_t st = (cudaStream_t)stream;
    {
        const int rc = gmf_stage_schedule(h, sigma, w_begin, w_end, st);
        if (rc) return rc;
    }
    if (gmf_tc_persistent(h)) {  // the range is one launch
        if (w_begin == w_end) return GMF_OK;
        cudaEvent_t t0 = nullptr, t1 = nullptr;
        if (h->trace_on) {
            if (h->trace_used == GMF_TRACE_POOL) {
                int rc = trace_collect(h, st);
                if (rc) return rc;
            }
            t0 = h->trace_ev[2 * h->trace_used];
            t1 = h->trace_ev[2 * h->trace_used + 1];
            h->trace_used++;
        }
        if (t0) CUDA_TRY(cudaEventRecord(t0, st));
        CUDA_TRY(gmf_tc_launch_epoch(h, w_begin, w_end, st));
        if (t1) CUDA_TRY(cudaEventRecord(t1, st));
        h->t += (int64_t)(w_end - w_begin) * h->per;
        return GMF_OK;
    }
    const StepArgs a = gmf_make_args(h);
    // A whole epoch replays one captured graph of its sweep launches (the
    // launches read sigma and the step factors from the buffers filled above).
    if (!h->trace_on && w_begin == 0 && w_end == h->nsw) {
        cudaGraphExec_t& graph = h->epoch_graph[h->ycur];  // the launches hold the count buffer's address
        if (!graph) {
            if (!h->capture_stream) CUDA_TRY(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            CUDA_TRY(cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal));
            for (int w = 0; w < h->nsw; w++) {
                cudaError_t e = launch_sweep(h, a, w, h->capture_stream);
                if (e != cudaSuccess) {
                    cudaStreamEndCapture(h->capture_stream, &g);
                    if (g) cudaGraphDestroy(g);
                    return fail(GMF_ERR_CUDA, "sweep launch during capture: %s", cudaGetErrorString(e));
                }
            }
            CUDA_TRY(cudaStreamEndCapture(h->capture_stream, &g));
            cudaError_t e = cudaGraphInstantiate(&graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                graph = nullptr;
                return fail(GMF_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
            }
        }
        CUDA_TRY(cudaGraphLaunch(graph, st));
        h->t += (int64_t)h->nsw * h->per;
        return GMF_OK;
    }
    for (int w = w_begin; w < w_end; w++) {
        if (h->trace_on) {
            if (h->trace_used == GMF_TRACE_POOL) {
                int rc = trace_collect(h, st);
                if (rc) return rc;
            }
            CUDA_TRY(launch_sweep(h, a, w, st, h->trace_ev[2 * h->trace_used], h->trace_ev[2 * h->trace_used + 1]));
            h->trace_used++;
        } else {
            CUDA_TRY(launch_sweep(h, a, w, st));
        }
        h->t += h->per;
    }
    return GMF_OK;
}

extern "C" int gmf_trace(gmf_model* h, int32_t enable) {
    if (!h) return fail(GMF_ERR_ARG, "gmf_trace: NULL handle");
    if (enable && !h->trace_ev) {
        h->trace_ev = new cudaEvent_t[2 * GMF_TRACE_POOL];
        for (int i = 0; i < 2 * GMF_TRACE_POOL; i++) CUDA_TRY(cudaEventCreate(&h->trace_ev[i]));
    }
    h->trace_on = enable ? 1 : 0;
    return GMF_OK;
}

extern "C" int gmf_trace_read(gmf_model* h, double* total_ms, int64_t* launches, void* stream) {
    if (!h || !total_ms || !launches) return fail(GMF_ERR_ARG, "gmf_trace_read: NULL argument");
    int rc = trace_collect(h, (cudaStream_t)stream);
    if (rc) return rc;
    *total_ms = h->trace_ms;
    *launches = h->trace_launches;
    h->trace_ms = 0.0;
    h->trace_launches = 0;
    return GMF_OK;
}

extern "C" int gmf_sgd_sweep_blocks(gmf_model* h, const int32_t* sigma, int32_t w, const int32_t* blocks,
                                    int32_t nblocks, void* stream) {
    if (!h || !sigma || (nblocks > 0 && !blocks)) return fail(GMF_ERR_ARG, "gmf_sgd_sweep_blocks: NULL argument");
    if (w < 0 || w >= h->nsw) return fail(GMF_ERR_ARG, "gmf_sgd_sweep_blocks: sweep %d outside [0, %d)", w, h->nsw);
    if (nblocks < 0 || nblocks > h->per)
        return fail(GMF_ERR_ARG, "gmf_sgd_sweep_blocks: %d blocks outside [0, %d]", nblocks, h->per);
    for (int i = 0; i < nblocks; i++)
        if (blocks[i] < 0 || blocks[i] >= h->per || (i > 0 && blocks[i] <= blocks[i - 1]))
            return fail(GMF_ERR_ARG, "gmf_sgd_sweep_blocks: blocks must increase within [0, %d)", h->per);
    if (!is_perm(sigma, h->nsw))
        return fail(GMF_ERR_ARG, "gmf_sgd_sweep_blocks: sigma is not a permutation of 0..%d", h->nsw - 1);
    if (h->cfg.alpha_mode == 1 && h->cfg.family != GMF_POISSON && h->cfg.family != GMF_BINOMIAL && nblocks < h->per)
        return fail(GMF_ERR_STATE, "gmf_sgd_sweep_blocks: the pooled NB shape update needs every block of the sweep");
    cudaStream_t st = (cudaStream_t)stream;
    {
        const int rc = gmf_stage_schedule(h, sigma, w, w + 1, st);
        if (rc) return rc;
    }
    if (nblocks > 0) {
        // a pageable copy of the list: staged before cudaMemcpyAsync returns, whatever memory the caller passed
        const std::vector<int32_t> kb(blocks, blocks + nblocks);
        CUDA_TRY(cudaMemcpyAsync(h->kmap, kb.data(), sizeof(int32_t) * nblocks, cudaMemcpyHostToDevice, st));
        StepArgs a = gmf_make_args(h);
        a.kmap = h->kmap;
        a.nk = nblocks;
        CUDA_TRY(launch_sweep(h, a, w, st));
    }
    h->t += h->per;
    return GMF_OK;
}

extern "C" int64_t gmf_chunk_bytes(const gmf_model* h, int32_t side, int32_t chunk) {
    if (!h || (side != 0 && side != 1)) return -1;
    const int64_t nb = side == 0 ? h->cfg.nb_row : h->cfg.nb_col;
    const int64_t tot = side == 0 ? h->n : h->m;
    const int64_t nch = (tot + nb - 1) / nb;
    if (chunk < 0 || chunk >= nch) return -1;
    const int64_t rows = std::min(nb, tot - (int64_t)chunk * nb);
    const int nf = side == 0 ? h->fr : h->fc;
    return rows * (h->KP + 2 * nf + 1) * (int64_t)sizeof(float);
}

extern "C" int gmf_chunk_state(gmf_model* h, int32_t side, int32_t chunk, void* buf, int32_t write, void* stream) {
    if (!h || !buf) return fail(GMF_ERR_ARG, "gmf_chunk_state: NULL argument");
    if (gmf_chunk_bytes(h, side, chunk) < 0)
        return fail(GMF_ERR_ARG, "gmf_chunk_state: side %d chunk %d out of range", side, chunk);
    if (write != 0 && write != 1) return fail(GMF_ERR_ARG, "gmf_chunk_state: write must be 0 or 1");
    const int64_t nb = side == 0 ? h->cfg.nb_row : h->cfg.nb_col;
    const int64_t tot = side == 0 ? h->n : h->m;
    const int64_t first = (int64_t)chunk * nb;
    const int rows = (int)std::min(nb, tot - first);
    if (side == 0)
        CUDA_TRY(gmf_launch_chunk_state(h->L, h->GbR, h->HbR, h->cntR, h->KP, h->fr, first, rows, (float*)buf, write,
                                        (cudaStream_t)stream));
    else
        CUDA_TRY(gmf_launch_chunk_state(h->R, h->GbC, h->HbC, h->cntC, h->KP, h->fc, first, rows, (float*)buf, write,
                                        (cudaStream_t)stream));
    return GMF_OK;
}

int gmf_gene_moments_run(gmf_model* h, double* sums, cudaStream_t st, const char** why);
static int check_err_word(gmf_model* h, cudaStream_t st);

extern "C" int gmf_set_gene_shapes(gmf_model* h, const double* alpha, void* stream) {
    if (!h || !alpha) return fail(GMF_ERR_ARG, "gmf_set_gene_shapes: NULL argument");
    if (h->cfg.family > GMF_NEGBIN) return fail(GMF_ERR_STATE, "gmf_set_gene_shapes: Poisson and negative binomial fits only");
    if (h->cfg.alpha_mode != 2) return fail(GMF_ERR_STATE, "gmf_set_gene_shapes: the fit has one shape (alpha_mode != 2)");
    std::vector<float> ac((size_t)h->m);
    for (int64_t jp = 0; jp < h->m; jp++) {
        const double v = alpha[h->h_cperm[jp]];
        if (!(v > 0) || !std::isfinite(v)) return fail(GMF_ERR_ARG, "gmf_set_gene_shapes: shapes must be positive");
        ac[jp] = (float)v;
    }
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(h->alpha_col, ac.data(), sizeof(float) * ac.size(), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return GMF_OK;
}

extern "C" int gmf_get_gene_shapes(gmf_model* h, double* alpha, void* stream) {
    if (!h || !alpha) return fail(GMF_ERR_ARG, "gmf_get_gene_shapes: NULL argument");
    if (h->cfg.alpha_mode != 2) return fail(GMF_ERR_STATE, "gmf_get_gene_shapes: the fit has one shape (alpha_mode != 2)");
    std::vector<float> ac((size_t)h->m);
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(ac.data(), h->alpha_col, sizeof(float) * ac.size(), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int64_t jp = 0; jp < h->m; jp++) alpha[h->h_cperm[jp]] = ac[jp];
    return GMF_OK;
}

extern "C" int gmf_gene_shape_moments(gmf_model* h, double eps, double cap, double* alpha_out, void* stream) {
    if (!h || !alpha_out) return fail(GMF_ERR_ARG, "gmf_gene_shape_moments: NULL argument");
    if (h->cfg.family > GMF_NEGBIN) return fail(GMF_ERR_STATE, "gmf_gene_shape_moments: Poisson and negative binomial fits only");
    if (!(eps > 0) || !(cap >= eps)) return fail(GMF_ERR_ARG, "gmf_gene_shape_moments: need 0 < eps <= cap");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<double> sums((size_t)2 * h->m);
    const char* why = "";
    const int rc = gmf_gene_moments_run(h, sums.data(), st, &why);
    if (rc) return fail(rc, "gmf_gene_shape_moments: %s", why);
    for (int64_t jp = 0; jp < h->m; jp++) {
        const double num = sums[2 * jp], den = sums[2 * jp + 1];
        alpha_out[h->h_cperm[jp]] = den > 0 ? std::min(std::max(num / den, eps), cap) : cap;
    }
    return check_err_word(h, st);
}

int gmf_gene_ml_run(gmf_model* h, double* alpha, int iters, double tol, double lo, double hi, int* iters_done,
                    cudaStream_t st, const char** why);

extern "C" int gmf_gene_shape_ml(gmf_model* h, const double* start, int32_t iters, double tol, double lo, double hi,
                                 double* alpha_out, int32_t* iters_done, void* stream) {
    if (!h || !alpha_out) return fail(GMF_ERR_ARG, "gmf_gene_shape_ml: NULL argument");
    if (h->cfg.family != GMF_NEGBIN) return fail(GMF_ERR_STATE, "gmf_gene_shape_ml: the fit is not negative binomial");
    if (iters < 1 || iters > 200) return fail(GMF_ERR_ARG, "gmf_gene_shape_ml: iters %d outside [1, 200]", iters);
    if (!(lo > 0) || !(hi >= lo) || !std::isfinite(hi) || !(tol >= 0))
        return fail(GMF_ERR_ARG, "gmf_gene_shape_ml: need 0 < lo <= hi < inf and tol >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<double> al((size_t)h->m);
    if (start) {
        for (int64_t jp = 0; jp < h->m; jp++) {
            const double v = start[h->h_cperm[jp]];
            if (!(v > 0) || !std::isfinite(v)) return fail(GMF_ERR_ARG, "gmf_gene_shape_ml: start shapes must be positive");
            al[jp] = std::min(std::max(v, lo), hi);
        }
    } else {
        std::vector<float> cur((size_t)(h->cfg.alpha_mode == 2 ? h->m : 1));
        CUDA_TRY(cudaMemcpyAsync(cur.data(), h->cfg.alpha_mode == 2 ? h->alpha_col : h->alpha,
                                 sizeof(float) * cur.size(), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        for (int64_t jp = 0; jp < h->m; jp++)
            al[jp] = std::min(std::max((double)cur[h->cfg.alpha_mode == 2 ? jp : 0], lo), hi);
    }
    const char* why = "";
    int done = 0;
    const int rc = gmf_gene_ml_run(h, al.data(), iters, tol, lo, hi, &done, st, &why);
    if (rc) return fail(rc, "gmf_gene_shape_ml: %s", why);
    for (int64_t jp = 0; jp < h->m; jp++) alpha_out[h->h_cperm[jp]] = al[jp];
    if (iters_done) *iters_done = done;
    return check_err_word(h, st);
}

int gmf_init_run(gmf_model* h, int power_iters, uint64_t seed, double* sv_out, cudaStream_t st, std::string* err);
int gmf_loadings_run(gmf_model* h, int n_steps, double* obj_out, cudaStream_t st, std::string* err);

// A new start: the smoothed derivatives, visit counts and t begin again.
static int restart_optimiser(gmf_model* h, cudaStream_t st) {
    CUDA_TRY(cudaMemsetAsync(h->GbR, 0, sizeof(float) * h->n * h->fr, st));
    CUDA_TRY(cudaMemsetAsync(h->HbR, 0, sizeof(float) * h->n * h->fr, st));
    CUDA_TRY(cudaMemsetAsync(h->GbC, 0, sizeof(float) * h->m * h->fc, st));
    CUDA_TRY(cudaMemsetAsync(h->HbC, 0, sizeof(float) * h->m * h->fc, st));
    CUDA_TRY(cudaMemsetAsync(h->cntR, 0, sizeof(int) * h->n, st));
    CUDA_TRY(cudaMemsetAsync(h->cntC, 0, sizeof(int) * h->m, st));
    h->t = 0;
    return GMF_OK;
}

extern "C" int gmf_fit_loadings(gmf_model* h, int32_t n_steps, double* obj_out, void* stream) {
    if (!h) return fail(GMF_ERR_ARG, "gmf_fit_loadings: NULL handle");
    if (h->cfg.family > GMF_NEGBIN) return fail(GMF_ERR_STATE, "gmf_fit_loadings: Poisson and negative binomial fits only");
    if (n_steps < 0 || n_steps > 100) return fail(GMF_ERR_ARG, "gmf_fit_loadings: n_steps %d outside [0, 100]", n_steps);
    if (h->cfg.missing) return fail(GMF_ERR_STATE, "gmf_fit_loadings: the column GLMs need every count observed");
    cudaStream_t st = (cudaStream_t)stream;
    std::string err;
    const int rc = gmf_loadings_run(h, n_steps, obj_out, st, &err);
    if (rc) return fail(rc, "gmf_fit_loadings: %s", err.c_str());
    const int rr = restart_optimiser(h, st);
    if (rr) return rr;
    return check_err_word(h, st);
}

extern "C" int gmf_initialize(gmf_model* h, int32_t power_iters, uint64_t seed, double* sv_out, void* stream) {
    if (!h) return fail(GMF_ERR_ARG, "gmf_initialize: NULL handle");
    if (h->cfg.family > GMF_NEGBIN) return fail(GMF_ERR_STATE, "gmf_initialize: Poisson and negative binomial fits only");
    if (power_iters < 0 || power_iters > 20)
        return fail(GMF_ERR_ARG, "gmf_initialize: power_iters %d outside [0, 20]", power_iters);
    if (h->cfg.missing) return fail(GMF_ERR_STATE, "gmf_initialize: the least-squares start needs every count observed");
    cudaStream_t st = (cudaStream_t)stream;
    std::string err;
    const int rc = gmf_init_run(h, power_iters, seed, sv_out, st, &err);
    if (rc) return fail(rc, "gmf_initialize: %s", err.c_str());
    // a new start: the smoothed derivatives, visit counts and t begin again
    CUDA_TRY(cudaMemsetAsync(h->GbR, 0, sizeof(float) * h->n * h->fr, st));
    CUDA_TRY(cudaMemsetAsync(h->HbR, 0, sizeof(float) * h->n * h->fr, st));
    CUDA_TRY(cudaMemsetAsync(h->GbC, 0, sizeof(float) * h->m * h->fc, st));
    CUDA_TRY(cudaMemsetAsync(h->HbC, 0, sizeof(float) * h->m * h->fc, st));
    CUDA_TRY(cudaMemsetAsync(h->cntR, 0, sizeof(int) * h->n, st));
    CUDA_TRY(cudaMemsetAsync(h->cntC, 0, sizeof(int) * h->m, st));
    h->t = 0;
    return check_err_word(h, st);
}

extern "C" int gmf_set_flow_lag(gmf_model* h, int32_t lag) {
    if (!h) return fail(GMF_ERR_ARG, "gmf_set_flow_lag: NULL handle");
    if (lag < 0 || lag > 64) return fail(GMF_ERR_ARG, "gmf_set_flow_lag: lag %d outside [0, 64]", lag);
    h->flow_lag = lag;
    return GMF_OK;
}

extern "C" int gmf_set_wait_limit(gmf_model* h, int64_t limit_ns, int32_t need_extra) {
    if (!h) return fail(GMF_ERR_ARG, "gmf_set_wait_limit: NULL handle");
    if (limit_ns < 0 || limit_ns > 60000000000ll)
        return fail(GMF_ERR_ARG, "gmf_set_wait_limit: limit_ns %lld outside [0, 6e10]", (long long)limit_ns);
    if (need_extra < 0) return fail(GMF_ERR_ARG, "gmf_set_wait_limit: need_extra %d < 0", need_extra);
    h->wait_ns = limit_ns;
    h->need_extra = need_extra;
    return GMF_OK;
}

extern "C" int gmf_sgd_epoch(gmf_model* h, const int32_t* sigma, void* stream) {
    if (!h) return fail(GMF_ERR_ARG, "gmf_sgd_epoch: NULL handle");
    return gmf_sgd_sweeps(h, sigma, 0, h->nsw, stream);
}

static int check_err_word(gmf_model* h, cudaStream_t st) {
    unsigned e = 0;
    CUDA_TRY(cudaMemcpyAsync(&e, h->err, sizeof e, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (e & GMF_DEVERR_TIMEOUT) return fail(GMF_ERR_TIMEOUT, "a device-side wait timed out");
    if (e & GMF_DEVERR_NONFINITE) return fail(GMF_ERR_NONFINITE, "a parameter update produced a non-finite value");
    if (e & GMF_DEVERR_BOUNDS) return fail(GMF_ERR_STATE, "a device-side bounds check failed");
    return GMF_OK;
}

extern "C" int gmf_deviance_async(gmf_model* h, double* d_out, void* stream) {
    if (!h || !d_out) return fail(GMF_ERR_ARG, "gmf_deviance_async: NULL argument");
    CUDA_TRY(gmf_launch_deviance(h, d_out, (cudaStream_t)stream));
    return GMF_OK;
}

int gmf_holdout_run(gmf_model* h, const void* Ytrue, double* out, cudaStream_t st, const char** why);
int gmf_loglik_run(gmf_model* h, double* out, cudaStream_t st, const char** why);

extern "C" int gmf_loglik(gmf_model* h, double* out, void* stream) {
    if (!h || !out) return fail(GMF_ERR_ARG, "gmf_loglik: NULL argument");
    if (h->cfg.family > GMF_NEGBIN) return fail(GMF_ERR_STATE, "gmf_loglik: Poisson and negative binomial fits only");
    cudaStream_t st = (cudaStream_t)stream;
    const char* why = "";
    const int rc = gmf_loglik_run(h, out, st, &why);
    if (rc) return fail(rc, "gmf_loglik: %s", why);
    return check_err_word(h, st);
}

extern "C" int gmf_holdout(gmf_model* h, const void* Ytrue, double* out, void* stream) {
    if (!h || !Ytrue || !out) return fail(GMF_ERR_ARG, "gmf_holdout: NULL argument");
    if (h->cfg.family > GMF_NEGBIN) return fail(GMF_ERR_STATE, "gmf_holdout: Poisson and negative binomial fits only");
    if (!h->cfg.missing) return fail(GMF_ERR_STATE, "gmf_holdout: the fit has no missing entries (cfg.missing = 0)");
    cudaStream_t st = (cudaStream_t)stream;
    const char* why = "";
    const int rc = gmf_holdout_run(h, Ytrue, out, st, &why);
    if (rc) return fail(rc, "gmf_holdout: %s", why);
    return check_err_word(h, st);
}

extern "C" int gmf_deviance(gmf_model* h, double* out_total, void* stream) {
    if (!h || !out_total) return fail(GMF_ERR_ARG, "gmf_deviance: NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(gmf_launch_deviance(h, h->devtot, st));
    CUDA_TRY(cudaMemcpyAsync(out_total, h->devtot, sizeof(double), cudaMemcpyDeviceToHost, st));
    return check_err_word(h, st);
}

extern "C" int gmf_get_params(gmf_model* h, double* B, double* G, double* U, double* V, double* alpha,
                              void* stream) {
    if (!h) return fail(GMF_ERR_ARG, "gmf_get_params: NULL handle");
    cudaStream_t st = (cudaStream_t)stream;
    const int K = h->KP, p = h->p, q = h->q, d = h->d;
    std::vector<float> L((size_t)h->n * K), R((size_t)h->m * K);
    float a = 0.f;
    CUDA_TRY(cudaMemcpyAsync(L.data(), h->L, sizeof(float) * L.size(), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(R.data(), h->R, sizeof(float) * R.size(), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(&a, h->alpha, sizeof(float), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int64_t ip = 0; ip < h->n; ip++) {
        const int64_t i = h->h_rperm[ip];
        const float* l = &L[(size_t)ip * K];
        if (G)
            for (int b = 0; b < q; b++) G[i * q + b] = l[1 + p + b];
        if (U)
            for (int c = 0; c < d; c++) U[i * d + c] = l[1 + p + q + c];
    }
    for (int64_t jp = 0; jp < h->m; jp++) {
        const int64_t j = h->h_cperm[jp];
        const float* r = &R[(size_t)jp * K];
        if (B)
            for (int b = 0; b < p; b++) B[j * p + b] = r[1 + b];
        if (V)
            for (int c = 0; c < d; c++) V[j * d + c] = r[1 + p + q + c];
    }
    if (alpha) *alpha = a;
    return check_err_word(h, st);
}

extern "C" int gmf_set_params(gmf_model* h, const double* B, const double* G, const double* U, const double* V,
                              const double* alpha, void* stream) {
    if (!h) return fail(GMF_ERR_ARG, "gmf_set_params: NULL handle");
    cudaStream_t st = (cudaStream_t)stream;
    const int K = h->KP, p = h->p, q = h->q, d = h->d;
    std::vector<float> L((size_t)h->n * K), R((size_t)h->m * K);
    CUDA_TRY(cudaMemcpyAsync(L.data(), h->L, sizeof(float) * L.size(), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(R.data(), h->R, sizeof(float) * R.size(), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int64_t ip = 0; ip < h->n; ip++) {
        const int64_t i = h->h_rperm[ip];
        float* l = &L[(size_t)ip * K];
        if (G)
            for (int b = 0; b < q; b++) l[1 + p + b] = (float)G[i * q + b];
        if (U)
            for (int c = 0; c < d; c++) l[1 + p + q + c] = (float)U[i * d + c];
    }
    for (int64_t jp = 0; jp < h->m; jp++) {
        const int64_t j = h->h_cperm[jp];
        float* r = &R[(size_t)jp * K];
        if (B)
            for (int b = 0; b < p; b++) r[1 + b] = (float)B[j * p + b];
        if (V)
            for (int c = 0; c < d; c++) r[1 + p + q + c] = (float)V[j * d + c];
    }
    CUDA_TRY(cudaMemcpyAsync(h->L, L.data(), sizeof(float) * L.size(), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(h->R, R.data(), sizeof(float) * R.size(), cudaMemcpyHostToDevice, st));
    if (alpha) {
        if (!(*alpha > 0)) return fail(GMF_ERR_ARG, "gmf_set_params: alpha must be > 0");
        float a = (float)*alpha;
        CUDA_TRY(cudaMemcpyAsync(h->alpha, &a, sizeof(float), cudaMemcpyHostToDevice, st));
    }
    CUDA_TRY(cudaMemsetAsync(h->err, 0, sizeof(unsigned), st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return GMF_OK;
}

// rows of a (rows x cols) permuted float matrix <-> original-order double matrix
static void unpermute(const std::vector<float>& src, double* dst, const int32_t* perm, int64_t rows, int cols) {
    for (int64_t ip = 0; ip < rows; ip++)
        for (int c = 0; c < cols; c++) dst[(int64_t)perm[ip] * cols + c] = src[(size_t)ip * cols + c];
}
static void permute_rows(const double* src, std::vector<float>& dst, const int32_t* perm, int64_t rows, int cols) {
    dst.resize((size_t)rows * cols);
    for (int64_t ip = 0; ip < rows; ip++)
        for (int c = 0; c < cols; c++) dst[(size_t)ip * cols + c] = (float)src[(int64_t)perm[ip] * cols + c];
}

extern "C" int gmf_get_ema(gmf_model* h, double* Gb_row, double* Hb_row, double* Gb_col, double* Hb_col,
                           int64_t* cnt_row, int64_t* cnt_col, int64_t* t_io, void* stream) {
    if (!h) return fail(GMF_ERR_ARG, "gmf_get_ema: NULL handle");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<float> buf;
    struct Item { double* dst; float* src; int64_t rows; int cols; const int32_t* perm; };
    Item items[] = {{Gb_row, h->GbR, h->n, h->fr, h->h_rperm}, {Hb_row, h->HbR, h->n, h->fr, h->h_rperm},
                    {Gb_col, h->GbC, h->m, h->fc, h->h_cperm}, {Hb_col, h->HbC, h->m, h->fc, h->h_cperm}};
    for (auto& it : items) {
        if (!it.dst) continue;
        buf.resize((size_t)it.rows * it.cols);
        CUDA_TRY(cudaMemcpyAsync(buf.data(), it.src, sizeof(float) * buf.size(), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        unpermute(buf, it.dst, it.perm, it.rows, it.cols);
    }
    struct CItem { int64_t* dst; int* src; int64_t rows; const int32_t* perm; };
    CItem citems[] = {{cnt_row, h->cntR, h->n, h->h_rperm}, {cnt_col, h->cntC, h->m, h->h_cperm}};
    for (auto& it : citems) {
        if (!it.dst) continue;
        std::vector<int> cb((size_t)it.rows);
        CUDA_TRY(cudaMemcpyAsync(cb.data(), it.src, sizeof(int) * cb.size(), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        for (int64_t ip = 0; ip < it.rows; ip++) it.dst[it.perm[ip]] = cb[(size_t)ip];
    }
    if (t_io) *t_io = h->t;
    return GMF_OK;
}

extern "C" int gmf_set_ema(gmf_model* h, const double* Gb_row, const double* Hb_row, const double* Gb_col,
                           const double* Hb_col, const int64_t* cnt_row, const int64_t* cnt_col, const int64_t* t_in,
                           void* stream) {
    if (!h) return fail(GMF_ERR_ARG, "gmf_set_ema: NULL handle");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<float> buf;
    struct Item { const double* src; float* dst; int64_t rows; int cols; const int32_t* perm; };
    Item items[] = {{Gb_row, h->GbR, h->n, h->fr, h->h_rperm}, {Hb_row, h->HbR, h->n, h->fr, h->h_rperm},
                    {Gb_col, h->GbC, h->m, h->fc, h->h_cperm}, {Hb_col, h->HbC, h->m, h->fc, h->h_cperm}};
    for (auto& it : items) {
        if (!it.src) continue;
        permute_rows(it.src, buf, it.perm, it.rows, it.cols);
        CUDA_TRY(cudaMemcpyAsync(it.dst, buf.data(), sizeof(float) * buf.size(), cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaStreamSynchronize(st));
    }
    struct CItem { const int64_t* src; int* dst; int64_t rows; const int32_t* perm; };
    CItem citems[] = {{cnt_row, h->cntR, h->n, h->h_rperm}, {cnt_col, h->cntC, h->m, h->h_cperm}};
    for (auto& it : citems) {
        if (!it.src) continue;
        std::vector<int> cb((size_t)it.rows);
        for (int64_t ip = 0; ip < it.rows; ip++) {
            const int64_t v = it.src[it.perm[ip]];
            if (v < 0 || v > INT32_MAX) return fail(GMF_ERR_ARG, "gmf_set_ema: visit counter out of range");
            cb[(size_t)ip] = (int)v;
        }
        CUDA_TRY(cudaMemcpyAsync(it.dst, cb.data(), sizeof(int) * cb.size(), cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaStreamSynchronize(st));
    }
    if (t_in) {
        if (*t_in < 0) return fail(GMF_ERR_ARG, "gmf_set_ema: t must be >= 0");
        h->t = *t_in;
    }
    CUDA_TRY(cudaMemsetAsync(h->err, 0, sizeof(unsigned), st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return GMF_OK;
}

extern "C" int gmf_orthogonalize(gmf_model* h, int32_t mode, void* stream) {
    if (!h) return fail(GMF_ERR_ARG, "gmf_orthogonalize: NULL handle");
    if (mode != GMF_ORTH_B1 && mode != GMF_ORTH_B2 && mode != GMF_ORTH_B3)
        return fail(GMF_ERR_ARG, "gmf_orthogonalize: mode must be GMF_ORTH_B1, B2 or B3");
    std::string err;
    int rc = gmf_orth_run(h, mode, (cudaStream_t)stream, &err);
    if (rc) return fail(rc, "gmf_orthogonalize: %s", err.c_str());
    return GMF_OK;
}

extern "C" int gmf_project_cells(gmf_model* h, const void* Ynew, int32_t y_dtype, int64_t n_new, const float* Xnew,
                                 const float* offset_new, const float* U_start, int32_t n_steps, float* U_out,
                                 float* G_out, float* dev_out, void* stream) {
    if (!h) return fail(GMF_ERR_ARG, "gmf_project_cells: NULL handle");
    if (h->cfg.family > GMF_NEGBIN) return fail(GMF_ERR_STATE, "gmf_project_cells: Poisson and negative binomial fits only");
    if (n_new < 0 || n_new > (int64_t)INT32_MAX) return fail(GMF_ERR_ARG, "gmf_project_cells: bad n_new");
    if (y_dtype != GMF_Y_INT32 && y_dtype != GMF_Y_UINT16) return fail(GMF_ERR_ARG, "gmf_project_cells: bad y_dtype");
    if (n_steps < 0 || n_steps > 1000) return fail(GMF_ERR_ARG, "gmf_project_cells: n_steps in [0, 1000]");
    if (n_new == 0) return GMF_OK;  // an empty batch (its pointers may be NULL)
    if (!Ynew || !U_out || !G_out) return fail(GMF_ERR_ARG, "gmf_project_cells: NULL argument");
    if (h->cfg.alpha_mode == 2)
        return fail(GMF_ERR_STATE, "gmf_project_cells: per-gene NB shapes are not supported by the projection");
    if (h->p > 0 && !Xnew) return fail(GMF_ERR_ARG, "gmf_project_cells: Xnew is NULL");
    std::string err;
    int rc = gmf_project_run(h, Ynew, y_dtype == GMF_Y_UINT16, n_new, Xnew, offset_new, U_start, n_steps, U_out,
                             G_out, dev_out, (cudaStream_t)stream, &err);
    if (rc) return fail(rc, "gmf_project_cells: %s", err.c_str());
    return GMF_OK;
}
