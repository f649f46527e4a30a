// The starting values of Sec. 4.1 in the least-squares form the paper gives
// for high-dimensional data: ordinary least squares on the link-transformed
// counts instead of the column and row GLMs, and the leading singular vectors
// of the remaining residual for both factors.
//
//   E     = log(Y + 1/2) - o 1'                                (n x m, FP32, in HBM)
//   B     = E' X (X'X)^-1          (m x p: one least-squares fit per gene, X shared)
//   Gamma = (E - X B') Z (Z'Z)^-1  (n x q: one least-squares fit per cell, Z shared)
//   E    <- E - X B' - Gamma Z'
//   E    ~= P diag(s) Q' (rank d), U = P diag(s)^(1/2), V = Q diag(s)^(1/2)
//
// The products with E run as cuBLAS SGEMMs (plain library GEMMs, FP32); the
// rank-d factorisation is a randomized subspace iteration (Halko, Martinsson
// and Tropp's range finder: d + 10 Gaussian test vectors, `power_iters` power
// steps, each basis orthonormalised by Cholesky QR twice in FP64 with DGEMMs);
// the small systems and the k x k eigen-decomposition run on the host in FP64.
// Everything is in the handle's permuted row and column order.
#include <cublas_v2.h>
#include <math.h>
#include <string.h>

#include <string>
#include <vector>

#include "gmf_internal.cuh"
#include "gmf_linalg.h"
#include "gmf_update.cuh"

namespace {

using namespace gmfla;

// E_ij = log(y_ij + 1/2) - o_i
__global__ void ztrans_kernel(const void* Y, int y16, int64_t n, int64_t m, const float* L, int KP, float* E) {
    const int64_t total = n * m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / m;
        const float y = y16 ? (float)((const unsigned short*)Y)[e] : (float)((const int*)Y)[e];
        E[e] = logf(y + 0.5f) - L[i * KP];
    }
}

// E_ij -= sum_{c = 1}^{c1 - 1} L_ic R_jc (the covariate and cell-intercept terms of eta)
constexpr int ST = 32;
__global__ void sub_fixed_kernel(float* E, int64_t n, int64_t m, const float* L, const float* R, int KP, int c1) {
    __shared__ float Ls[ST][GMF_KMAX + 1], Rs[ST][GMF_KMAX + 1];
    const int64_t i0 = (int64_t)blockIdx.y * ST, j0 = (int64_t)blockIdx.x * ST;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int e = ty * ST + tx; e < ST * c1; e += ST * 8) {
        const int r = e / c1, c = e - r * c1;
        Ls[r][c] = i0 + r < n ? L[(i0 + r) * KP + c] : 0.f;
        Rs[r][c] = j0 + r < m ? R[(j0 + r) * KP + c] : 0.f;
    }
    __syncthreads();
    for (int rr = ty; rr < ST; rr += 8) {
        const int64_t i = i0 + rr, j = j0 + tx;
        if (i >= n || j >= m) continue;
        float s = 0.f;
        for (int c = 1; c < c1; c++) s = fmaf(Ls[rr][c], Rs[tx][c], s);
        E[i * m + j] -= s;
    }
}

__global__ void to_double_kernel(const float* x, double* y, int64_t count) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        y[e] = (double)x[e];
}
__global__ void to_float_kernel(const double* x, float* y, int64_t count) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        y[e] = (float)x[e];
}

int grid_of(int64_t count) { return (int)std::min<int64_t>((count + 255) / 256, 8192); }

// SplitMix64 (Steele, Lea and Flood) and the Box-Muller transform: the Gaussian test vectors.
struct Rng {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return ((double)(next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    double normal() { return sqrt(-2.0 * log(uniform())) * cos(6.283185307179586 * uniform()); }
};

struct Work {
    std::vector<void*> ptrs;
    cudaStream_t st;
    ~Work() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
    }
    template <typename T>
    T* alloc(size_t count) {
        void* p = nullptr;
        if (cudaMallocAsync(&p, sizeof(T) * std::max<size_t>(count, 1), st) != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return (T*)p;
    }
};

#define IN_CU(expr)                                        \
    do {                                                   \
        cudaError_t e_ = (expr);                           \
        if (e_ != cudaSuccess) {                           \
            *err = std::string(#expr) + ": " + cudaGetErrorString(e_); \
            return GMF_ERR_CUDA;                           \
        }                                                  \
    } while (0)
#define IN_BL(expr)                                        \
    do {                                                   \
        if ((expr) != CUBLAS_STATUS_SUCCESS) {             \
            *err = std::string("cuBLAS: ") + #expr;        \
            return GMF_ERR_CUDA;                           \
        }                                                  \
    } while (0)

// Orthonormalise the columns of the rows x k column-major FP64 matrix A (ld
// rows) in place by Cholesky QR, twice: A <- A R^-1 with R'R = A'A.
int cholqr2(cublasHandle_t bl, double* A, int64_t rows, int k, double* G, double* Ri, cudaStream_t st,
            std::string* err) {
    const double one = 1.0, zero = 0.0;
    std::vector<double> g((size_t)k * k);
    for (int rep = 0; rep < 2; rep++) {
        IN_BL(cublasDgemm(bl, CUBLAS_OP_T, CUBLAS_OP_N, k, k, (int)rows, &one, A, (int)rows, A, (int)rows, &zero, G, k));
        IN_CU(cudaMemcpyAsync(g.data(), G, sizeof(double) * g.size(), cudaMemcpyDeviceToHost, st));
        IN_CU(cudaStreamSynchronize(st));
        Mat C;
        if (!cholesky(g, k, C)) {
            *err = "the residual has rank below the requested number of factors";
            return GMF_ERR_STATE;
        }
        const Mat Rinv = upper_inverse(transpose(C, k, k), k);   // R = C' (upper), row-major
        const Mat Rc = transpose(Rinv, k, k);                      // column-major for cuBLAS
        IN_CU(cudaMemcpyAsync(Ri, Rc.data(), sizeof(double) * Rc.size(), cudaMemcpyHostToDevice, st));
        IN_BL(cublasDtrmm(bl, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, (int)rows, k,
                          &one, Ri, k, A, (int)rows, A, (int)rows));
    }
    return GMF_OK;
}

// ---- column GLMs for the loadings (the last step of Sec. 4.1). One launch per
// chunk of rows: thread = gene j of a segment of the chunk's rows; eta (from the
// chunk's SGEMM, in E) becomes w Ddot in place and w Dddot in DD (Sec. 3, log
// link); the segment's weighted unit deviances (Table S1, App. B) are summed
// with compensation and added to devpart[seg][j] (the same thread across the
// chunks, so the sums are deterministic).
__global__ void glm_col_kernel(const void* Y, int y16, const float* W, float* E, float* DD, double* devpart,
                               int64_t r0, int rows, int64_t m, int seg_rows, const float* alpha_p,
                               const float* alpha_col, int nb, float clamp) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int s = blockIdx.y;
    const int i0 = s * seg_rows, i1 = min(rows, i0 + seg_rows);
    const float a = alpha_col ? alpha_col[j] : *alpha_p;
    float sum = 0.f, comp = 0.f;
    for (int i = i0; i < i1; i++) {
        const int64_t g = (r0 + i) * m + j, c = (int64_t)i * m + j;
        const float y = y16 ? (float)((const unsigned short*)Y)[g] : (float)((const int*)Y)[g];
        const float w = W ? W[g] : 1.f;
        const float e = fminf(fmaxf(E[c], -clamp), clamp);
        const float mu = expf(e);
        const float f = nb ? a / (a + mu) : 1.f;
        E[c] = w * f * (y - mu);
        DD[c] = w * f * mu;
        const float hd = y > 0.f ? gmfdev::half_dev_ratio(nb, y, e, mu, a) : (nb ? a * log1pf(mu / a) : mu);
        const float t = 2.f * w * hd - comp;
        const float u = sum + t;
        comp = (u - sum) - t;
        sum = u;
    }
    devpart[(int64_t)s * m + j] += (double)sum;
}

// KR[i][pair(a, b)] = u_ia u_ib, a <= b (pairs in row order of the upper triangle), for the chunk's rows.
__global__ void kr_kernel(const float* L, int KP, int c0, int64_t r0, int rows, int d, int P, float* KR) {
    const int64_t total = (int64_t)rows * P;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / P;
        int pr = (int)(e - i * P), a = 0;
        while (pr >= d - a) {
            pr -= d - a;
            a++;
        }
        const int b = a + pr;
        const float* u = L + (r0 + i) * KP + c0;
        KR[e] = u[a] * u[b];
    }
}

}  // namespace

int gmf_init_run(gmf_model* h, int power_iters, uint64_t seed, double* sv_out, cudaStream_t st, std::string* err) {
    const int64_t n = h->n, m = h->m;
    const int p = h->p, q = h->q, d = h->d, KP = h->KP;
    Work w{{}, st};
    float* E = w.alloc<float>((size_t)n * m);
    if (!E) {
        *err = "no device memory for the n x m residual";
        return GMF_ERR_OOM;
    }
    cublasHandle_t bl = nullptr;
    if (cublasCreate(&bl) != CUBLAS_STATUS_SUCCESS) {
        *err = "cublasCreate failed";
        return GMF_ERR_CUDA;
    }
    struct BlGuard {
        cublasHandle_t b;
        ~BlGuard() { cublasDestroy(b); }
    } guard{bl};
    IN_BL(cublasSetStream(bl, st));
    IN_BL(cublasSetMathMode(bl, CUBLAS_PEDANTIC_MATH));   // FP32 products, no TF32
    const float onef = 1.f, zerof = 0.f;

    ztrans_kernel<<<grid_of(n * m), 256, 0, st>>>(h->Yp, h->y16, n, m, h->L, KP, E);
    IN_CU(cudaGetLastError());

    // host copies of the fixed covariates (permuted order): X = L[:, 1..p], Z = R[:, 1+p..1+p+q]
    std::vector<float> Lh((size_t)n * KP), Rh((size_t)m * KP);
    IN_CU(cudaMemcpyAsync(Lh.data(), h->L, sizeof(float) * Lh.size(), cudaMemcpyDeviceToHost, st));
    IN_CU(cudaMemcpyAsync(Rh.data(), h->R, sizeof(float) * Rh.size(), cudaMemcpyDeviceToHost, st));

    // B: S1 = E' X (m x p, column-major = row-major p x m)
    Mat B((size_t)m * p, 0.0);
    if (p > 0) {
        float* S1 = w.alloc<float>((size_t)m * p);
        IN_BL(cublasSgemm(bl, CUBLAS_OP_N, CUBLAS_OP_T, (int)m, p, (int)n, &onef, E, (int)m, h->L + 1, KP, &zerof, S1,
                          (int)m));
        std::vector<float> s1((size_t)m * p);
        IN_CU(cudaMemcpyAsync(s1.data(), S1, sizeof(float) * s1.size(), cudaMemcpyDeviceToHost, st));
        IN_CU(cudaStreamSynchronize(st));
        Mat XtX((size_t)p * p, 0.0);
        for (int64_t i = 0; i < n; i++)
            for (int a = 0; a < p; a++)
                for (int b = 0; b < p; b++) XtX[a * p + b] += (double)Lh[i * KP + 1 + a] * Lh[i * KP + 1 + b];
        Mat rhs((size_t)p * m);   // p x m
        for (int a = 0; a < p; a++)
            for (int64_t j = 0; j < m; j++) rhs[a * m + j] = s1[(size_t)a * m + j];
        if (!spd_solve(XtX, p, rhs, (int)m)) {
            *err = "X'X is singular";
            return GMF_ERR_STATE;
        }
        for (int64_t j = 0; j < m; j++)
            for (int a = 0; a < p; a++) B[j * p + a] = rhs[a * m + j];
    } else {
        IN_CU(cudaStreamSynchronize(st));
    }
    // Gamma: S2 = E Z (n x q, column-major q x n = row-major n x q), minus X (B' Z)
    Mat G((size_t)n * q, 0.0);
    if (q > 0) {
        float* S2 = w.alloc<float>((size_t)n * q);
        IN_BL(cublasSgemm(bl, CUBLAS_OP_N, CUBLAS_OP_N, q, (int)n, (int)m, &onef, h->R + 1 + p, KP, E, (int)m, &zerof,
                          S2, q));
        std::vector<float> s2((size_t)n * q);
        IN_CU(cudaMemcpyAsync(s2.data(), S2, sizeof(float) * s2.size(), cudaMemcpyDeviceToHost, st));
        IN_CU(cudaStreamSynchronize(st));
        Mat ZtZ((size_t)q * q, 0.0), BtZ((size_t)p * q, 0.0);
        for (int64_t j = 0; j < m; j++)
            for (int a = 0; a < q; a++) {
                const double za = Rh[j * KP + 1 + p + a];
                for (int b = 0; b < q; b++) ZtZ[a * q + b] += za * Rh[j * KP + 1 + p + b];
                for (int b = 0; b < p; b++) BtZ[b * q + a] += B[j * p + b] * za;
            }
        Mat rhs((size_t)q * n);   // q x n
        for (int64_t i = 0; i < n; i++)
            for (int a = 0; a < q; a++) {
                double v = s2[(size_t)i * q + a];
                for (int b = 0; b < p; b++) v -= (double)Lh[i * KP + 1 + b] * BtZ[b * q + a];
                rhs[a * n + i] = v;
            }
        if (!spd_solve(ZtZ, q, rhs, (int)n)) {
            *err = "Z'Z is singular";
            return GMF_ERR_STATE;
        }
        for (int64_t i = 0; i < n; i++)
            for (int a = 0; a < q; a++) G[i * q + a] = rhs[a * n + i];
    }
    // write B and Gamma into the factors, then E <- E - X B' - Gamma Z'
    for (int64_t j = 0; j < m; j++)
        for (int a = 0; a < p; a++) Rh[j * KP + 1 + a] = (float)B[j * p + a];
    for (int64_t i = 0; i < n; i++)
        for (int a = 0; a < q; a++) Lh[i * KP + 1 + p + a] = (float)G[i * q + a];
    for (int64_t i = 0; i < n; i++)
        for (int c = 1 + p + q; c < 1 + p + q + d; c++) Lh[i * KP + c] = 0.f;
    for (int64_t j = 0; j < m; j++)
        for (int c = 1 + p + q; c < 1 + p + q + d; c++) Rh[j * KP + c] = 0.f;
    IN_CU(cudaMemcpyAsync(h->L, Lh.data(), sizeof(float) * Lh.size(), cudaMemcpyHostToDevice, st));
    IN_CU(cudaMemcpyAsync(h->R, Rh.data(), sizeof(float) * Rh.size(), cudaMemcpyHostToDevice, st));
    if (1 + p + q > 1) {
        sub_fixed_kernel<<<dim3((unsigned)((m + ST - 1) / ST), (unsigned)((n + ST - 1) / ST)), dim3(ST, 8), 0, st>>>(
            E, n, m, h->L, h->R, KP, 1 + p + q);
        IN_CU(cudaGetLastError());
    }

    if (d > 0) {
        const int k = (int)std::min<int64_t>(d + 10, std::min(n, m));
        // column-major operands: Ec = E' (m x n, ld m); Omega / Qm (m x k, ld m); Qn (n x k, ld n)
        float* Om = w.alloc<float>((size_t)m * k);
        float* Yf = w.alloc<float>((size_t)n * k);
        double* Yd = w.alloc<double>((size_t)n * k);
        float* Zf = w.alloc<float>((size_t)m * k);
        double* Zd = w.alloc<double>((size_t)m * k);
        double* Gd = w.alloc<double>((size_t)k * k);
        double* Ri = w.alloc<double>((size_t)k * k);
        if (!Om || !Yf || !Yd || !Zf || !Zd || !Gd || !Ri) {
            *err = "no device memory for the subspace iteration";
            return GMF_ERR_OOM;
        }
        {
            std::vector<float> om((size_t)m * k);
            Rng rng{seed};
            for (auto& v : om) v = (float)rng.normal();
            IN_CU(cudaMemcpyAsync(Om, om.data(), sizeof(float) * om.size(), cudaMemcpyHostToDevice, st));
            IN_CU(cudaStreamSynchronize(st));   // om leaves scope
        }
        // Y = E Om (n x k, column-major ld n): Y = Ec' Om
        auto left = [&](const float* Mm) -> int {
            IN_BL(cublasSgemm(bl, CUBLAS_OP_T, CUBLAS_OP_N, (int)n, k, (int)m, &onef, E, (int)m, Mm, (int)m, &zerof, Yf,
                              (int)n));
            to_double_kernel<<<grid_of(n * k), 256, 0, st>>>(Yf, Yd, n * k);
            IN_CU(cudaGetLastError());
            int rc = cholqr2(bl, Yd, n, k, Gd, Ri, st, err);
            if (rc) return rc;
            to_float_kernel<<<grid_of(n * k), 256, 0, st>>>(Yd, Yf, n * k);
            IN_CU(cudaGetLastError());
            return GMF_OK;
        };
        // Z = E' Q (m x k, column-major ld m): Z = Ec Q
        auto right = [&](bool orth) -> int {
            IN_BL(cublasSgemm(bl, CUBLAS_OP_N, CUBLAS_OP_N, (int)m, k, (int)n, &onef, E, (int)m, Yf, (int)n, &zerof, Zf,
                              (int)m));
            if (!orth) return GMF_OK;
            to_double_kernel<<<grid_of(m * k), 256, 0, st>>>(Zf, Zd, m * k);
            IN_CU(cudaGetLastError());
            int rc = cholqr2(bl, Zd, m, k, Gd, Ri, st, err);
            if (rc) return rc;
            to_float_kernel<<<grid_of(m * k), 256, 0, st>>>(Zd, Zf, m * k);
            IN_CU(cudaGetLastError());
            return GMF_OK;
        };
        int rc = left(Om);
        for (int it = 0; it < power_iters && rc == GMF_OK; it++) {
            rc = right(true);
            if (rc == GMF_OK) rc = left(Zf);
        }
        if (rc == GMF_OK) rc = right(false);   // Zf = E' Q: the projection B' = (Q' E)'
        if (rc) return rc;
        // host: B B' = Zf' Zf (k x k) = W diag(s^2) W'
        std::vector<float> zf((size_t)m * k);
        IN_CU(cudaMemcpyAsync(zf.data(), Zf, sizeof(float) * zf.size(), cudaMemcpyDeviceToHost, st));
        IN_CU(cudaStreamSynchronize(st));
        Mat BBt((size_t)k * k, 0.0);
        for (int a = 0; a < k; a++)
            for (int b = 0; b <= a; b++) {
                double s = 0.0;
                for (int64_t j = 0; j < m; j++) s += (double)zf[(size_t)a * m + j] * zf[(size_t)b * m + j];
                BBt[a * k + b] = BBt[b * k + a] = s;
            }
        Mat Wv;
        std::vector<double> ev;
        eigh_jacobi(BBt, k, Wv, ev);
        std::vector<int> ord(k);
        for (int a = 0; a < k; a++) ord[a] = a;
        std::sort(ord.begin(), ord.end(), [&](int x, int y) { return ev[x] > ev[y]; });
        std::vector<double> s(d);
        for (int c = 0; c < d; c++) s[c] = sqrt(std::max(ev[ord[c]], 0.0));
        if (sv_out)
            for (int c = 0; c < d; c++) sv_out[c] = s[c];
        // V = Zf W_d diag(s)^(-1/2)  (m x d, host);  U = Q W_d diag(s)^(1/2)  (n x d, device)
        for (int64_t j = 0; j < m; j++)
            for (int c = 0; c < d; c++) {
                double v = 0.0;
                for (int a = 0; a < k; a++) v += (double)zf[(size_t)a * m + j] * Wv[a * k + ord[c]];
                Rh[j * KP + 1 + p + q + c] = s[c] > 0 ? (float)(v / sqrt(s[c])) : 0.f;
            }
        std::vector<float> Wu((size_t)k * d);   // column-major k x d
        for (int c = 0; c < d; c++)
            for (int a = 0; a < k; a++) Wu[(size_t)c * k + a] = (float)(Wv[a * k + ord[c]] * sqrt(s[c]));
        float* Wd = w.alloc<float>((size_t)k * d);
        float* Ud = w.alloc<float>((size_t)n * d);
        if (!Wd || !Ud) {
            *err = "no device memory for the scores";
            return GMF_ERR_OOM;
        }
        IN_CU(cudaMemcpyAsync(Wd, Wu.data(), sizeof(float) * Wu.size(), cudaMemcpyHostToDevice, st));
        // U' (d x n, column-major = row-major n x d) = Wd' Q'
        IN_BL(cublasSgemm(bl, CUBLAS_OP_T, CUBLAS_OP_T, d, (int)n, k, &onef, Wd, k, Yf, (int)n, &zerof, Ud, d));
        IN_CU(cudaMemcpy2DAsync(h->L + 1 + p + q, sizeof(float) * KP, Ud, sizeof(float) * d, sizeof(float) * d, n,
                                cudaMemcpyDeviceToDevice, st));
        IN_CU(cudaMemcpyAsync(h->R, Rh.data(), sizeof(float) * Rh.size(), cudaMemcpyHostToDevice, st));
        IN_CU(cudaStreamSynchronize(st));   // Wu, Rh leave scope after the copies
    } else {
        IN_CU(cudaStreamSynchronize(st));
    }
    return GMF_OK;
}

// Column GLMs for V given U, B and Gamma (the last step of Sec. 4.1): for each
// gene, Fisher scoring of f_j(v) = 0.5 sum_i w_ij D(y_ij, mu_ij) + 0.5 lam_V |v|^2
// with the step control of the per-cell projection. Per pass, over chunks of
// rows: eta = L R' (SGEMM), the derivatives and deviances (glm_col_kernel),
// G += U' (w Ddot) and H += KR(U)' (w Dddot) (SGEMMs; H packed by pairs); then
// on the host, per gene in FP64: accept or halve, and the Fisher step
// (H_j + lam I)^-1 (G_j - lam v_j) by Cholesky. obj_out: sum_j f_j at the result.
int gmf_loadings_run(gmf_model* h, int n_steps, double* obj_out, cudaStream_t st, std::string* err) {
    const int64_t n = h->n, m = h->m;
    const int p = h->p, q = h->q, d = h->d, KP = h->KP, K = h->K;
    const int c0 = 1 + p + q, P = d * (d + 1) / 2;
    const double lam = h->cfg.lambda[3];
    const int64_t rows = std::min<int64_t>(n, std::max<int64_t>(256, (int64_t)(1 << 22) / m));
    const int SEG = 32, seg_rows = (int)((rows + SEG - 1) / SEG);
    Work w{{}, st};
    float* E = w.alloc<float>((size_t)rows * m);
    float* DD = w.alloc<float>((size_t)rows * m);
    float* KR = w.alloc<float>((size_t)rows * std::max(P, 1));
    float* G = w.alloc<float>((size_t)std::max(d, 1) * m);
    float* H = w.alloc<float>((size_t)std::max(P, 1) * m);
    double* devpart = w.alloc<double>((size_t)SEG * m);
    if (!E || !DD || !KR || !G || !H || !devpart) {
        *err = "no device memory for the chunk buffers";
        return GMF_ERR_OOM;
    }
    cublasHandle_t bl = nullptr;
    if (cublasCreate(&bl) != CUBLAS_STATUS_SUCCESS) {
        *err = "cublasCreate failed";
        return GMF_ERR_CUDA;
    }
    struct BlGuard {
        cublasHandle_t b;
        ~BlGuard() { cublasDestroy(b); }
    } guard{bl};
    IN_BL(cublasSetStream(bl, st));
    IN_BL(cublasSetMathMode(bl, CUBLAS_PEDANTIC_MATH));   // FP32 products, no TF32
    const float onef = 1.f, zerof = 0.f;

    std::vector<float> Rh((size_t)m * KP);
    IN_CU(cudaMemcpyAsync(Rh.data(), h->R, sizeof(float) * Rh.size(), cudaMemcpyDeviceToHost, st));
    IN_CU(cudaStreamSynchronize(st));
    Mat V((size_t)m * d), best((size_t)m * d), step((size_t)m * d, 0.0);
    for (int64_t j = 0; j < m; j++)
        for (int c = 0; c < d; c++) V[j * d + c] = Rh[j * KP + c0 + c];
    best = V;
    std::vector<double> f_best(m, INFINITY);
    std::vector<float> Gh((size_t)d * m), Hh((size_t)P * m);
    std::vector<double> devh((size_t)SEG * m);
    const int nb = h->cfg.family == GMF_NEGBIN;
    for (int k = 0; k <= n_steps; k++) {   // pass k evaluates V; passes 0 .. n_steps-1 also step
        IN_CU(cudaMemsetAsync(devpart, 0, sizeof(double) * SEG * m, st));
        for (int64_t r0 = 0; r0 < n; r0 += rows) {
            const int nr = (int)std::min<int64_t>(rows, n - r0);
            const float beta = r0 == 0 ? 0.f : 1.f;
            // eta (row-major nr x m) = L_chunk R'
            IN_BL(cublasSgemm(bl, CUBLAS_OP_T, CUBLAS_OP_N, (int)m, nr, K, &onef, h->R, KP, h->L + r0 * KP, KP, &zerof,
                              E, (int)m));
            glm_col_kernel<<<dim3((unsigned)((m + 255) / 256), (unsigned)((nr + seg_rows - 1) / seg_rows)), 256, 0,
                             st>>>(h->Yp, h->y16, h->Wp, E, DD, devpart, r0, nr, m, seg_rows, h->alpha,
                                   h->cfg.alpha_mode == 2 ? h->alpha_col : nullptr, nb, (float)h->cfg.eta_clamp);
            IN_CU(cudaGetLastError());
            if (d > 0) {
                // G (d x m, column-major) += U_chunk' (w Ddot)
                IN_BL(cublasSgemm(bl, CUBLAS_OP_N, CUBLAS_OP_T, d, (int)m, nr, &onef, h->L + r0 * KP + c0, KP, E,
                                  (int)m, &beta, G, d));
                kr_kernel<<<grid_of((int64_t)nr * P), 256, 0, st>>>(h->L, KP, c0, r0, nr, d, P, KR);
                IN_CU(cudaGetLastError());
                // H (P x m, column-major) += KR(U_chunk)' (w Dddot)
                IN_BL(cublasSgemm(bl, CUBLAS_OP_N, CUBLAS_OP_T, P, (int)m, nr, &onef, KR, P, DD, (int)m, &beta, H, P));
            }
        }
        IN_CU(cudaMemcpyAsync(devh.data(), devpart, sizeof(double) * devh.size(), cudaMemcpyDeviceToHost, st));
        if (d > 0) {
            IN_CU(cudaMemcpyAsync(Gh.data(), G, sizeof(float) * Gh.size(), cudaMemcpyDeviceToHost, st));
            IN_CU(cudaMemcpyAsync(Hh.data(), H, sizeof(float) * Hh.size(), cudaMemcpyDeviceToHost, st));
        }
        IN_CU(cudaStreamSynchronize(st));
        for (int64_t j = 0; j < m; j++) {
            double dev = 0.0, vv = 0.0;
            for (int s = 0; s < SEG; s++) dev += devh[(size_t)s * m + j];
            for (int c = 0; c < d; c++) vv += V[j * d + c] * V[j * d + c];
            const double f = 0.5 * dev + 0.5 * lam * vv;
            double* vj = &V[j * d];
            if (k == 0 || f <= f_best[j] + 1e-5 * (1.0 + fabs(f_best[j]))) {
                f_best[j] = f;
                for (int c = 0; c < d; c++) best[j * d + c] = vj[c];
                if (k < n_steps && d > 0) {
                    Mat F((size_t)d * d), g((size_t)d);
                    const float* Hj = &Hh[(size_t)j * P];
                    int pr = 0;
                    for (int a = 0; a < d; a++)
                        for (int b = a; b < d; b++, pr++) F[a * d + b] = F[b * d + a] = (double)Hj[pr];
                    for (int a = 0; a < d; a++) {
                        F[a * d + a] += lam;
                        g[a] = (double)Gh[(size_t)j * d + a] - lam * best[j * d + a];
                    }
                    if (spd_solve(F, d, g, 1))
                        for (int c = 0; c < d; c++) step[j * d + c] = g[c];
                    else
                        for (int c = 0; c < d; c++) step[j * d + c] = 0.0;
                    for (int c = 0; c < d; c++) vj[c] = best[j * d + c] + step[j * d + c];
                }
            } else {
                for (int c = 0; c < d; c++) {
                    step[j * d + c] *= 0.5;
                    vj[c] = best[j * d + c] + step[j * d + c];
                }
            }
        }
        const Mat& up = k == n_steps ? best : V;
        for (int64_t j = 0; j < m; j++)
            for (int c = 0; c < d; c++) Rh[j * KP + c0 + c] = (float)up[j * d + c];
        IN_CU(cudaMemcpyAsync(h->R, Rh.data(), sizeof(float) * Rh.size(), cudaMemcpyHostToDevice, st));
    }
    IN_CU(cudaStreamSynchronize(st));
    if (obj_out) {
        double t = 0.0;
        for (int64_t j = 0; j < m; j++) t += f_best[j];
        *obj_out = t;
    }
    return GMF_OK;
}
