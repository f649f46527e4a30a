// Algorithm 2 (identifiability projection and orthogonalisation, Sec. 2.1 and
// its appendix) in FP64 on the device:
//   1. D_G = (X'X)^-1 X' Gamma;  Gamma -= X D_G;  B += Z D_G'
//   2. D_U = (X'X)^-1 X' U;      U -= X D_U;      B += V D_U'
//   3. D_V = (Z'Z)^-1 Z' V;      V -= Z D_V;      Gamma += U D_V'   (with the new U)
//   4. (B1) U V' = (U Ru^-1 P) S (V Rv^-1 Q)' with U'U = Ru'Ru, V'V = Rv'Rv and
//      Ru Rv' = P S Q' (a d x d SVD): U <- U Ru^-1 P S, V <- V Rv^-1 Q;
//      (B2) U <- U Ru^-1 P, V <- V Rv^-1 Q S; sign rule on V (B1) or U (B2);
//      (B3) whiten by S = cov(U): U <- U S^-1/2, V <- V S^1/2, then Q from the QR
//      of the first d rows of V' so that V Q is lower triangular, and
//      D = diag(sign(diag(V Q))).
// The tall reductions (X'[X,Gamma,U], Z'[Z,V], U'U, 1'U, V'V) and the row /
// column updates run on the device in FP64 with fixed-order block partials;
// the d x d factorizations run on the host in FP64.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "gmf_internal.cuh"
#include "gmf_linalg.h"

namespace {

constexpr int NT = 256;
constexpr int GRAM_ROWS = 2048;   // rows per block of a Gram reduction

// Wr = [X | Gamma | U | 1] (n x cr, cr = p+q+d+1) and Wc = [Z | V | B] (m x cc) from L and R.
__global__ void pack_rows(const float* L, int KP, int p, int q, int d, int64_t n, double* Wr) {
    const int cr = p + q + d + 1;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * cr; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / cr;
        const int c = (int)(e - i * cr);
        Wr[e] = c < p + q + d ? (double)L[i * KP + 1 + c] : 1.0;
    }
}
__global__ void pack_cols(const float* R, int KP, int p, int q, int d, int64_t m, double* Wc) {
    const int cc = q + d + p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m * cc; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / cc;
        const int c = (int)(e - j * cc);
        // R row: [1 | B (p) | Z (q) | V (d)]  ->  Wc row: [Z | V | B]
        const int src = c < q ? 1 + p + c : (c < q + d ? 1 + p + c : 1 + (c - q - d));
        Wc[e] = (double)R[j * KP + src];
    }
}

// Partial A'B over a block of rows: A = W[:, a0:a0+na], B = W[:, b0:b0+nb].
__global__ void gram_partial(const double* W, int ld, int64_t rows, int a0, int na, int b0, int nb, double* part) {
    const int64_t r0 = (int64_t)blockIdx.x * GRAM_ROWS;
    const int64_t r1 = min(rows, r0 + GRAM_ROWS);
    const int E = na * nb;
    for (int e = threadIdx.x; e < E; e += NT) {
        const int x = e / nb, y = e - x * nb;
        double s = 0.0;
        for (int64_t i = r0; i < r1; i++) s += W[i * ld + a0 + x] * W[i * ld + b0 + y];
        part[(int64_t)blockIdx.x * E + e] = s;
    }
}
__global__ void gram_sum(const double* part, int blocks, int E, double* out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < blocks; b++) s += part[(int64_t)b * E + e];
        out[e] = s;
    }
}

// Steps 1-3 on the row side: u' = u - D_U' x;  gamma' = gamma - D_G' x + D_V u'.
// M: D_G (p x q) | D_U (p x d) | D_V (q x d), row-major, contiguous.
__global__ void project_rows(double* Wr, int64_t n, int p, int q, int d, const double* M) {
    const int cr = p + q + d + 1;
    const double* DG = M;
    const double* DU = DG + p * q;
    const double* DV = DU + p * d;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double* w = Wr + i * cr;
        const double* x = w;
        double* g = w + p;
        double* u = w + p + q;
        for (int c = 0; c < d; c++) {
            double s = u[c];
            for (int a = 0; a < p; a++) s -= DU[a * d + c] * x[a];
            u[c] = s;
        }
        for (int b = 0; b < q; b++) {
            double s = g[b];
            for (int a = 0; a < p; a++) s -= DG[a * q + b] * x[a];
            for (int c = 0; c < d; c++) s += DV[b * d + c] * u[c];
            g[b] = s;
        }
    }
}
// Column side: beta' = beta + D_G z + D_U v;  v' = v - D_V' z.
__global__ void project_cols(double* Wc, int64_t m, int p, int q, int d, const double* M) {
    const int cc = q + d + p;
    const double* DG = M;
    const double* DU = DG + p * q;
    const double* DV = DU + p * d;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        double* w = Wc + j * cc;
        const double* z = w;
        double* v = w + q;
        double* b = w + q + d;
        for (int a = 0; a < p; a++) {
            double s = b[a];
            for (int c = 0; c < q; c++) s += DG[a * q + c] * z[c];
            for (int c = 0; c < d; c++) s += DU[a * d + c] * v[c];
            b[a] = s;
        }
        for (int c = 0; c < d; c++) {
            double s = v[c];
            for (int e = 0; e < q; e++) s -= DV[e * d + c] * z[e];
            v[c] = s;
        }
    }
}

// Rotation and write-back: U <- U Tu (rows), Gamma -> L; V <- V Tv, B -> R (FP32 storage).
__global__ void finish_rows(const double* Wr, int64_t n, int p, int q, int d, const double* Tu, float* L, int KP) {
    const int cr = p + q + d + 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double* w = Wr + i * cr;
        float* l = L + i * KP;
        for (int b = 0; b < q; b++) l[1 + p + b] = (float)w[p + b];
        for (int c = 0; c < d; c++) {
            double s = 0.0;
            for (int e = 0; e < d; e++) s += w[p + q + e] * Tu[e * d + c];
            l[1 + p + q + c] = (float)s;
        }
    }
}
__global__ void finish_cols(const double* Wc, int64_t m, int p, int q, int d, const double* Tv, float* R, int KP) {
    const int cc = q + d + p;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const double* w = Wc + j * cc;
        float* r = R + j * KP;
        for (int a = 0; a < p; a++) r[1 + a] = (float)w[q + d + a];
        for (int c = 0; c < d; c++) {
            double s = 0.0;
            for (int e = 0; e < d; e++) s += w[q + e] * Tv[e * d + c];
            r[1 + p + q + c] = (float)s;
        }
    }
}

using namespace gmfla;


struct Dev {
    std::vector<void*> ptrs;
    ~Dev() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <typename T>
    T* alloc(size_t n) {
        void* p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return (T*)p;
    }
};

int grid_for(int64_t n) { return (int)std::min<int64_t>((n + NT - 1) / NT, 4096); }

// A'B of columns of W on the device, result to host (row-major na x nb).
bool gram(const double* W, int ld, int64_t rows, int a0, int na, int b0, int nb, double* part, double* dout,
          Mat& out, cudaStream_t st) {
    const int blocks = (int)((rows + GRAM_ROWS - 1) / GRAM_ROWS);
    gram_partial<<<blocks, NT, 0, st>>>(W, ld, rows, a0, na, b0, nb, part);
    gram_sum<<<std::max(1, (na * nb + NT - 1) / NT), NT, 0, st>>>(part, blocks, na * nb, dout);
    out.assign((size_t)na * nb, 0.0);
    return cudaMemcpyAsync(out.data(), dout, sizeof(double) * na * nb, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
           cudaStreamSynchronize(st) == cudaSuccess;
}

}  // namespace

int gmf_orth_run(gmf_model* h, int mode, cudaStream_t st, std::string* err) {
    const int p = h->p, q = h->q, d = h->d;
    const int64_t n = h->n, m = h->m;
    const int cr = p + q + d + 1, cc = q + d + p;
    if (p < 1 || q < 1) {
        *err = "Algorithm 2 needs at least one column in X and in Z";
        return GMF_ERR_ARG;
    }
    Dev dv;
    double* Wr = dv.alloc<double>((size_t)n * cr);
    double* Wc = dv.alloc<double>((size_t)m * cc);
    const int64_t maxrows = std::max(n, m);
    const int maxE = std::max(std::max(p * cr, q * cc), d * d + d);
    double* part = dv.alloc<double>((size_t)((maxrows + GRAM_ROWS - 1) / GRAM_ROWS) * maxE);
    double* dout = dv.alloc<double>((size_t)maxE);
    double* dM = dv.alloc<double>((size_t)(p * q + p * d + q * d + 2 * d * d + 2));
    if (!Wr || !Wc || !part || !dout || !dM) {
        *err = "device allocation failed";
        return GMF_ERR_OOM;
    }
    pack_rows<<<grid_for(n * cr), NT, 0, st>>>(h->L, h->KP, p, q, d, n, Wr);
    pack_cols<<<grid_for(m * cc), NT, 0, st>>>(h->R, h->KP, p, q, d, m, Wc);

    // Steps 1-3: X'[X, Gamma, U] and Z'[Z, V] (V is unchanged by steps 1-2).
    Mat XW, ZW;
    if (!gram(Wr, cr, n, 0, p, 0, cr, part, dout, XW, st) || !gram(Wc, cc, m, 0, q, 0, cc, part, dout, ZW, st)) {
        *err = "Gram reduction failed";
        return GMF_ERR_CUDA;
    }
    Mat XtX((size_t)p * p), ZtZ((size_t)q * q), DG((size_t)p * q), DU((size_t)p * d), DV((size_t)q * d);
    for (int a = 0; a < p; a++) {
        for (int b = 0; b < p; b++) XtX[a * p + b] = XW[a * cr + b];
        for (int b = 0; b < q; b++) DG[a * q + b] = XW[a * cr + p + b];
        for (int c = 0; c < d; c++) DU[a * d + c] = XW[a * cr + p + q + c];
    }
    for (int a = 0; a < q; a++) {
        for (int b = 0; b < q; b++) ZtZ[a * q + b] = ZW[a * cc + b];
        for (int c = 0; c < d; c++) DV[a * d + c] = ZW[a * cc + q + c];
    }
    if (!spd_solve(XtX, p, DG, q) || !spd_solve(XtX, p, DU, d) || !spd_solve(ZtZ, q, DV, d)) {
        *err = "X'X or Z'Z is singular (covariates must have full column rank)";
        return GMF_ERR_STATE;
    }
    {
        Mat M;
        M.insert(M.end(), DG.begin(), DG.end());
        M.insert(M.end(), DU.begin(), DU.end());
        M.insert(M.end(), DV.begin(), DV.end());
        cudaMemcpyAsync(dM, M.data(), sizeof(double) * M.size(), cudaMemcpyHostToDevice, st);
        project_rows<<<grid_for(n), NT, 0, st>>>(Wr, n, p, q, d, dM);
        project_cols<<<grid_for(m), NT, 0, st>>>(Wc, m, p, q, d, dM);
    }
    Mat Tu((size_t)d * d, 0.0), Tv((size_t)d * d, 0.0);
    if (d > 0) {
        Mat Gu, Gv, su;
        if (!gram(Wr, cr, n, p + q, d, p + q, d, part, dout, Gu, st) ||
            !gram(Wr, cr, n, p + q + d, 1, p + q, d, part, dout, su, st) ||
            !gram(Wc, cc, m, q, d, q, d, part, dout, Gv, st)) {
            *err = "Gram reduction failed";
            return GMF_ERR_CUDA;
        }
        // first rows of V (and U) in the caller's original order, after the projection
        std::vector<int32_t> cinv(m), rinv(n);
        for (int64_t j = 0; j < m; j++) cinv[h->h_cperm[j]] = (int32_t)j;
        for (int64_t i = 0; i < n; i++) rinv[h->h_rperm[i]] = (int32_t)i;
        auto fetch_rows = [&](const double* W, int ld, int off, const std::vector<int32_t>& inv, int64_t count,
                              Mat& out) {
            out.assign((size_t)count * d, 0.0);
            std::vector<double> row(ld);
            for (int64_t r = 0; r < count; r++) {
                cudaMemcpyAsync(row.data(), W + (int64_t)inv[r] * ld, sizeof(double) * ld, cudaMemcpyDeviceToHost, st);
                cudaStreamSynchronize(st);
                for (int c = 0; c < d; c++) out[r * d + c] = row[off + c];
            }
        };
        auto sign_fix = [&](const Mat& rows, int64_t count, const Mat& T, Mat& T1, Mat& T2) {
            // first entry of magnitude > 1e-12 of each column of rows*T made positive (applied to T1 and T2)
            const Mat Y = matmul(rows, T, (int)count, d, d);
            for (int c = 0; c < d; c++) {
                double sgn = 1.0;
                for (int64_t r = 0; r < count; r++)
                    if (fabs(Y[r * d + c]) > 1e-12) {
                        sgn = Y[r * d + c] < 0 ? -1.0 : 1.0;
                        break;
                    }
                for (int e = 0; e < d; e++) {
                    T1[e * d + c] *= sgn;
                    T2[e * d + c] *= sgn;
                }
            }
        };
        if (mode == GMF_ORTH_B1 || mode == GMF_ORTH_B2) {
            Mat Cu, Cv;
            if (!cholesky(Gu, d, Cu) || !cholesky(Gv, d, Cv)) {
                *err = "U or V is rank deficient";
                return GMF_ERR_STATE;
            }
            const Mat Ru = transpose(Cu, d, d), Rv = transpose(Cv, d, d);  // U'U = Ru'Ru
            Mat P, Q;
            std::vector<double> S;
            svd_jacobi(matmul(Ru, transpose(Rv, d, d), d, d, d), d, P, S, Q);
            Mat Su((size_t)d * d, 0.0), Sv((size_t)d * d, 0.0);
            for (int c = 0; c < d; c++) {
                Su[c * d + c] = mode == GMF_ORTH_B1 ? S[c] : 1.0;
                Sv[c * d + c] = mode == GMF_ORTH_B1 ? 1.0 : S[c];
            }
            Tu = matmul(matmul(upper_inverse(Ru, d), P, d, d, d), Su, d, d, d);
            Tv = matmul(matmul(upper_inverse(Rv, d), Q, d, d, d), Sv, d, d, d);
            const int64_t cnt = std::min<int64_t>(mode == GMF_ORTH_B1 ? m : n, 8);
            Mat rows;
            if (mode == GMF_ORTH_B1) {
                fetch_rows(Wc, cc, q, cinv, cnt, rows);
                sign_fix(rows, cnt, Tv, Tu, Tv);
            } else {
                fetch_rows(Wr, cr, p + q, rinv, cnt, rows);
                sign_fix(rows, cnt, Tu, Tu, Tv);
            }
        } else {
            // (B3): S = (U'U - (1/n) U'1 1'U) / n
            Mat Sm((size_t)d * d);
            for (int a = 0; a < d; a++)
                for (int b = 0; b < d; b++) Sm[a * d + b] = (Gu[a * d + b] - su[a] * su[b] / (double)n) / (double)n;
            Mat E;
            std::vector<double> wv;
            eigh_jacobi(Sm, d, E, wv);
            Mat Sh((size_t)d * d, 0.0), Smh((size_t)d * d, 0.0);
            for (int a = 0; a < d; a++)
                for (int b = 0; b < d; b++) {
                    double s1 = 0, s2 = 0;
                    for (int c = 0; c < d; c++) {
                        if (!(wv[c] > 0)) continue;
                        s1 += E[a * d + c] * sqrt(wv[c]) * E[b * d + c];
                        s2 += E[a * d + c] / sqrt(wv[c]) * E[b * d + c];
                    }
                    Sh[a * d + b] = s1;
                    Smh[a * d + b] = s2;
                }
            if (m < d) {
                *err = "(B3) needs m >= d";
                return GMF_ERR_STATE;
            }
            Mat V1;
            fetch_rows(Wc, cc, q, cinv, d, V1);
            const Mat V1w = matmul(V1, Sh, d, d, d);  // whitened first d rows
            Mat Q;
            qr_householder(transpose(V1w, d, d), d, Q);  // V1w' = Q R  ->  V1w Q = R' (lower triangular)
            Tu = matmul(Smh, Q, d, d, d);
            Tv = matmul(Sh, Q, d, d, d);
            const Mat Vt = matmul(V1, Tv, d, d, d);
            for (int c = 0; c < d; c++) {
                const double sgn = Vt[c * d + c] < 0 ? -1.0 : 1.0;
                for (int e = 0; e < d; e++) {
                    Tu[e * d + c] *= sgn;
                    Tv[e * d + c] *= sgn;
                }
            }
        }
        cudaMemcpyAsync(dM, Tu.data(), sizeof(double) * d * d, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(dM + d * d, Tv.data(), sizeof(double) * d * d, cudaMemcpyHostToDevice, st);
    }
    finish_rows<<<grid_for(n), NT, 0, st>>>(Wr, n, p, q, d, dM, h->L, h->KP);
    finish_cols<<<grid_for(m), NT, 0, st>>>(Wc, m, p, q, d, dM + d * d, h->R, h->KP);
    // the smoothed derivatives and visit counters refer to the old basis
    cudaMemsetAsync(h->GbR, 0, sizeof(float) * n * h->fr, st);
    cudaMemsetAsync(h->HbR, 0, sizeof(float) * n * h->fr, st);
    cudaMemsetAsync(h->GbC, 0, sizeof(float) * m * h->fc, st);
    cudaMemsetAsync(h->HbC, 0, sizeof(float) * m * h->fc, st);
    cudaMemsetAsync(h->cntR, 0, sizeof(int) * n, st);
    cudaMemsetAsync(h->cntC, 0, sizeof(int) * m, st);
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        *err = cudaGetErrorString(e);
        return GMF_ERR_CUDA;
    }
    return GMF_OK;
}
