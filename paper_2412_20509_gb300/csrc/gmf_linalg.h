// Host FP64 dense linear algebra for small (k x k) problems: Cholesky, SPD
// solves, triangular inverses, one-sided Jacobi SVD, cyclic Jacobi symmetric
// eigen-decomposition and Householder QR. Used by Algorithm 2
// (gmf_orthogonalize) and by the initialisation of Sec. 4.1.
#pragma once

#include <math.h>

#include <algorithm>
#include <vector>

namespace gmfla {

// ------------------------------------------------------------------ host d x d linear algebra (FP64)
using Mat = std::vector<double>;  // row-major

// Lower Cholesky A = C C'; false if A is not positive definite.
inline bool cholesky(const Mat& A, int k, Mat& C) {
    C.assign((size_t)k * k, 0.0);
    for (int i = 0; i < k; i++) {
        for (int j = 0; j <= i; j++) {
            double s = A[i * k + j];
            for (int t = 0; t < j; t++) s -= C[i * k + t] * C[j * k + t];
            if (i == j) {
                if (!(s > 0.0)) return false;
                C[i * k + i] = sqrt(s);
            } else {
                C[i * k + j] = s / C[j * k + j];
            }
        }
    }
    return true;
}
// Solve A X = B for SPD A (k x k), B k x r (in place).
inline bool spd_solve(const Mat& A, int k, Mat& B, int r) {
    Mat C;
    if (!cholesky(A, k, C)) return false;
    for (int col = 0; col < r; col++) {
        for (int i = 0; i < k; i++) {
            double s = B[i * r + col];
            for (int t = 0; t < i; t++) s -= C[i * k + t] * B[t * r + col];
            B[i * r + col] = s / C[i * k + i];
        }
        for (int i = k - 1; i >= 0; i--) {
            double s = B[i * r + col];
            for (int t = i + 1; t < k; t++) s -= C[t * k + i] * B[t * r + col];
            B[i * r + col] = s / C[i * k + i];
        }
    }
    return true;
}
inline Mat matmul(const Mat& A, const Mat& B, int a, int b, int c) {
    Mat C((size_t)a * c, 0.0);
    for (int i = 0; i < a; i++)
        for (int t = 0; t < b; t++)
            for (int j = 0; j < c; j++) C[i * c + j] += A[i * b + t] * B[t * c + j];
    return C;
}
inline Mat transpose(const Mat& A, int a, int b) {
    Mat T((size_t)a * b);
    for (int i = 0; i < a; i++)
        for (int j = 0; j < b; j++) T[j * a + i] = A[i * b + j];
    return T;
}
// Inverse of an upper-triangular matrix.
inline Mat upper_inverse(const Mat& R, int k) {
    Mat X((size_t)k * k, 0.0);
    for (int j = 0; j < k; j++) {
        X[j * k + j] = 1.0 / R[j * k + j];
        for (int i = j - 1; i >= 0; i--) {
            double s = 0.0;
            for (int t = i + 1; t <= j; t++) s += R[i * k + t] * X[t * k + j];
            X[i * k + j] = -s / R[i * k + i];
        }
    }
    return X;
}
// One-sided Jacobi SVD of a square A = P diag(S) Q', S decreasing.
inline void svd_jacobi(const Mat& A, int k, Mat& P, std::vector<double>& S, Mat& Q) {
    Mat W = A;  // columns rotated towards orthogonality: W = A Q
    Q.assign((size_t)k * k, 0.0);
    for (int i = 0; i < k; i++) Q[i * k + i] = 1.0;
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = 0.0;
        for (int a = 0; a < k - 1; a++)
            for (int b = a + 1; b < k; b++) {
                double aa = 0, bb = 0, ab = 0;
                for (int i = 0; i < k; i++) {
                    aa += W[i * k + a] * W[i * k + a];
                    bb += W[i * k + b] * W[i * k + b];
                    ab += W[i * k + a] * W[i * k + b];
                }
                if (fabs(ab) <= 1e-15 * sqrt(aa * bb) || ab == 0.0) continue;
                off = std::max(off, fabs(ab) / sqrt(aa * bb));
                const double zeta = (bb - aa) / (2.0 * ab);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                for (int i = 0; i < k; i++) {
                    const double wa = W[i * k + a], wb = W[i * k + b];
                    W[i * k + a] = c * wa - s * wb;
                    W[i * k + b] = s * wa + c * wb;
                    const double qa = Q[i * k + a], qb = Q[i * k + b];
                    Q[i * k + a] = c * qa - s * qb;
                    Q[i * k + b] = s * qa + c * qb;
                }
            }
        if (off < 1e-15) break;
    }
    S.assign(k, 0.0);
    for (int j = 0; j < k; j++) {
        double s = 0;
        for (int i = 0; i < k; i++) s += W[i * k + j] * W[i * k + j];
        S[j] = sqrt(s);
    }
    std::vector<int> ord(k);
    for (int j = 0; j < k; j++) ord[j] = j;
    std::sort(ord.begin(), ord.end(), [&](int x, int y) { return S[x] > S[y]; });
    Mat P2((size_t)k * k), Q2((size_t)k * k);
    std::vector<double> S2(k);
    for (int jj = 0; jj < k; jj++) {
        const int j = ord[jj];
        S2[jj] = S[j];
        for (int i = 0; i < k; i++) {
            P2[i * k + jj] = S[j] > 0 ? W[i * k + j] / S[j] : 0.0;
            Q2[i * k + jj] = Q[i * k + j];
        }
    }
    P = P2;
    Q = Q2;
    S = S2;
}
// Symmetric eigen-decomposition by cyclic Jacobi: A = E diag(w) E'.
inline void eigh_jacobi(Mat A, int k, Mat& E, std::vector<double>& w) {
    E.assign((size_t)k * k, 0.0);
    for (int i = 0; i < k; i++) E[i * k + i] = 1.0;
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0;
        for (int a = 0; a < k; a++)
            for (int b = a + 1; b < k; b++) off += A[a * k + b] * A[a * k + b];
        if (off < 1e-30) break;
        for (int a = 0; a < k - 1; a++)
            for (int b = a + 1; b < k; b++) {
                const double apq = A[a * k + b];
                if (fabs(apq) < 1e-300) continue;
                const double theta = (A[b * k + b] - A[a * k + a]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int i = 0; i < k; i++) {
                    const double ia = A[i * k + a], ib = A[i * k + b];
                    A[i * k + a] = c * ia - s * ib;
                    A[i * k + b] = s * ia + c * ib;
                }
                for (int i = 0; i < k; i++) {
                    const double ai = A[a * k + i], bi = A[b * k + i];
                    A[a * k + i] = c * ai - s * bi;
                    A[b * k + i] = s * ai + c * bi;
                }
                for (int i = 0; i < k; i++) {
                    const double ea = E[i * k + a], eb = E[i * k + b];
                    E[i * k + a] = c * ea - s * eb;
                    E[i * k + b] = s * ea + c * eb;
                }
            }
    }
    w.assign(k, 0.0);
    for (int i = 0; i < k; i++) w[i] = A[i * k + i];
}
// Householder QR of a square A: A = Q R.
inline void qr_householder(const Mat& A, int k, Mat& Q) {
    Mat R = A;
    Q.assign((size_t)k * k, 0.0);
    for (int i = 0; i < k; i++) Q[i * k + i] = 1.0;
    for (int j = 0; j < k - 1; j++) {
        double norm = 0;
        for (int i = j; i < k; i++) norm += R[i * k + j] * R[i * k + j];
        norm = sqrt(norm);
        if (norm == 0.0) continue;
        std::vector<double> v(k, 0.0);
        const double alpha = R[j * k + j] > 0 ? -norm : norm;
        for (int i = j; i < k; i++) v[i] = R[i * k + j];
        v[j] -= alpha;
        double vn = 0;
        for (int i = j; i < k; i++) vn += v[i] * v[i];
        if (vn == 0.0) continue;
        for (int c = 0; c < k; c++) {  // R <- (I - 2vv'/v'v) R
            double s = 0;
            for (int i = j; i < k; i++) s += v[i] * R[i * k + c];
            s = 2.0 * s / vn;
            for (int i = j; i < k; i++) R[i * k + c] -= s * v[i];
        }
        for (int r = 0; r < k; r++) {  // Q <- Q (I - 2vv'/v'v)
            double s = 0;
            for (int i = j; i < k; i++) s += Q[r * k + i] * v[i];
            s = 2.0 * s / vn;
            for (int i = j; i < k; i++) Q[r * k + i] -= s * v[i];
        }
    }
}

}  // namespace gmfla
