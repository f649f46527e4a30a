/*
 * gmf_oracle.c -- plain, single-threaded FP64 reference of block-wise adaptive
 * SGD for generalized matrix factorization (arXiv 2412.20509).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code, header or table with the
 * CUDA library and is written directly from the paper:
 *
 *   model ........... Sec. 2, eq. 1-3 (linear predictor with an offset, App. B)
 *   objective ....... eq. 6 (penalised negative log-likelihood)
 *   derivatives ..... Sec. 3 (D-dot, D-ddot with the Fisher weight alpha(mu)=1)
 *   block estimators  eq. 15 and App. B (covariate extension)
 *   update .......... eq. 11, 12, 14 (EMA, bias correction, local step)
 *   loop ............ Algorithm 1
 *   NB shape ........ App. B, stochastic moment estimator
 *   dispersion ...... App. B, smoothed stochastic Pearson estimator
 *   deviance ........ Table S1 and App. B (NB)
 *
 * Readings of points the paper leaves open (each is also a config field):
 *   - Sign: the block gradient is the derivative of the penalised NEGATIVE
 *     log-likelihood, G = -(m/|J|) sum_j Ddot_ij R_jc + lambda theta, where
 *     Ddot = w (y - mu) / (phi nu(mu) g'(mu)) as printed in Sec. 3; the
 *     curvature H = (m/|J|) sum_j Dddot_ij R_jc^2 + lambda + damping > 0.
 *   - The scale factors use the actual chunk sizes m/|J| and n/|I|.
 *   - Both sides of a block use the parameters from before the block's step.
 *   - The global step t counts blocks from 1; rho_t = k0/(1+k0 k1 t)^tau.
 *   - bias_corr 0: c_t = (1-a2^t)/(1-a1^t) as printed (global t);
 *     bias_corr 1: c = (1-(1-a2)^k)/(1-(1-a1)^k), k = visits of that row/column.
 *   - Epoch: with r row chunks and s column chunks (r >= s), sweep w visits the
 *     s blocks (I_{(sigma_w + k) mod r}, J_k), k = 0..s-1, so every block is
 *     visited once per epoch.  If r < s the roles are swapped.  The blocks of
 *     a sweep are processed here one after the other, in order k.
 *   - NB shape: moment sums pooled over one sweep; the smoothed shape is
 *     updated once at the end of the sweep with rho of the sweep's first block;
 *     skipped when the denominator is not positive.
 *   - eta is clamped to [-eta_clamp, eta_clamp] before the inverse link.
 *   - Families (Table S1): Poisson, NB, Bernoulli with phi = 1; Gaussian,
 *     Gamma and inverse Gaussian with a dispersion phi.  Links: log for the
 *     count families (Sec. 2), identity for the Gaussian and logit for the
 *     Bernoulli (their canonical links), log for the Gamma and the inverse
 *     Gaussian (their canonical links 1/mu and 1/mu^2 leave mu > 0 to the
 *     optimiser; the log link keeps it, and Sec. 2 allows any link).  The
 *     family's scalar parameter is held in one slot: the NB shape, or phi.
 *   - phi (alpha_mode 1 for the three families with a dispersion): the
 *     Pearson sum w (y - mu)^2 / nu(mu) pooled over one sweep, scaled by
 *     nm / (entries of the sweep) and divided by the model's residual degrees
 *     of freedom N = nm - mp - nq - (n + m) d - 1, then smoothed as the NB
 *     shape is (rho of the sweep's first block, floored at eps); skipped when
 *     N <= 0.  Missing entries are left out of the sum and of the count.
 *   - eta is clamped for every family, the identity link included.
 *   - Continuous responses are float32 (y_dtype 2); NaN marks a missing one.
 *   - Per-gene NB shapes (alpha_mode 2): gene j has its own fixed shape alpha_j
 *     (the model of App. B with the shape made column-specific, as the data
 *     laws draw it); the derivatives and deviance of entry (i, j) use alpha_j.
 *   - Missing entries (missing = 1): a count equal to the sentinel (-1 for
 *     int32 counts, 65535 for uint16) is not observed. As Sec. 3.2 prescribes
 *     for an incomplete matrix, each block step first imputes it with the
 *     current prediction, y_ij <- mu_ij, so its score term is zero and its
 *     Fisher weight stays; it adds nothing to the deviance (D(mu, mu) = 0).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int64_t n, m;
    int32_t p, q, d;
    int32_t family;     /* 0 Poisson, 1 NB, 2 Gaussian, 3 Bernoulli, 4 Gamma, 5 inverse Gaussian */
    int32_t nb_row, nb_col;
    int32_t bias_corr;  /* 0 printed formula, 1 per-visit */
    int32_t alpha_mode; /* 0 fixed NB shape / phi, 1 stochastic estimator (NB moments, Pearson phi),
                           2 fixed per-gene NB shapes */
    int32_t missing;    /* 1: the sentinel count marks a missing entry (imputed by mu, Sec. 3.2) */
    double lambda[4];   /* penalties on B, Gamma, U, V */
    double a1, a2;      /* EMA weights of eq. 12 */
    double k0, k1, tau; /* learning-rate schedule */
    double damping;     /* added to every curvature estimate */
    double eps;         /* floor of the NB shape update */
    double eta_clamp;
} gmfo_config;

typedef struct {
    const void* Y;         /* n x m responses, row-major, original order */
    int32_t y_dtype;       /* 0 int32, 1 uint16, 2 float32 */
    const double* W;       /* n x m weights or NULL (= 1) */
    const double* X;       /* n x p */
    const double* Z;       /* m x q */
    const double* offset;  /* n or NULL */
    const int32_t* row_perm; /* n: chunk c of rows is row_perm[c*nb_row ...] */
    const int32_t* col_perm; /* m */
    const double* alpha_col; /* m per-gene NB shapes (alpha_mode 2), original order, or NULL */
} gmfo_data;

typedef struct {
    double* B;      /* m x p */
    double* G;      /* n x q  (Gamma) */
    double* U;      /* n x d */
    double* V;      /* m x d */
    double* Gb_row; /* n x (q+d): smoothed gradient of [Gamma, U] */
    double* Hb_row; /* n x (q+d): smoothed curvature of [Gamma, U] */
    double* Gb_col; /* m x (p+d): smoothed gradient of [B, V] */
    double* Hb_col; /* m x (p+d) */
    int64_t* cnt_row; /* n: visits of each row */
    int64_t* cnt_col; /* m */
    double* alpha;  /* the family's scalar: smoothed NB shape, or dispersion phi */
    int64_t* t;     /* blocks processed so far */
} gmfo_state;

static double y_at(const gmfo_data* D, int64_t m, int64_t i, int64_t j) {
    if (D->y_dtype == 0) return (double)((const int32_t*)D->Y)[i * m + j];
    if (D->y_dtype == 2) return (double)((const float*)D->Y)[i * m + j];
    return (double)((const uint16_t*)D->Y)[i * m + j];
}

/* Entry (i, j) is missing: missing values are on and the count is the sentinel. */
static int missing_at(const gmfo_config* c, const gmfo_data* D, int64_t i, int64_t j) {
    if (!c->missing) return 0;
    if (D->y_dtype == 0) return ((const int32_t*)D->Y)[i * c->m + j] == -1;
    if (D->y_dtype == 2) return isnan(((const float*)D->Y)[i * c->m + j]);
    return ((const uint16_t*)D->Y)[i * c->m + j] == 65535;
}

static double w_at(const gmfo_data* D, int64_t m, int64_t i, int64_t j) {
    return D->W ? D->W[i * m + j] : 1.0;
}

/* Variance function nu(mu) of Table S1 (alpha: the NB shape). */
static double variance_fn(int family, double mu, double alpha) {
    switch (family) {
    case 0: return mu;
    case 1: return mu * (1.0 + mu / alpha);
    case 2: return 1.0;
    case 3: return mu * (1.0 - mu);
    case 4: return mu * mu;
    default: return mu * mu * mu;
    }
}

/* The families with a free dispersion phi (Gaussian, Gamma, inverse Gaussian). */
static int has_dispersion(int family) { return family == 2 || family == 4 || family == 5; }

/* Inverse link: identity (Gaussian), logistic (Bernoulli), exp (the others). */
static double inv_link(int family, double e) {
    if (family == 2) return e;
    if (family == 3) return 1.0 / (1.0 + exp(-e));
    return exp(e);
}

/* g'(mu) of the same links. */
static double link_deriv(int family, double mu) {
    if (family == 2) return 1.0;
    if (family == 3) return 1.0 / (mu * (1.0 - mu));
    return 1.0 / mu;
}

/*
 * Per-entry derivatives of Sec. 3:  Ddot = w (y - mu) / (phi nu(mu) g'(mu)),
 * Dddot = w / (phi nu(mu) g'(mu)^2), the expected (Fisher) second derivative,
 * alpha(mu) = 1.  scal is the family's scalar: the NB shape, or phi for the
 * families with a dispersion (phi = 1 for the others).
 */
void gmfo_entry(int family, double y, double eta, double w, double scal, double clamp,
                double* mu_out, double* ddot, double* dddot) {
    double e = eta;
    if (e > clamp) e = clamp;
    if (e < -clamp) e = -clamp;
    const double mu = inv_link(family, e);
    const double nu = variance_fn(family, mu, scal);
    const double gdot = link_deriv(family, mu);
    const double phi = has_dispersion(family) ? scal : 1.0;
    if (mu_out) *mu_out = mu;
    if (ddot) *ddot = w * (y - mu) / (phi * nu * gdot);
    if (dddot) *dddot = w / (phi * nu * gdot * gdot);
}

/* x log(x / z) with 0 log 0 = 0. */
static double xlogxz(double x, double z) { return x > 0 ? x * log(x / z) : 0.0; }

/* Unit deviance D(y, mu) = 2 w [D / 2a(phi) of Table S1] (App. B for NB), not divided by phi. */
double gmfo_entry_deviance(int family, double y, double mu, double w, double alpha) {
    switch (family) {
    case 0: return 2.0 * w * (xlogxz(y, mu) - (y - mu));
    case 1: return 2.0 * w * (xlogxz(y, mu) - (y + alpha) * log((y + alpha) / (mu + alpha)));
    case 2: return w * (y - mu) * (y - mu);
    case 3: return 2.0 * w * (xlogxz(y, mu) + xlogxz(1.0 - y, 1.0 - mu));
    case 4: return 2.0 * w * ((y - mu) / mu - log(y / mu));
    default: return w * (y - mu) * (y - mu) / (y * mu * mu);
    }
}

/* eta_ij = o_i + x_i' beta_j + gamma_i' z_j + u_i' v_j   (eq. 3 plus the offset) */
static double eta_at(const gmfo_config* c, const gmfo_data* D, const gmfo_state* S,
                     int64_t i, int64_t j) {
    double e = D->offset ? D->offset[i] : 0.0;
    for (int a = 0; a < c->p; a++) e += D->X[i * c->p + a] * S->B[j * c->p + a];
    for (int b = 0; b < c->q; b++) e += S->G[i * c->q + b] * D->Z[j * c->q + b];
    for (int h = 0; h < c->d; h++) e += S->U[i * c->d + h] * S->V[j * c->d + h];
    return e;
}

/*
 * Block estimators of eq. 15 in the covariate form of App. B, without the
 * penalty and damping terms (those are added by the update):
 *   Grow[i,c] = -(m/|J|) sum_j Ddot_ij [Z, V]_jc     Hrow = (m/|J|) sum_j Dddot_ij [Z*Z, V*V]_jc
 *   Gcol[j,c] = -(n/|I|) sum_i Ddot_ij [X, U]_ic     Hcol = (n/|I|) sum_i Dddot_ij [X*X, U*U]_ic
 * Row outputs are |I| x (q+d), column outputs |J| x (p+d).  nb_sums (may be
 * NULL) accumulates sum w mu^2 and sum w ((y-mu)^2 - mu) over the block (NB),
 * or the Pearson sum w (y - mu)^2 / nu(mu) and the number of observed entries
 * (families with a dispersion).
 */
int gmfo_block_grad(const gmfo_config* c, const gmfo_data* D, const gmfo_state* S, double alpha,
                    const int32_t* I, int64_t nI, const int32_t* J, int64_t mJ,
                    double* Grow, double* Hrow, double* Gcol, double* Hcol, double* nb_sums) {
    const int64_t n = c->n, m = c->m;
    const int p = c->p, q = c->q, d = c->d;
    const int fr = q + d, fc = p + d;
    memset(Grow, 0, sizeof(double) * nI * fr);
    memset(Hrow, 0, sizeof(double) * nI * fr);
    memset(Gcol, 0, sizeof(double) * mJ * fc);
    memset(Hcol, 0, sizeof(double) * mJ * fc);
    const double srow = (double)m / (double)mJ;
    const double scol = (double)n / (double)nI;
    for (int64_t a = 0; a < nI; a++) {
        const int64_t i = I[a];
        for (int64_t b = 0; b < mJ; b++) {
            const int64_t j = J[b];
            double mu, dd, ddd;
            const double eta = eta_at(c, D, S, i, j), w = w_at(D, m, i, j);
            const double aj = D->alpha_col ? D->alpha_col[j] : alpha;
            double y = y_at(D, m, i, j);
            if (missing_at(c, D, i, j)) gmfo_entry(c->family, 0.0, eta, w, aj, c->eta_clamp, &y, NULL, NULL);
            gmfo_entry(c->family, y, eta, w, aj, c->eta_clamp, &mu, &dd, &ddd);
            if (nb_sums && has_dispersion(c->family)) {
                if (!missing_at(c, D, i, j)) {
                    nb_sums[0] += w * (y - mu) * (y - mu) / variance_fn(c->family, mu, aj);
                    nb_sums[1] += 1.0;
                }
            } else if (nb_sums) {
                nb_sums[0] += w * mu * mu;
                nb_sums[1] += w * ((y - mu) * (y - mu) - mu);
            }
            /* row side: [Gamma, U] against [Z, V] */
            for (int k = 0; k < q; k++) {
                const double r = D->Z[j * q + k];
                Grow[a * fr + k] -= srow * dd * r;
                Hrow[a * fr + k] += srow * ddd * r * r;
            }
            for (int k = 0; k < d; k++) {
                const double r = S->V[j * d + k];
                Grow[a * fr + q + k] -= srow * dd * r;
                Hrow[a * fr + q + k] += srow * ddd * r * r;
            }
            /* column side: [B, V] against [X, U] */
            for (int k = 0; k < p; k++) {
                const double l = D->X[i * p + k];
                Gcol[b * fc + k] -= scol * dd * l;
                Hcol[b * fc + k] += scol * ddd * l * l;
            }
            for (int k = 0; k < d; k++) {
                const double l = S->U[i * d + k];
                Gcol[b * fc + p + k] -= scol * dd * l;
                Hcol[b * fc + p + k] += scol * ddd * l * l;
            }
        }
    }
    return 0;
}

static double rho_at(const gmfo_config* c, int64_t t) {
    return c->k0 / pow(1.0 + c->k0 * c->k1 * (double)t, c->tau);
}

static double bias_factor(const gmfo_config* c, int64_t t, int64_t visits) {
    if (c->bias_corr == 0) return (1.0 - pow(c->a2, (double)t)) / (1.0 - pow(c->a1, (double)t));
    return (1.0 - pow(1.0 - c->a2, (double)visits)) / (1.0 - pow(1.0 - c->a1, (double)visits));
}

/* EMA (eq. 12) and local step (eq. 14) of one free parameter. */
static void step_one(const gmfo_config* c, double* theta, double* gbar, double* hbar,
                     double ghat, double hhat, double rho, double cf) {
    *gbar = (1.0 - c->a1) * (*gbar) + c->a1 * ghat;
    *hbar = (1.0 - c->a2) * (*hbar) + c->a2 * hhat;
    *theta -= rho * cf * (*gbar) / (*hbar);
}

/*
 * One block step of Algorithm 1 (steps 2-4), with both sides computed from the
 * pre-step parameters and then updated.
 */
int gmfo_block_step(const gmfo_config* c, const gmfo_data* D, gmfo_state* S,
                    const int32_t* I, int64_t nI, const int32_t* J, int64_t mJ, double* nb_sums) {
    const int p = c->p, q = c->q, d = c->d;
    const int fr = q + d, fc = p + d;
    double* Grow = (double*)malloc(sizeof(double) * nI * fr);
    double* Hrow = (double*)malloc(sizeof(double) * nI * fr);
    double* Gcol = (double*)malloc(sizeof(double) * mJ * fc);
    double* Hcol = (double*)malloc(sizeof(double) * mJ * fc);
    if (!Grow || !Hrow || !Gcol || !Hcol) { free(Grow); free(Hrow); free(Gcol); free(Hcol); return -3; }
    gmfo_block_grad(c, D, S, *S->alpha, I, nI, J, mJ, Grow, Hrow, Gcol, Hcol, nb_sums);

    const int64_t t = ++(*S->t);
    const double rho = rho_at(c, t);
    /* column side: B (lambda[0]) then V (lambda[3]) */
    for (int64_t b = 0; b < mJ; b++) {
        const int64_t j = J[b];
        const int64_t k = ++S->cnt_col[j];
        const double cf = bias_factor(c, t, k);
        for (int e = 0; e < fc; e++) {
            double* theta = e < p ? &S->B[j * p + e] : &S->V[j * d + (e - p)];
            const double lam = e < p ? c->lambda[0] : c->lambda[3];
            const double gh = Gcol[b * fc + e] + lam * (*theta);
            const double hh = Hcol[b * fc + e] + lam + c->damping;
            step_one(c, theta, &S->Gb_col[j * fc + e], &S->Hb_col[j * fc + e], gh, hh, rho, cf);
        }
    }
    /* row side: Gamma (lambda[1]) then U (lambda[2]) */
    for (int64_t a = 0; a < nI; a++) {
        const int64_t i = I[a];
        const int64_t k = ++S->cnt_row[i];
        const double cf = bias_factor(c, t, k);
        for (int e = 0; e < fr; e++) {
            double* theta = e < q ? &S->G[i * q + e] : &S->U[i * d + (e - q)];
            const double lam = e < q ? c->lambda[1] : c->lambda[2];
            const double gh = Grow[a * fr + e] + lam * (*theta);
            const double hh = Hrow[a * fr + e] + lam + c->damping;
            step_one(c, theta, &S->Gb_row[i * fr + e], &S->Hb_row[i * fr + e], gh, hh, rho, cf);
        }
    }
    free(Grow); free(Hrow); free(Gcol); free(Hcol);
    return 0;
}

static void chunk(const int32_t* perm, int64_t total, int64_t size, int64_t c,
                  const int32_t** idx, int64_t* len) {
    const int64_t lo = c * size;
    int64_t hi = lo + size;
    if (hi > total) hi = total;
    *idx = perm + lo;
    *len = hi - lo;
}

/* Sweeps [w0, w1) of the epoch defined by sigma (schedule in the header). */
int gmfo_sgd_sweeps(const gmfo_config* c, const gmfo_data* D, gmfo_state* S, const int32_t* sigma,
                    int64_t w0, int64_t w1) {
    const int64_t r = (c->n + c->nb_row - 1) / c->nb_row;
    const int64_t s = (c->m + c->nb_col - 1) / c->nb_col;
    const int swap = r < s;
    const int64_t per = swap ? r : s;     /* blocks per sweep */
    for (int64_t w = w0; w < w1; w++) {
        double sums[2] = {0.0, 0.0};
        const int64_t t_first = *S->t + 1;
        for (int64_t k = 0; k < per; k++) {
            const int64_t rc = swap ? k : (sigma[w] + k) % r;
            const int64_t cc = swap ? (sigma[w] + k) % s : k;
            const int32_t *I, *J;
            int64_t nI, mJ;
            chunk(D->row_perm, c->n, c->nb_row, rc, &I, &nI);
            chunk(D->col_perm, c->m, c->nb_col, cc, &J, &mJ);
            int rc2 = gmfo_block_step(c, D, S, I, nI, J, mJ, sums);
            if (rc2) return rc2;
        }
        if (c->family == 1 && c->alpha_mode == 1 && sums[1] > 0.0) {
            double ahat = sums[0] / sums[1];
            if (ahat < c->eps) ahat = c->eps;
            const double rho = rho_at(c, t_first);
            *S->alpha = (1.0 - rho) * (*S->alpha) + rho * ahat;
        }
        if (has_dispersion(c->family) && c->alpha_mode == 1 && sums[1] > 0.0) {
            const double nm = (double)c->n * (double)c->m;
            const double dof = nm - (double)c->m * c->p - (double)c->n * c->q - (double)(c->n + c->m) * c->d - 1.0;
            if (dof > 0.0) {
                double phat = (nm / sums[1]) * sums[0] / dof;
                if (phat < c->eps) phat = c->eps;
                const double rho = rho_at(c, t_first);
                *S->alpha = (1.0 - rho) * (*S->alpha) + rho * phat;
            }
        }
    }
    return 0;
}

/* Sweep w restricted to the listed blocks (strictly increasing indices in
 * [0, per)), for a fit whose sweeps are split over several ranks: block k
 * takes global step t_first + k as in the whole sweep, and t ends at
 * t_first - 1 + per. The pooled NB shape update needs every block of the
 * sweep (returns -2 for a partial list with alpha_mode 1). */
int gmfo_sgd_sweep_blocks(const gmfo_config* c, const gmfo_data* D, gmfo_state* S, const int32_t* sigma, int64_t w,
                          const int32_t* blocks, int64_t nblocks) {
    const int64_t r = (c->n + c->nb_row - 1) / c->nb_row;
    const int64_t s = (c->m + c->nb_col - 1) / c->nb_col;
    const int swap = r < s;
    const int64_t per = swap ? r : s;
    if (nblocks == per) return gmfo_sgd_sweeps(c, D, S, sigma, w, w + 1);
    if ((c->family == 1 || has_dispersion(c->family)) && c->alpha_mode == 1) return -2;
    const int64_t t0 = *S->t;
    double sums[2] = {0.0, 0.0};
    for (int64_t b = 0; b < nblocks; b++) {
        const int64_t k = blocks[b];
        if (k < 0 || k >= per || (b > 0 && k <= blocks[b - 1])) return -1;
        const int64_t rc = swap ? k : (sigma[w] + k) % r;
        const int64_t cc = swap ? (sigma[w] + k) % s : k;
        const int32_t *I, *J;
        int64_t nI, mJ;
        chunk(D->row_perm, c->n, c->nb_row, rc, &I, &nI);
        chunk(D->col_perm, c->m, c->nb_col, cc, &J, &mJ);
        *S->t = t0 + k;   /* the block step raises it to t0 + k + 1 */
        int rc2 = gmfo_block_step(c, D, S, I, nI, J, mJ, sums);
        if (rc2) return rc2;
    }
    *S->t = t0 + per;
    return 0;
}

/* One epoch of Algorithm 1: all max(r, s) sweeps. */
int gmfo_sgd_epoch(const gmfo_config* c, const gmfo_data* D, gmfo_state* S, const int32_t* sigma) {
    const int64_t r = (c->n + c->nb_row - 1) / c->nb_row;
    const int64_t s = (c->m + c->nb_col - 1) / c->nb_col;
    return gmfo_sgd_sweeps(c, D, S, sigma, 0, r < s ? s : r);
}

/* Total deviance sum_ij D(y_ij, mu_ij) (Table S1, App. B) at the current parameters. */
double gmfo_deviance(const gmfo_config* c, const gmfo_data* D, const gmfo_state* S) {
    double total = 0.0;
    for (int64_t i = 0; i < c->n; i++) {
        for (int64_t j = 0; j < c->m; j++) {
            double mu;
            if (missing_at(c, D, i, j)) continue;   /* y <- mu: D(mu, mu) = 0 */
            const double aj = D->alpha_col ? D->alpha_col[j] : *S->alpha;
            gmfo_entry(c->family, 0.0, eta_at(c, D, S, i, j), 1.0, aj, c->eta_clamp, &mu, NULL, NULL);
            total += gmfo_entry_deviance(c->family, y_at(D, c->m, i, j), mu, w_at(D, c->m, i, j), aj);
        }
    }
    return total;
}

/* Linear predictor of the listed entries (i, j) -> out, for sampled checks. */
void gmfo_eta_entries(const gmfo_config* c, const gmfo_data* D, const gmfo_state* S,
                      const int64_t* ii, const int64_t* jj, int64_t count, double* out) {
    for (int64_t k = 0; k < count; k++) out[k] = eta_at(c, D, S, ii[k], jj[k]);
}
