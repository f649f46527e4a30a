/*
 * gmf.h -- C ABI of the GB300 (sm_103a) library for block-wise adaptive SGD on
 * generalized matrix factorization (GMF) models of count matrices
 * (Castiglione, Segers, Clement, Risso; arXiv 2412.20509).
 *
 * Model (Sec. 2, eq. 1-3; offset as in Sec. 4.1 and App. B):
 *   y_ij ~ EF(mu_ij),  log mu_ij = eta_ij = o_i + x_i'beta_j + gamma_i'z_j + u_i'v_j
 * with rows i = 1..n (cells) and columns j = 1..m (genes); X (n x p) and
 * Z (m x q) are fixed covariates, B (m x p), Gamma (n x q), U (n x d),
 * V (m x d) are fitted. Families: Poisson and negative binomial with shape
 * alpha (Table S1, App. B), log link, dispersion phi = 1.
 *
 * Conventions for every entry point:
 *   - Return value: GMF_OK (0) or a negative GMF_ERR_* code; nothing throws.
 *     gmf_last_error() returns a thread-local message for the last failure.
 *   - Matrices are dense, row-major, C-contiguous.
 *   - "host" pointers are ordinary CPU memory (pageable or pinned); "device"
 *     pointers are CUDA global memory of the current device.
 *   - stream is a cudaStream_t (NULL = legacy default stream). Work is
 *     enqueued on it; functions documented as synchronous wait for it.
 *   - The handle owns all of its device memory. Caller buffers are only read
 *     during the call (or, for outputs, written before a synchronous return),
 *     except where a function states otherwise (gmf_update_y_async, and the
 *     work that asynchronous functions enqueue on their stream).
 *   - A handle must not be used from two host threads at once.
 */
#ifndef GMF_H
#define GMF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    GMF_OK = 0,
    GMF_ERR_ARG = -1,       /* invalid argument (shape, pointer, value) */
    GMF_ERR_CUDA = -2,      /* a CUDA runtime/driver call failed */
    GMF_ERR_OOM = -3,       /* device or host allocation failed */
    GMF_ERR_TIMEOUT = -4,   /* a bounded device-side wait gave up */
    GMF_ERR_NONFINITE = -5, /* a non-finite value was produced */
    GMF_ERR_STATE = -6      /* handle not in a state that allows the call */
};

/* Families of Table S1 and their links: log for the Poisson, the negative
   binomial, the Gamma and the inverse Gaussian; identity for the Gaussian and
   logit for the Bernoulli (their canonical links). The Gaussian, Gamma and
   inverse Gaussian have a dispersion phi (App. B), held where the negative
   binomial holds its shape (alpha0, gmf_get_params' alpha). */
enum {
    GMF_POISSON = 0,
    GMF_NEGBIN = 1,
    GMF_GAUSSIAN = 2,   /* float32 responses */
    GMF_BINOMIAL = 3,   /* Bernoulli: responses in [0, 1] (counts 0 / 1, or float32) */
    GMF_GAMMA = 4,      /* float32 responses > 0 */
    GMF_INVGAUSS = 5    /* float32 responses > 0 */
};
enum { GMF_Y_INT32 = 0, GMF_Y_UINT16 = 1, GMF_Y_FLOAT32 = 2 };  /* response storage type */
/* missing-entry markers (cfg.missing = 1); float32 responses mark a missing entry by NaN */
enum { GMF_MISSING_INT32 = -1, GMF_MISSING_UINT16 = 65535 };
enum {
    GMF_PREC_FP32 = 0,   /* FP32 on the CUDA cores throughout (reference path) */
    GMF_PREC_MIXED = 1   /* tcgen05 tensor cores: eta as split-BF16 (3 products),
                            gradient/curvature contractions in BF16, FP32 accumulate */
};
enum { GMF_ORTH_B1 = 1, GMF_ORTH_B2 = 2, GMF_ORTH_B3 = 3 };  /* Sec. 2.1 */
enum {
    /* Mixed precision: where the tiles of a block fit one thread-block cluster
       (at most 16 tiles of 128 x 128, with room for the clusters of a sweep on
       the device), the strip updates run inside the tile launch and the tiles
       exchange their partial sums through distributed shared memory. This flag
       keeps them in their own launch instead. Both give bitwise equal results. */
    GMF_FLAG_NO_CLUSTER = 1,
    /* Mixed precision: run a whole epoch (or sweep range) as one persistent
       launch instead of one or two launches per sweep. Bitwise equal results.
       In cluster mode (fixed NB shape or Poisson) each cluster runs its block
       of every sweep in turn and waits only for the blocks that updated its
       moving strip earlier in the epoch (see gmf_strip_schedule); on the
       20000 x 2000 benchmark this is about 6% slower than the per-sweep
       cluster launches, since the blocks of a cluster form a serial chain
       through the fixed strip. Otherwise (blocks of more than 16 tiles, or
       GMF_FLAG_NO_CLUSTER; any NB shape mode) the launch is a dataflow of
       tile and update items taken in a fixed order by all resident CTAs, each
       item waiting only for the updates of the strips it reads (see
       gmf_set_flow_lag), so tiles of the next sweep run while the last tiles
       and the updates of the current one finish. Without a device that can
       keep every CTA resident the per-sweep launches stay (gmf_epoch_mode
       tells which mode runs). */
    GMF_FLAG_PERSIST = 2,
    /* Mixed precision: gmf_deviance computes eta in FP32 on the CUDA cores (the
       kernel of the FP32 path) instead of from the block step's split-BF16
       tensor-core products. */
    GMF_FLAG_SIMT_DEVIANCE = 4,
    /* gmf_update_y_async: copy the counts by the copy engines into a device
       staging buffer and permute them on the stream, even where the device
       could gather them straight from host memory. The gather's CTAs take SM
       room from kernels running beside it (an SM that holds one has registers
       for one block-step tile instead of two), while the copy engines are
       otherwise idle; the permutation then runs on the stream (a read and a
       write of n x m counts in HBM). Costs two staging buffers of n x m
       counts. */
    GMF_FLAG_STAGED_UPLOAD = 8
};

typedef struct gmf_model gmf_model;  /* opaque, library-owned */

/*
 * Fit configuration. Defaults in brackets are the paper's sgdGMF settings
 * (App. C) where it states them, otherwise the library's reading.
 */
typedef struct {
    int64_t n, m;        /* rows (cells) and columns (genes) of Y */
    int32_t p, q, d;     /* columns of X, columns of Z, latent rank (d >= 0) */
    int32_t family;      /* GMF_POISSON, GMF_NEGBIN, GMF_GAUSSIAN, GMF_BINOMIAL, GMF_GAMMA or GMF_INVGAUSS */
    int32_t nb_row;      /* row minibatch size n* (rows per partition chunk) */
    int32_t nb_col;      /* column minibatch size m* */
    int32_t bias_corr;   /* 0: c_t = (1-a2^t)/(1-a1^t), global block count t (eq. 11);
                            1: c = (1-(1-a2)^k)/(1-(1-a1)^k), k = visits of the row/column */
    int32_t alpha_mode;  /* NB: 0 shape fixed; 1 stochastic moment estimator (App. B), pooled per
                            sweep; 2 one fixed shape per gene (gmf_set_gene_shapes).
                            Gaussian, Gamma, inverse Gaussian: 0 phi fixed; 1 the smoothed stochastic
                            Pearson estimator of App. B, pooled per sweep: the sweep's sum of
                            w (y - mu)^2 / nu(mu) times nm / (its observed entries), over the residual
                            degrees of freedom nm - mp - nq - (n+m)d - 1, smoothed with rho of the
                            sweep's first block (floored at eps). Poisson, Bernoulli: 0. */
    int32_t precision;   /* GMF_PREC_FP32 or GMF_PREC_MIXED */
    int32_t flags;       /* GMF_FLAG_* bits; 0 for the defaults */
    int32_t missing;     /* 1: a count equal to GMF_MISSING_INT32 / GMF_MISSING_UINT16 marks an entry
                            that is not observed; every block step imputes it with the current mean,
                            y_ij <- mu_ij (Sec. 3.2), so it adds no score and no deviance but keeps its
                            Fisher weight. uint16 counts are then at most 65534. [0: all observed] */
    double lambda[4];    /* ridge penalties on (B, Gamma, U, V), eq. 6 [0, 0, 1, 0] */
    double a1, a2;       /* EMA weights of eq. 12 [0.1, 0.01] */
    double k0, k1, tau;  /* rho_t = k0 / (1 + k0 k1 t)^tau (Sec. 3.2) [0.01, 1e-3, 0.75] */
    double damping;      /* added to every curvature estimate [1e-3] */
    double eps;          /* floor of the NB shape and dispersion updates (App. B) [1e-8] */
    double eta_clamp;    /* eta is clamped to [-eta_clamp, eta_clamp] before the inverse link [30] */
} gmf_config;

/* Fill *cfg with the defaults above for the given sizes. */
void gmf_config_default(gmf_config* cfg, int64_t n, int64_t m, int32_t p, int32_t q, int32_t d,
                        int32_t family, int32_t nb_row, int32_t nb_col);

/*
 * gmf_init -- create a fit (model of Sec. 2, state of Algorithm 1).
 *
 * The random partitions {I_1..I_r} and {J_1..J_s} of Algorithm 1 are fixed
 * here, once, as in the algorithm: row chunk c is rows
 * row_perm[c*nb_row .. min(n,(c+1)*nb_row)-1], column chunk c likewise with
 * col_perm and nb_col (the last chunk may be smaller). The library stores Y
 * (and W) and the parameters permuted so that every block is contiguous.
 *
 *   Y           n x m responses: counts (y_dtype GMF_Y_INT32 or GMF_Y_UINT16,
 *               >= 0) for the Poisson, NB and Bernoulli families, float32
 *               (GMF_Y_FLOAT32) for the Gaussian, Gamma, inverse Gaussian and
 *               Bernoulli; host or device memory as y_on_device says. Copied.
 *               Fits of the families beyond Poisson and NB support the block
 *               step, the deviance, the orthogonalisation and the parameter /
 *               state calls; the count-model calls (projection, held-out
 *               metrics, log-likelihood, start, gene shapes, rank sweep)
 *               return GMF_ERR_STATE for them.
 *   W           NULL (all weights 1) or n x m float32 weights w_ij > 0
 *               (a_ij(phi) = phi/w_ij, Sec. 2), same memory space as Y. Copied.
 *   X, Z        host double, n x p and m x q.  offset: host double n, or NULL.
 *   row_perm    host int32 permutation of 0..n-1; col_perm of 0..m-1.
 *   B0..V0      host double starting values (m x p, n x q, n x d, m x d).
 *   alpha0      starting NB shape, or starting dispersion phi (> 0; ignored for
 *               the Poisson and Bernoulli families).
 * The smoothed derivatives start at zero and t at 0. Synchronous.
 * Errors: GMF_ERR_ARG for bad sizes/pointers/permutations, GMF_ERR_OOM, GMF_ERR_CUDA.
 */
int gmf_init(gmf_model** out, const gmf_config* cfg,
             const void* Y, int32_t y_dtype, int32_t y_on_device, const float* W,
             const double* X, const double* Z, const double* offset,
             const int32_t* row_perm, const int32_t* col_perm,
             const double* B0, const double* G0, const double* U0, const double* V0,
             double alpha0, void* stream);

/*
 * gmf_update_y -- replace the counts (same n, m and dtype as at init) from
 * host or device memory, e.g. a new batch of a streamed matrix. Asynchronous
 * on the stream for device sources; for host sources the call returns once
 * the host buffer may be reused.
 */
int gmf_update_y(gmf_model* h, const void* Y, int32_t y_on_device, void* stream);

/*
 * gmf_update_y_async -- replace the counts from a host buffer without waiting:
 * for streaming a sequence of count matrices of the same shape. Work enqueued
 * on `stream` before this call sees the old counts, work enqueued after it the
 * new ones. When the device can read Y (page-locked, mapped memory:
 * cudaHostAlloc, cudaHostRegister with mapping, torch's pin_memory; any host
 * memory where the device reads pageable memory, as on Grace-based systems),
 * Y is 16-byte aligned, and a row of counts is a multiple of 16 bytes of at
 * most 48 KiB, one gather kernel on the library's
 * copy stream reads Y over the host link and writes the permuted counts into
 * the handle's second count buffer (allocated on first use, n x m counts), and
 * the handle switches buffers: the upload overlaps work already enqueued on
 * `stream`, which keeps reading the previous buffer. Otherwise (and always
 * with GMF_FLAG_STAGED_UPLOAD) the counts are copied on the copy stream into
 * one of two device staging buffers and permuted in place on `stream` after
 * the copy. Y: host, n x m counts of the
 * init dtype; it must stay unchanged until `stream` has passed the work
 * enqueued by this call (e.g. after a later synchronous call on it). At most
 * two calls may be in flight on one handle. The paper has no counterpart (a
 * deployment variant of gmf_update_y). Errors: GMF_ERR_ARG, GMF_ERR_STATE (a
 * handle that reads another handle's counts), GMF_ERR_CUDA.
 */
int gmf_update_y_async(gmf_model* h, const void* Y, void* stream);

/* Count buffers the handle holds on the device: 1, or 2 once gmf_update_y_async
 * took the direct path. -1 for a NULL handle. */
int32_t gmf_count_buffers(const gmf_model* h);

/* Number of sweeps per epoch: max(r, s) with r = ceil(n/nb_row), s = ceil(m/nb_col). */
int32_t gmf_num_sweeps(const gmf_model* h);

/* Kernel launches per sweep of gmf_sgd_epoch / gmf_sgd_sweeps: 1 when the
 * strip updates run inside the tile launch (cluster mode, see
 * GMF_FLAG_NO_CLUSTER), else 2 (tiles, then updates); 0 when a sweep range is
 * one persistent launch (GMF_FLAG_PERSIST). -1 for a NULL handle. */
int32_t gmf_launches_per_sweep(const gmf_model* h);

/* How gmf_sgd_epoch / gmf_sgd_sweeps launch: GMF_EPOCH_SEPARATE (per sweep, a
 * tile launch and an update launch), GMF_EPOCH_CLUSTER (per sweep, one
 * launch), GMF_EPOCH_PERSISTENT (one launch for the whole sweep range). -1 for
 * a NULL handle. */
enum { GMF_EPOCH_SEPARATE = 0, GMF_EPOCH_CLUSTER = 1, GMF_EPOCH_PERSISTENT = 2 };
int32_t gmf_epoch_mode(const gmf_model* h);

/*
 * gmf_strip_schedule -- the dependency counts of a persistent sweep range
 * (host only, no device work). Algorithm 1's sweeps give block k of sweep w a
 * fixed strip (column block k when r >= s, row block k otherwise), which only
 * block k of other sweeps touches, and a moving strip m(w, k) = (sigma[w] + k)
 * mod r (mod s when r < s). need_out[(w - w_begin) * per + k], per = min(r,
 * s), receives the number of sweeps w' in [w_begin, w) whose blocks visit
 * m(w, k): block k of sweep w may read that strip once that many earlier
 * visits have written it back. sigma: host, the epoch's S = max(r, s) sweep
 * offsets; need_out: host, (w_end - w_begin) * per int32. Errors:
 * GMF_ERR_ARG (r or s < 1, a range outside [0, S], an offset outside [0, S),
 * NULL pointers).
 */
int gmf_strip_schedule(int32_t r, int32_t s, const int32_t* sigma, int32_t w_begin, int32_t w_end,
                       int32_t* need_out);

/*
 * gmf_sgd_epoch -- one epoch of Algorithm 1: every block (I_a, J_b) once.
 *
 * sigma: host int32 permutation of 0..S-1, S = gmf_num_sweeps(h) (the
 * sampling of I in Algorithm 1). With r >= s, sweep w visits the s blocks
 * (I_{(sigma[w]+k) mod r}, J_k), k = 0..s-1; with r < s the roles swap. The
 * blocks of one sweep are disjoint in rows and columns and run concurrently.
 * Per block (eq. 15 with App. B, eq. 12, eq. 14): eta, mu = exp(eta), the
 * derivatives Ddot, Dddot (Sec. 3), the minibatch gradient and diagonal
 * curvature of [Gamma, U]_I and [B, V]_J, EMA smoothing and the local step
 * theta <- theta - rho_t c_t Gbar/Hbar, with both sides using the block's
 * pre-step parameters. NB with alpha_mode 1: the shape is updated once per
 * sweep from moment sums pooled over the sweep. t advances by one per block.
 * Each sweep is two kernel launches (the tiles, then the strip updates), with
 * programmatic stream serialization between them, or one (cluster mode), or
 * the whole epoch is one persistent launch (see gmf_epoch_mode).
 * Asynchronous on the stream (sigma is copied before return).
 */
int gmf_sgd_epoch(gmf_model* h, const int32_t* sigma, void* stream);

/*
 * gmf_sgd_sweeps -- run only sweeps [w_begin, w_end) of the epoch defined by
 * sigma (same semantics as gmf_sgd_epoch; t advances by the blocks run).
 */
int gmf_sgd_sweeps(gmf_model* h, const int32_t* sigma, int32_t w_begin, int32_t w_end, void* stream);

/*
 * Sharded sweeps (several ranks, each with its own handle and GPU). The s
 * blocks of one sweep of Algorithm 1 touch disjoint row and column chunks
 * (Sec. 3.2: their block estimators and local steps commute), so the blocks
 * of a sweep can run on different ranks. With r >= s a rank that owns column
 * chunk k runs block k of every sweep: its column chunks' state never moves,
 * and after each sweep the row chunks the sweep updated are copied to every
 * other rank (with r < s the roles swap). Done in the sweep order, this gives
 * every rank the parameters of the single-handle fit bit for bit.
 *
 * gmf_sgd_sweep_blocks -- sweep w of the epoch defined by sigma (as
 *   gmf_sgd_sweeps), restricted to the blocks k listed in `blocks` (host,
 *   strictly increasing, within [0, per), per = min(r, s); copied before
 *   return); nblocks = 0 runs nothing. Block k still takes its step factor
 *   from its place in the sweep, and t advances by per, as if every block had
 *   run. A pooled NB shape update (alpha_mode 1) needs every block of the sweep
 *   (GMF_ERR_STATE otherwise). Asynchronous on the stream. Errors: GMF_ERR_ARG,
 *   GMF_ERR_STATE, GMF_ERR_CUDA.
 * gmf_chunk_bytes -- bytes of the packed state of row chunk (side 0) or
 *   column chunk (side 1) `chunk`: rows x (KP + 2 nf + 1) floats, where KP is
 *   the factor row stride (1+p+q+d rounded up to 4) and nf = q+d (rows) or p+d
 *   (columns); -1 for a NULL handle or an index out of range.
 * gmf_chunk_state -- copy that state to (write = 0) or from (write = 1) the
 *   device buffer buf, row by row in the partition's order: [the augmented
 *   factor row (L or R, eta = L R') | smoothed gradients | smoothed curvatures
 *   (eq. 12) | visit count (int32 bits)]. Asynchronous on the stream. Errors:
 *   GMF_ERR_ARG (NULL pointers, side / chunk out of range), GMF_ERR_CUDA.
 */
int gmf_sgd_sweep_blocks(gmf_model* h, const int32_t* sigma, int32_t w, const int32_t* blocks, int32_t nblocks,
                         void* stream);
int64_t gmf_chunk_bytes(const gmf_model* h, int32_t side, int32_t chunk);
int gmf_chunk_state(gmf_model* h, int32_t side, int32_t chunk, void* buf, int32_t write, void* stream);

/*
 * gmf_deviance -- total deviance sum_ij D(y_ij, mu_ij) at the current
 * parameters (Table S1; App. B for NB, with the current shape), each entry in
 * FP32, summed per tile with compensation and combined in FP64. eta: FP32 on
 * the CUDA cores for FP32 handles (and with GMF_FLAG_SIMT_DEVIANCE); on
 * mixed-precision handles the block step's split-BF16 tensor-core products
 * (relative error of eta a few 1e-6 of sum_k |L_ik R_jk|). Entries marked
 * missing (cfg.missing = 1) add nothing (D(mu, mu) = 0 after imputation).
 * Synchronous; *out_total is host memory.
 */
int gmf_deviance(gmf_model* h, double* out_total, void* stream);

/*
 * gmf_holdout -- out-of-sample reconstruction error of a fit trained with
 * held-out entries marked missing (cfg.missing = 1), the evaluation of Sec. 5.2.
 * The held-out set V is the entries marked missing in the fit's counts; Ytrue
 * (device, n x m counts of the init dtype, the caller's original row and
 * column order) holds their true values (its other entries are not read).
 * out (host, 4 doubles): [0] Error = sum_V [log((1+y)/(1+mu))]^2 /
 * sum_V [log((1+y)/(1+ybar))]^2, [1] Deviance = sum_V D(y, mu) /
 * sum_V D(y, ybar) with D the Poisson unit deviance (Table S1), ybar the mean of
 * the observed counts, [2] ybar, [3] |V|; mu = exp(eta) at the current
 * parameters. FP32 terms, FP64 sums. Synchronous; allocates a few KB of
 * device workspace on the stream. Errors: GMF_ERR_ARG, GMF_ERR_STATE (no
 * missing entries, or cfg.missing = 0), GMF_ERR_CUDA, GMF_ERR_OOM.
 */
int gmf_holdout(gmf_model* h, const void* Ytrue, double* out, void* stream);

/*
 * gmf_loglik -- the log-likelihood and the Pearson statistic of the observed
 * entries at the current parameters, for information criteria (AIC, BIC:
 * Sec. 4.2) and the Pearson dispersion estimate (App. B, "Unknown dispersion
 * parameter"). out (host, 3 doubles): [0] sum_ij w_ij log f(y_ij; mu_ij) with
 * the full densities of Table S1's Poisson and negative binomial laws (log-gamma
 * terms included; NB with the current shape), [1] sum_ij w_ij (y_ij - mu_ij)^2 /
 * nu(mu_ij), [2] the number of observed entries. Entries marked missing are
 * left out. FP32 terms (lgammaf), FP64 sums. Synchronous; allocates a few KB
 * of device workspace on the stream. Errors: GMF_ERR_ARG, GMF_ERR_CUDA,
 * GMF_ERR_OOM.
 */
int gmf_loglik(gmf_model* h, double* out, void* stream);

/* As gmf_deviance, but writes the FP64 total to device memory d_out and does not synchronize. */
int gmf_deviance_async(gmf_model* h, double* d_out, void* stream);

/*
 * gmf_get_params / gmf_set_params -- copy the parameters out / in, host
 * double, original (unpermuted) order: B m x p, G (Gamma) n x q, U n x d,
 * V m x d, and the NB shape. Any pointer may be NULL to skip it. Synchronous.
 */
int gmf_get_params(gmf_model* h, double* B, double* G, double* U, double* V, double* alpha, void* stream);
int gmf_set_params(gmf_model* h, const double* B, const double* G, const double* U, const double* V,
                   const double* alpha, void* stream);

/*
 * gmf_get_ema / gmf_set_ema -- the optimiser state of eq. 12: smoothed
 * gradient and curvature of [Gamma, U] (n x (q+d)) and [B, V] (m x (p+d)),
 * visit counters (n and m), and the block count t. Host, original order,
 * synchronous; NULL pointers are skipped (t is skipped when t_io is NULL).
 * With gmf_get_params these make a complete checkpoint.
 */
int gmf_get_ema(gmf_model* h, double* Gb_row, double* Hb_row, double* Gb_col, double* Hb_col,
                int64_t* cnt_row, int64_t* cnt_col, int64_t* t_io, void* stream);
int gmf_set_ema(gmf_model* h, const double* Gb_row, const double* Hb_row, const double* Gb_col,
                const double* Hb_col, const int64_t* cnt_row, const int64_t* cnt_col, const int64_t* t_in,
                void* stream);

/*
 * gmf_orthogonalize -- Algorithm 2 (Sec. 2.1 and its appendix): project Gamma
 * and U off span(X) and V off span(Z) while moving the removed parts into B
 * and Gamma (eta unchanged), then impose (B1), (B2) or (B3). Computed in
 * FP64 on the device (Gram reductions over n and m) with a d x d SVD /
 * eigen-decomposition on the host. Resets the smoothed derivatives and visit
 * counters (they refer to the old basis). Synchronous.
 */
int gmf_orthogonalize(gmf_model* h, int32_t mode, void* stream);

/*
 * gmf_project_cells -- scores of new cells with the column side fixed
 * (B, V, Z and the NB shape of the fit). Each new row i solves the row
 * problem of Sec. 3 (rows separate given V) by n_steps exact Fisher-scoring
 * steps on theta_i = [gamma_i, u_i] (the row step of AIRWLS, Sec. 3.1):
 *   theta <- theta + (R' diag(Dddot_i) R + Lambda)^-1 (R' Ddot_i - Lambda theta),  R = [Z, V].
 * Start: u_i = U_start row (NULL: zeros); gamma_i0 (the first Z column, exact
 * when it is the intercept) in closed form log(max(sum_j y_ij, 0.5) /
 * sum_j exp(eta_ij without gamma)), the other gamma 0. Requires 1 <= q + d <= 32.
 * Step control (the paper states none for this problem): each of the n_steps + 1
 * passes over the genes evaluates f = 0.5 dev_i + 0.5 theta' Lambda theta at
 * the current point; a point with f <= f_best + 1e-5 (1 + |f_best|) is taken
 * and stepped from, otherwise the last step is halved from the best point.
 * The outputs are the best point and its deviance. n_steps = 0 returns the start.
 * Precision: on a GMF_PREC_MIXED handle with q + d <= 22, q >= 1, p <= 8, uint16
 * counts (16-byte aligned, m a multiple of 8) the Fisher matrices are formed on
 * the tensor cores from BF16 weights and BF16 products r_ja r_jb (FP32
 * accumulate); the score, eta and the deviance stay FP32. Otherwise FP32 throughout.
 * Ynew columns are genes in the caller's original order.
 *   Ynew      device, n_new x m counts (y_dtype)
 *   Xnew      device float32, n_new x p;  offset_new: device float32 n_new or NULL
 *   U_start   device float32 n_new x d or NULL
 *   U_out     device float32 n_new x d;  G_out: device float32 n_new x q
 *   dev_out   device float32 n_new (per-cell deviance at the result) or NULL
 * n_new = 0 is an empty batch: nothing is read or written (pointers may be NULL).
 * Asynchronous on the stream. Allocates its workspace from the handle.
 * Errors: GMF_ERR_ARG (n_new < 0, bad y_dtype, n_steps outside [0, 1000], NULL
 * pointers of a non-empty batch), GMF_ERR_CUDA.
 */
int gmf_project_cells(gmf_model* h, const void* Ynew, int32_t y_dtype, int64_t n_new,
                      const float* Xnew, const float* offset_new, const float* U_start,
                      int32_t n_steps, float* U_out, float* G_out, float* dev_out, void* stream);

/*
 * Batched rank sweep: fits of the same model with different latent ranks on one
 * count matrix (the grid of fits that rank selection by information criteria or
 * held-out deviance needs, Sec. 4.2).
 *
 * gmf_sweep_init -- arguments as gmf_init, for n_models models of ranks
 * d_list[0..n_models-1] (cfg->d is ignored). The starting values are arrays of
 * n_models host pointers: B0[i] m x p, G0[i] n x q, U0[i] n x d_list[i],
 * V0[i] m x d_list[i], alpha0[i]. The counts, weights and partitions are stored
 * once and read by every model. Synchronous.
 * gmf_sweep_epoch -- one epoch of every model (same sigma semantics as
 * gmf_sgd_epoch): per sweep, the models, heaviest first, go in groups (all of
 * them by default, see gmf_sweep_set_group); one tile launch covers the models
 * of a group and one update launch their strips.
 * Results equal running each model's own gmf_sgd_epoch, whatever the grouping.
 * gmf_sweep_set_group -- models per launch group: 1..n_models, 0 for all,
 *   GMF_SWEEP_SEQUENTIAL: each model's own epoch (gmf_sgd_epoch's launches and
 *   graph), model after model, or GMF_SWEEP_PERSISTENT (mixed precision): per
 *   sweep, one cooperative persistent launch for all models, whose CTAs (as many
 *   as fit on the device) take the tiles of every model, heaviest model first,
 *   pass a grid barrier (bounded by the global timer, GMF_ERR_TIMEOUT past 2 s)
 *   and take the strip updates. Errors: GMF_ERR_ARG (outside [-1, n_models]
 *   and not GMF_SWEEP_PERSISTENT, or GMF_SWEEP_PERSISTENT on the FP32 path).
 * gmf_sweep_group -- the current group size (n_models when all,
 *   GMF_SWEEP_SEQUENTIAL, GMF_SWEEP_PERSISTENT); -2 for NULL.
 * gmf_sweep_autotune -- times sweeps [0, n_sweeps) of the epoch defined by
 *   sigma (1 <= n_sweeps <= S) for the group sizes n_models, ceil(n_models/2),
 *   ..., 1, for GMF_SWEEP_SEQUENTIAL and (mixed precision) GMF_SWEEP_PERSISTENT,
 *   each from the same state (the models' parameters, smoothed derivatives,
 *   visit counts, shapes and t are saved before and restored after), and keeps
 *   the fastest. group_out (host, may be NULL): the chosen setting; ms_out
 *   (host, n_models + 2 floats, may be NULL): the time of group size g at
 *   ms_out[g - 1], of the sequential setting at ms_out[n_models] and of the
 *   persistent launch at ms_out[n_models + 1], -1 where not tried. Synchronous; needs device memory for
 *   one copy of the models' state. Errors: GMF_ERR_ARG, GMF_ERR_OOM, GMF_ERR_CUDA.
 * gmf_sweep_model -- the i-th model's handle, owned by the sweep and valid until
 * gmf_sweep_free, for gmf_deviance, gmf_get_params, gmf_orthogonalize, ...
 * (NULL if i is out of range). gmf_update_y is not allowed on models i > 0.
 */
typedef struct gmf_sweep gmf_sweep;
enum { GMF_SWEEP_SEQUENTIAL = -1, GMF_SWEEP_PERSISTENT = -3 };
int gmf_sweep_init(gmf_sweep** out, const gmf_config* cfg, const int32_t* d_list, int32_t n_models, const void* Y,
                   int32_t y_dtype, int32_t y_on_device, const float* W, const double* X, const double* Z,
                   const double* offset, const int32_t* row_perm, const int32_t* col_perm, const double* const* B0,
                   const double* const* G0, const double* const* U0, const double* const* V0, const double* alpha0,
                   void* stream);
int gmf_sweep_epoch(gmf_sweep* s, const int32_t* sigma, void* stream);
int gmf_sweep_set_group(gmf_sweep* s, int32_t group);
int32_t gmf_sweep_group(const gmf_sweep* s);
int gmf_sweep_autotune(gmf_sweep* s, const int32_t* sigma, int32_t n_sweeps, int32_t* group_out, float* ms_out,
                       void* stream);
gmf_model* gmf_sweep_model(gmf_sweep* s, int32_t i);
void gmf_sweep_free(gmf_sweep* s);

/*
 * Warm-start encoder for gmf_project_cells (the paper has no network; it
 * supplies the training targets -- the fitted, orthogonalised scores U -- and
 * the per-cell projection the network warms up):
 *   x = log(1 + y);  h1 = gelu(W1 x + b1);  h2 = gelu(W2 h1 + b2);  o = W3 h2 + b3
 * with gelu(t) = t Phi(t), trained by minimising mean (o - target)^2 with Adam.
 * Parameters are FP32: W1 n_h1 x n_in, W2 n_h2 x n_h1, W3 n_out x n_h2 (row-major),
 * biases vectors. All products run on the library's FP32 tiled GEMM kernel.
 *
 * gmf_mlp_create     -- zero parameters; max_batch bounds the rows of one
 *                       forward chunk / training batch (activations are sized for it).
 * gmf_mlp_set_params / gmf_mlp_get_params / gmf_mlp_get_grads -- host FP32 copies
 *                       (NULL pointers are skipped); set_params also resets Adam.
 * gmf_mlp_forward    -- o for `rows` cells: Y device rows x n_in counts
 *                       (y_dtype), out device rows x n_out. Asynchronous.
 *                       rows = 0: nothing to do (pointers may be NULL).
 * gmf_mlp_loss_grad  -- loss (device float, may be NULL) and the gradients of one
 *                       batch (rows <= max_batch) into the network. Asynchronous.
 * gmf_mlp_adam       -- one Adam step with the stored gradients. Asynchronous.
 * gmf_mlp_set_precision -- GMF_PREC_FP32 (the default: every product in FP32) or
 *                       GMF_PREC_MIXED: the first layer, z1 = W1 log(1 + y) + b1, runs on
 *                       the tcgen05 tensor cores with W1 and log(1 + y) rounded to BF16
 *                       (round to nearest even) and FP32 accumulation; the other layers and
 *                       the gradients stay FP32. Needs n_h1 a multiple of 16 in [16, 256];
 *                       the counts passed later must be 16-byte aligned with n_in * sizeof(count)
 *                       a multiple of 16 (GMF_ERR_ARG otherwise). Keeps a BF16 copy of W1,
 *                       refreshed by set_params and every Adam step.
 * gmf_mlp_train      -- `epochs` passes of minibatches of `batch` rows in an order
 *                       drawn from `seed` (SplitMix64 on the host); losses (host,
 *                       may be NULL) receives the mean loss of each epoch. Allocates
 *                       rows int64 + epochs doubles of workspace for the call; the
 *                       host waits only once per epoch. Synchronous.
 */
typedef struct gmf_mlp gmf_mlp;
int gmf_mlp_create(gmf_mlp** out, int32_t n_in, int32_t n_h1, int32_t n_h2, int32_t n_out, int32_t max_batch,
                   void* stream);
int gmf_mlp_set_params(gmf_mlp* net, const float* W1, const float* b1, const float* W2, const float* b2,
                       const float* W3, const float* b3, void* stream);
int gmf_mlp_get_params(gmf_mlp* net, float* W1, float* b1, float* W2, float* b2, float* W3, float* b3, void* stream);
int gmf_mlp_get_grads(gmf_mlp* net, float* W1, float* b1, float* W2, float* b2, float* W3, float* b3, void* stream);
int gmf_mlp_forward(gmf_mlp* net, const void* Y, int32_t y_dtype, int64_t rows, float* out, void* stream);
int gmf_mlp_loss_grad(gmf_mlp* net, const void* Y, int32_t y_dtype, int64_t rows, const float* target, float* loss,
                      void* stream);
int gmf_mlp_adam(gmf_mlp* net, float lr, float beta1, float beta2, float eps, void* stream);
int gmf_mlp_set_precision(gmf_mlp* net, int32_t precision, void* stream);
int gmf_mlp_train(gmf_mlp* net, const void* Y, int32_t y_dtype, int64_t rows, const float* target, int32_t epochs,
                  int32_t batch, float lr, uint64_t seed, float* losses, void* stream);
void gmf_mlp_free(gmf_mlp* net);

/*
 * gmf_trace -- enable (1) or disable (0) timing of the block-step tile kernels:
 * while enabled, every sweep's tile launch is bracketed by CUDA events recorded
 * on the launching stream (the strip-update launch that follows is not timed);
 * in the persistent mode (gmf_epoch_mode) the one launch of each
 * gmf_sgd_epoch / gmf_sgd_sweeps call is. gmf_trace_read synchronizes the
 * stream, returns the summed kernel time in milliseconds and the number of
 * timed launches since the last read, and resets both. Costs one event pair
 * per timed launch.
 */
int gmf_trace(gmf_model* h, int32_t enable);
int gmf_trace_read(gmf_model* h, double* total_ms, int64_t* launches, void* stream);

/*
 * gmf_deviance_noalloc -- the total deviance of gmf_deviance, for callers that
 * cannot allocate device memory: a plug-in running inside a framework that
 * owns all device memory through its own pool (a cudaMalloc of its own would
 * take memory the framework has already handed out, or is not allowed at
 * all), or a monitoring call that must not change the memory a long-running
 * fit sees. The paper has no counterpart; this is a deployment variant of
 * gmf_deviance that needs no handle and allocates nothing.
 *
 *   Y       device, n x m counts (y_dtype GMF_Y_INT32 or GMF_Y_UINT16)
 *   W       device float32 n x m weights, or NULL (all 1)
 *   L       device float32 n x ld, row i = [o_i, x_i', gamma_i', u_i', padding]
 *   R       device float32 m x ld, row j = [1, beta_j', z_j', v_j', padding]
 *   K       1 + p + q + d columns used (1..64), ld >= K
 *   family  GMF_POISSON or GMF_NEGBIN (shape alpha > 0), eta_clamp > 0
 *   d_out   device double: receives sum_ij D(y_ij, mu_ij), eta = L R'
 * Asynchronous on the stream. Its scratch is a library-owned static device
 * array of 262144 FP64 partial sums (2 MiB, held by every GPU that loads the
 * library until the process exits), so ceil(n/64) * ceil(m/64) must not exceed
 * 262144; larger sizes return GMF_ERR_ARG. The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture (a failed lookup returns GMF_ERR_CUDA, and
 * gmf_last_error() gives the CUDA error text). All calls share the array (each call overwrites
 * every slot it reads before reading it): calls that may overlap on the GPU
 * race and must be ordered by the caller (same stream, or events).
 */
int gmf_deviance_noalloc(const void* Y, int32_t y_dtype, const float* W, int64_t n, int64_t m, const float* L,
                         const float* R, int32_t K, int32_t ld, int32_t family, float alpha, float eta_clamp,
                         double* d_out, void* stream);

/*
 * Per-gene negative binomial shapes (alpha_mode 2): the model of App. B with
 * the shape made gene-specific, y_ij ~ NB(mu_ij, alpha_j), as scRNA-seq counts
 * are usually modelled (and as the synthetic laws draw them). The derivatives,
 * the deviance and the log-likelihood of entry (i, j) use alpha_j; the shapes
 * stay fixed during gmf_sgd_epoch. gmf_project_cells does not take them.
 * gmf_set_gene_shapes / gmf_get_gene_shapes -- the m shapes (host double, the
 *   caller's gene order; > 0). Synchronous. Errors: GMF_ERR_ARG, GMF_ERR_STATE
 *   (alpha_mode != 2).
 * gmf_gene_shape_moments -- App. B's moment estimator applied to each gene's
 *   column at the current parameters, alpha_j = sum_i w mu^2 /
 *   sum_i w {(y - mu)^2 - mu} over the observed entries, clipped to [eps, cap];
 *   a gene whose denominator is not positive gets cap. alpha_out: host, m
 *   doubles, the caller's gene order. Any alpha_mode (e.g. estimate the shapes
 *   from a fit with one shape, then continue with them). Synchronous. Errors:
 *   GMF_ERR_ARG, GMF_ERR_OOM, GMF_ERR_CUDA.
 */
int gmf_set_gene_shapes(gmf_model* h, const double* alpha, void* stream);
int gmf_get_gene_shapes(gmf_model* h, double* alpha, void* stream);
int gmf_gene_shape_moments(gmf_model* h, double eps, double cap, double* alpha_out, void* stream);

/*
 * gmf_gene_shape_ml -- maximum-likelihood negative binomial shape of every gene
 * with the fit's means held fixed: for gene j, alpha_j maximises the NB
 * log-likelihood of App. B (Table S1's NB density, the lgamma terms included)
 * over the gene's observed entries, weights applied. Newton's method in
 * log alpha, all genes at once: each iteration is one pass over the counts
 * forming l'_j and l''_j (digamma and trigamma differences: exact sums of
 * 1/(alpha + k) for counts below 16, shifted asymptotic series above; FP32 terms
 * with compensated sums, FP64 across threads), then per gene a Newton step
 * where l is concave in log alpha, else a unit step uphill; steps are capped at
 * 1 in log alpha and alpha is kept in [lo, hi] (a gene without overdispersion
 * goes to hi). A gene stops when its step is at most tol. start (m values,
 * caller's gene order) is the first iterate, or NULL for the fit's current
 * shapes (per gene with alpha_mode 2, else the one shape). alpha_out (host, m
 * values, caller's order) receives the estimates and iters_done (may be NULL)
 * the passes made (1 <= iters <= 200). The shapes of the fit are not changed
 * (gmf_set_gene_shapes sets them). Synchronous.
 * Errors: GMF_ERR_ARG (NULL pointers, values out of range), GMF_ERR_STATE (not
 * a negative binomial fit), GMF_ERR_OOM, GMF_ERR_CUDA, and the handle's status
 * word (GMF_ERR_TIMEOUT, GMF_ERR_NONFINITE).
 */
int gmf_gene_shape_ml(gmf_model* h, const double* start, int32_t iters, double tol, double lo, double hi,
                      double* alpha_out, int32_t* iters_done, void* stream);

/*
 * gmf_initialize -- the starting values of Sec. 4.1 in the least-squares form
 * the paper gives for high-dimensional data, written over the handle's B,
 * Gamma, U and V (X, Z, the offset, the counts and the NB shape are kept):
 *   E = log(Y + 1/2) - o 1';  B = E' X (X'X)^-1;  Gamma = (E - X B') Z (Z'Z)^-1;
 *   U = P diag(s)^(1/2), V = Q diag(s)^(1/2) from the rank-d truncated SVD
 *   P diag(s) Q' of E - X B' - Gamma Z'.
 * The n x m residual is formed in FP32 in device memory (4 n m bytes, allocated
 * and released on the stream); its products run as FP32 cuBLAS GEMMs; the
 * truncated SVD is a randomized subspace iteration (d + 10 Gaussian test
 * vectors drawn from `seed`, power_iters power steps in [0, 20], each basis
 * orthonormalised in FP64); small systems are solved in FP64 on the host. The
 * smoothed derivatives, visit counts and t restart from zero. sv_out (host, d
 * doubles, may be NULL) receives s, the residual's leading singular values (a
 * scree for rank selection, Sec. 4.2). Synchronous. Errors: GMF_ERR_ARG,
 * GMF_ERR_STATE (missing entries, X'X or Z'Z singular, a residual of rank < d),
 * GMF_ERR_OOM, GMF_ERR_CUDA.
 */
int gmf_initialize(gmf_model* h, int32_t power_iters, uint64_t seed, double* sv_out, void* stream);

/*
 * gmf_fit_loadings -- the last step of the start of Sec. 4.1: with the scores
 * U and the regression effects B, Gamma held fixed, one GLM per gene for its
 * loadings v_j, the scores as the design and o_i + x_i'beta_j + gamma_i'z_j as
 * the offset. Each gene minimises f_j(v) = 0.5 sum_i w_ij D(y_ij, mu_ij) +
 * 0.5 lambda_V |v|^2 (eq. 6 restricted to v_j; the current NB shape) by
 * Fisher scoring from the handle's V, v <- v + (U' diag(w Dddot) U +
 * lambda_V I)^-1 (U' w Ddot - lambda_V v), for n_steps passes with step
 * control: a pass whose f_j exceeds the best by more than 1e-5 (1 + |f_best|)
 * halves that gene's last step from its best point (the reading used for the
 * per-cell projection). Usually called after gmf_initialize, whose V it
 * replaces. Per pass, in chunks of rows: eta, the derivatives and the
 * deviances on the device, U' (w Ddot) and the packed Fisher matrices as FP32
 * cuBLAS GEMMs (plain library GEMMs); the d x d solves in FP64 on the host.
 * obj_out (host, may be NULL): sum_j f_j at the result. The smoothed
 * derivatives, visit counts and t restart from zero. Synchronous; allocates
 * its chunk buffers on the stream (about 2 x 16 MB). Errors: GMF_ERR_ARG
 * (n_steps outside [0, 100]), GMF_ERR_STATE (families beyond Poisson and NB,
 * missing entries), GMF_ERR_OOM, GMF_ERR_CUDA.
 */
int gmf_fit_loadings(gmf_model* h, int32_t n_steps, double* obj_out, void* stream);

/*
 * gmf_set_wait_limit -- testing hook for the failure detection of the
 * persistent epoch (GMF_FLAG_PERSIST), whose blocks wait on the global timer
 * for the earlier visits of their moving strip (gmf_strip_schedule).
 * limit_ns replaces the 2 s limit of one such wait (0 restores it; at most
 * 6e10). need_extra (>= 0) is added to every dependency count staged by later
 * gmf_sgd_epoch / gmf_sgd_sweeps calls: with need_extra > 0 no wait can be
 * satisfied, so every wait gives up after limit_ns, the launch still runs to
 * its end (no copy or MMA is left in flight), and the next synchronous call
 * (gmf_deviance, gmf_get_params) returns GMF_ERR_TIMEOUT. The handle's status
 * word keeps the flag: make a new handle to go on fitting. Other launch modes
 * do not wait on strips and ignore both values. The paper has no counterpart.
 * Errors: GMF_ERR_ARG (NULL handle, values out of range).
 */
int gmf_set_wait_limit(gmf_model* h, int64_t limit_ns, int32_t need_extra);

/*
 * gmf_set_flow_lag -- item order of the dataflow epoch (GMF_FLAG_PERSIST
 * outside cluster mode): a block's update units are queued once `lag` further
 * tile groups (blocks) have been queued after its tiles, or earlier where a
 * later tile reads what they write (0 <= lag <= 64, default 2). A larger lag
 * leaves the updates less waiting for their tiles, a smaller one frees the
 * next sweep's tiles sooner. Takes effect from the next gmf_sgd_epoch /
 * gmf_sgd_sweeps; results are bitwise the same for every lag. The paper has
 * no counterpart. Errors: GMF_ERR_ARG (NULL handle, lag out of range).
 */
int gmf_set_flow_lag(gmf_model* h, int32_t lag);

/* Release the handle and all of its device memory (NULL is allowed). */
void gmf_free(gmf_model* h);

/* Thread-local description of the last error on this thread ("" if none). */
const char* gmf_last_error(void);

/* Library version string. */
const char* gmf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GMF_H */
