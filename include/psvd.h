/*
 * psvd -- SVD of batched tall matrices through the polar decomposition,
 * with a numerically stable (regularized) backward pass.  GB300 (sm_103a).
 *
 * The method ("Fast Differentiable SVD on GPU via Polar Decomposition"):
 *   forward  (Algorithm 1): normalize M (Algorithm 2), compute the polar factor W
 *            by odd-cubic polynomial iterations X <- X (c1 I + c3 X^T X) (CANS,
 *            Appendix A.4 / B.8), H = (W^T M)_sym, EVD H = V Sigma V^T, U = W V,
 *            QR of U if a column norm of U is off 1 by more than eps_qr
 *            (Appendix A.2).
 *   backward (Algorithm 4): the regularized polar + EVD pseudo-gradient,
 *            evaluated from the cached factors only (no iterate is stored).
 *
 * Conventions for every entry point
 *  - Matrices are row-major and batch-contiguous: element (b, i, j) of an
 *    m x n batch lives at p[b*m*n + i*n + j].  m >= n >= 1, batch >= 1
 *    (callers transpose wide matrices and swap U and V).
 *  - Every pointer argument is a DEVICE pointer owned by the caller unless its
 *    comment says otherwise; the library never frees or retains it.
 *  - The library allocates no memory: every call takes a caller-owned device
 *    workspace of at least psvd_*_workspace_bytes(...) bytes, 256-byte aligned.
 *  - All work is enqueued on `stream` (a cudaStream_t passed as void*; NULL =
 *    legacy default stream).  Unless stated otherwise calls are asynchronous: they
 *    never wait for the GPU, the return value reports argument and launch errors only,
 *    and per-matrix outcomes land in the device-side psvd_info array.  Iterations
 *    whose length is decided on the GPU (the polar steps, the learned schedule's
 *    conservative rerun in psvd_polar_fwd) are enqueued for their whole step budget;
 *    launches that find nothing left to do return at once.  psvd_svd_fwd is the one
 *    call that synchronizes (see there).
 *  - Calls on the same workspace must not overlap on the GPU.
 */
#ifndef PSVD_H
#define PSVD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define PSVD_OK                 0
#define PSVD_NOT_CONVERGED      1   /* iteration cap reached; outputs still written   */
#define PSVD_ERR_ARG           -1   /* bad size, m < n, null required pointer, ...    */
#define PSVD_ERR_WORKSPACE     -2   /* ws_bytes smaller than the query says           */
#define PSVD_ERR_NONFINITE     -3   /* input had NaN/Inf; outputs are NaN-filled      */
#define PSVD_ERR_CUDA          -4   /* a CUDA launch/runtime call failed               */
#define PSVD_ERR_TIMEOUT       -5   /* a bounded device-side wait expired             */
#define PSVD_ERR_UNSUPPORTED   -6   /* device is not sm_103 / sm_100 class            */

/* ---- options ----------------------------------------------------------- */
#define PSVD_PREC_FP32       0   /* every product FP32-accurate (split hi+lo TF32, "3xTF32") */
#define PSVD_PREC_MIXED      1   /* TF32 steps -> 3xTF32 polish, switched per matrix from the
                                    measured orthogonality residual; with the learned
                                    schedule, bounds below PSVD_MIXED_LB_MIN start at 3xTF32 */
#define PSVD_PREC_MIXED_BF16 2   /* BF16 early steps -> TF32 -> 3xTF32 polish; the BF16
                                    rounding leaves a rotation that the eigenbasis correction
                                    undoes only to first order (reconstruction ~1e-5 at
                                    n = 4096, kappa = 10)                                    */

#define PSVD_SCHED_CANS     0 /* conservative CANS: preprocessing for [t,1] then greedy
                                 optimal cubics from [1-delta, 1+delta] (Appendix B.8)     */
#define PSVD_SCHED_LEARNED  1 /* greedy optimal cubics from [l_b, 1], l_b a predicted lower
                                 bound of sigma_min(X0) per matrix (opts.lower_bound), each
                                 applied to x / 1.01 while the interval is wider than 1e-2
                                 (undamped, they lose accuracy from small bounds: ~2e-4
                                 relative reconstruction at kappa = 1e6)                     */
#define PSVD_SCHED_NS       2 /* classical Newton-Schulz, p(x) = 1.5 x - 0.5 x^3           */
#define PSVD_SCHED_PE       3 /* comparison schedule of the polar-iteration ablation (Appendix B),
                                 Polar-Express style: the greedy optimal cubics from [l_b, 1]
                                 (opts.lower_bound), each applied to x / 1.01 until that stops
                                 shrinking the interval (the damped fixed point, ~1.5e-4 from
                                 1), then undamped.  No budget, no conservative rerun.        */

typedef struct psvd_opts {
    int    precision;     /* PSVD_PREC_*                                        default 0    */
    int    schedule;      /* PSVD_SCHED_*                                       default 0    */
    double delta;         /* CANS delta (Appendix B.8)                          default 0.99 */
    int    pre_iters;     /* CANS preprocessing steps                           default 2    */
    int    max_iter;      /* cap on main polynomial steps (Appendix A.4)        default 50   */
    double tol;           /* stop when ||X^T X - I||_F / sqrt(n) <= tol         default 1e-5 */
    double eps_qr;        /* QR fallback threshold on | ||U_i|| - 1 |           default 1e-5 */
    const float *lower_bound; /* DEVICE [batch]: schedule 1's lower bounds (NULL otherwise) */
    int    budget;        /* schedule 1: steps allowed before the conservative rerun
                             (0 = automatic: predicted steps + 5)                           */
    double *res_history;  /* DEVICE [(max_iter + pre_iters + 1) x batch] or NULL: entry
                             k * batch + b receives ||X_k^T X_k - I||_F / sqrt(n) at step k
                             of matrix b (0 once it has finished; psvd_polar_fwd with schedule
                             1: the conservative rerun's steps for the matrices it reran)     */
    int    preqr;         /* 1: for m > n, factor M = Q R first (blocked Householder QR on the
                             GPU, psvd_qr), run the method on the n x n factor R and return
                             U = Q U_R (svd_fwd) or W = Q W_R, H = H_R (polar_fwd) -- the QR
                             preprocessing of rectangular inputs of Section 4.1.  A learned
                             schedule's lower bounds then refer to R.  0 (default): the
                             method runs on M itself.  Needs m <= 23040; psvd_polar_fwd_noalloc
                             rejects it.                                                      */
} psvd_opts;

/* Fills *o with the defaults above (host pointer). */
void psvd_default_opts(psvd_opts *o);

/* Per-matrix outcome, written to a DEVICE array of `batch` records. */
typedef struct psvd_info {
    int   status;          /* PSVD_OK, PSVD_NOT_CONVERGED, PSVD_ERR_NONFINITE, or (svd_fwd)
                              PSVD_ERR_TIMEOUT if a bounded device wait expired          */
    int   iters;           /* polynomial steps applied                                  */
    int   qr_fallback;     /* 1 if U was re-orthogonalized by QR (Algorithm 1's QR fallback) */
    int   sched_fallback;  /* 1 if the learned schedule missed tol and the conservative
                              schedule was rerun                                          */
    int   prec_fallback;   /* svd_fwd, mixed precision: 1 if a check below failed and the
                              matrix was recomputed on the FP32-accurate path            */
    int   steps_bf16;      /* steps taken in each precision (mixed path)                 */
    int   steps_tf32;
    int   steps_3xtf32;
    float ortho_resid;     /* final ||W^T W - I||_F / sqrt(n)                            */
    float scale;           /* sqrt(||M||_1 ||M||_inf) of Algorithm 2                     */
    float corr_max;        /* svd_fwd, mixed precision: max |X_ij| of the rotation that
                              the eigenbasis correction applied (0 otherwise)           */
    float recon_est;       /* svd_fwd, mixed precision: ||A - U S V^T||_F / ||A||_F of the
                              mixed result, estimated from 8 Rademacher probe vectors
                              (Hutchinson's estimator, float-float sums; 0 otherwise)   */
} psvd_info;

/* Mixed-precision svd_fwd keeps a matrix's BF16/TF32 result only while both checks
 * hold, and recomputes it on the FP32-accurate path otherwise (prec_fallback = 1):
 *  - corr_max <= PSVD_MIXED_CORR_MAX: the eigenbasis correction is first order, and
 *    rotations this large leave it outside its range of validity;
 *  - recon_est <= PSVD_MIXED_RECON_MAX, half the FP32 reconstruction gate of 1e-5: this
 *    sees the dense second-order error of the correction (whose largest entry stays
 *    small while its norm grows like sqrt(n) times it -- BF16 steps at n = 4096), and,
 *    for m > n, the part of A that the low-precision steps left outside the polar
 *    factor's column space (the steps multiply X on the right and never repair it). */
#define PSVD_MIXED_CORR_MAX 2e-3
#define PSVD_MIXED_RECON_MAX 5e-6

/* PSVD_PREC_MIXED with the learned schedule: a matrix whose lower bound (opts.lower_bound,
 * in units of X0 = M / sqrt(||M||_1 ||M||_inf)) is below PSVD_MIXED_LB_MIN starts on the
 * 3xTF32 rung.  TF32 steps at such small singular values leave corrections above
 * PSVD_MIXED_CORR_MAX, and the matrix would be recomputed anyway (measured at n = 4096:
 * kappa = 1e2 keeps its TF32 result, kappa = 1e3 and above fall back).  steps_tf32 = 0
 * in psvd_info shows that the gate applied. */
#define PSVD_MIXED_LB_MIN 5e-5

/* ---- workspace queries ---------------------------------------------------- */
size_t psvd_polar_workspace_bytes(int64_t batch, int64_t m, int64_t n, const psvd_opts *opts);
size_t psvd_svd_workspace_bytes(int64_t batch, int64_t m, int64_t n, const psvd_opts *opts);
size_t psvd_svd_bwd_workspace_bytes(int64_t batch, int64_t m, int64_t n);
size_t psvd_polar_bwd_workspace_bytes(int64_t batch, int64_t m, int64_t n);
size_t psvd_eigh_workspace_bytes(int64_t batch, int64_t n);

/* ---- forward ----------------------------------------------------------------
 * psvd_polar_fwd -- right polar decomposition M = W H (Definition 2.1) by
 *   Algorithm 1, polar-factor part: W (m x n, W^T W = I) and H = (W^T M)_sym (n x n, FP64
 *   symmetrization, stored FP32).  A: batch x m x n input (read only).
 *   W: batch x m x n out.  H: batch x n x n out (may be NULL).  info: batch records.
 */
int psvd_polar_fwd(const float *A, float *W, float *H, int64_t batch, int64_t m, int64_t n,
                   const psvd_opts *opts, void *ws, size_t ws_bytes, psvd_info *info,
                   void *stream);

/* psvd_polar_fwd_noalloc -- psvd_polar_fwd for callers that cannot allocate device
 *   memory (no counterpart in the paper): a real-time loop whose allocator calls are
 *   forbidden because they can block or fragment memory, an embedding that hands all
 *   device memory to its own memory manager, or a plugin that is given only its input
 *   and output buffers.  Same arguments, checks and results as psvd_polar_fwd minus
 *   the workspace: the scratch is a fixed device array inside the library, of
 *   psvd_polar_noalloc_capacity() bytes (64 MiB), held on every GPU that loads the
 *   library until the process exits.  A problem whose psvd_polar_workspace_bytes exceeds
 *   it is rejected with PSVD_ERR_WORKSPACE before any work (psvd_last_error gives the
 *   needed and available bytes).  The first call on each device (and the first after a
 *   cudaDeviceReset) looks up the array's device address with that device current.
 *   Every call shares the one array and leaves its
 *   contents behind (each call clears what it needs), so calls that overlap on the GPU
 *   -- other streams, other host threads -- race; serialize them.  Calls no
 *   cudaMalloc/cudaFree and no allocating library routine. */
int psvd_polar_fwd_noalloc(const float *A, float *W, float *H, int64_t batch, int64_t m, int64_t n,
                           const psvd_opts *opts, psvd_info *info, void *stream);
size_t psvd_polar_noalloc_capacity(void);

/* psvd_svd_fwd -- thin SVD M = U Sigma V^T by Algorithm 1.
 *   U: batch x m x n, S: batch x n (descending, >= 0 up to rounding), VT: batch x n x n
 *   (rows are right singular vectors; each V column's largest-|.| entry is positive).
 *   The call synchronizes `stream` once, after its first pass, to read the per-matrix
 *   flags: the column-norm check of Algorithm 1 (those matrices get the QR fallback) and,
 *   in the mixed modes or with the learned schedule, the checks above and the learned
 *   schedule's misses (those matrices are recomputed on the plain FP32-accurate path, whose
 *   own QR decision is one more synchronization when it has matrices to recompute).  The
 *   fallbacks, rare by construction, then run only for the matrices that need them. */
int psvd_svd_fwd(const float *A, float *U, float *S, float *VT, int64_t batch, int64_t m,
                 int64_t n, const psvd_opts *opts, void *ws, size_t ws_bytes,
                 psvd_info *info, void *stream);

/* psvd_eigh -- symmetric EVD H = V diag(S) V^T (the EVD of Algorithm 1) of a batch of
 *   n x n symmetric matrices (only the upper triangle is read).  S descending,
 *   VT rows = eigenvectors with the sign convention above. */
int psvd_eigh(const float *Hs, float *S, float *VT, int64_t batch, int64_t n,
              void *ws, size_t ws_bytes, void *stream);

/* psvd_eigh_dc -- the same EVD by spectral divide and conquer on the polar decomposition,
 *   nearly all of it products on the tensor cores: W = sign(H - mu I) as the polar factor of
 *   H - mu I by the CANS iteration of Algorithm 1 (mu = the midpoint of the two middle
 *   entries of diag(H)), the projector P = (I + W)/2, orthonormal bases V1, V2 of range(P)
 *   and range(I - P) as polar factors of P Omega and (I - P) Omega' (Omega a fixed seeded
 *   Gaussian) refined once through P, then the halves V1^T H V1 and V2^T H V2 recursively,
 *   with blocks of at most 512 rows (or below depth 6), and blocks within 1e-5 of a multiple
 *   of I, solved by the tridiagonal eigensolver of psvd_eigh; V = [V1 Z1, V2 Z2].  Same
 *   outputs and conventions as psvd_eigh.  The matrices of the batch are solved in turn, and
 *   the call synchronizes `stream` twice at every split (it reads diag(H) with the largest
 *   off-diagonal magnitude, then trace(P)).  Workspace: psvd_eigh_dc_workspace_bytes(n), for
 *   one matrix at a time. */
size_t psvd_eigh_dc_workspace_bytes(int64_t n);
int psvd_eigh_dc(const float *Hs, float *S, float *VT, int64_t batch, int64_t n, void *ws,
                 size_t ws_bytes, void *stream);

/* ---- backward ----------------------------------------------------------------
 * psvd_svd_bwd -- Algorithm 4's backward pass from the cached factors:
 *   W = U V^T, Wbar = Ubar V^T, Vbar_tot = Vbar + W^T Ubar,
 *   B = (V^T Vbar_tot - Vbar_tot^T V)/2, Hbar = V (diag(Sbar) + K_eps^T o B) V^T,
 *   R_eps = V Sigma (Sigma^2 + eps^(1/2))^-1 V^T, C = (Hbar - R_eps M^T Wbar R_eps)_sym,
 *   X = V (T_eps o V^T C V) V^T, Mbar = Wbar R_eps + 2 M X.
 *   dU / dS / dVT are the incoming gradients of U, S and V^T; any may be NULL (zero).
 *   kreg_mode selects K_eps: 0 = (s_i-s_j)/((s_i-s_j)^2 + eps^(1/2)) as in Algorithm 4,
 *   1 = (s_i-s_j)/((s_i-s_j)^2 + eps^2) as in Section 5.2, 2 = exact 1/(s_i-s_j) with
 *   ties (|s_i-s_j| <= 1e-6 s_max) masked and eps = 0 in R and T.
 *   dA: batch x m x n out. */
int psvd_svd_bwd(const float *A, const float *U, const float *S, const float *VT,
                 const float *dU, const float *dS, const float *dVT, float *dA,
                 int64_t batch, int64_t m, int64_t n, double eps, int kreg_mode,
                 void *ws, size_t ws_bytes, void *stream);

/* psvd_polar_bwd -- Algorithm 3 (Proposition 3.2): from M, W, H and the incoming
 *   gradients dW (m x n, may be NULL) and dH (n x n, may be NULL; its symmetric part
 *   is used), computes the EVD of H and
 *   Mbar = Wbar H_eps^-1 + 2 M V (T_eps o V^T B V) V^T with
 *   B = (Hbar - H_eps^-1 M^T Wbar H_eps^-1)_sym.  eps = 0 gives Theorem 3.1. */
int psvd_polar_bwd(const float *A, const float *W, const float *H, const float *dW,
                   const float *dH, float *dA, int64_t batch, int64_t m, int64_t n,
                   double eps, void *ws, size_t ws_bytes, void *stream);

/* psvd_eigh_bwd -- the EVD pseudo-gradient of Theorem 4.3 for H = V diag(S) V^T (as returned
 *   by psvd_eigh): Hbar = V (diag(Sbar) + 1/2 K^T o (V^T Vbar - Vbar^T V)) V^T, with
 *   Vbar = dVT^T the gradient of V.  kreg_mode selects K as for psvd_svd_bwd: 0 = Tikhonov
 *   K_eps with eps^(1/2) (Algorithm 4's form), 1 = K_eps with eps^2 (Section 5.2's form),
 *   2 = exact 1/(s_i - s_j) with ties (|s_i - s_j| <= 1e-6 s_max) masked (eps must then be 0,
 *   and eps > 0 otherwise).  S: batch x n, VT: batch x n x n (rows = eigenvectors);
 *   dS (batch x n) and dVT (batch x n x n) may be NULL (zero).  dH: batch x n x n out
 *   (symmetric).  Three split-TF32 products of n^3 each. */
size_t psvd_eigh_bwd_workspace_bytes(int64_t batch, int64_t n);
int psvd_eigh_bwd(const float *S, const float *VT, const float *dS, const float *dVT, float *dH,
                  int64_t batch, int64_t n, double eps, int kreg_mode, void *ws, size_t ws_bytes,
                  void *stream);

/* ---- learned schedule (the lower-bound predictor) ---------------------------
 * psvd_sketch_features -- 8 features per matrix of X0 = M / sqrt(||M||_1 ||M||_inf):
 *   logs of Hutchinson estimates of tr(G^k)/n, k = 1..4 (G = X0^T X0) with the caller's
 *   Rademacher probes Z (DEVICE, batch x n x s, entries +-1), log(||X0||_F^2 / n),
 *   log(f4/f3), log(n)/10, log(m/n).  F: batch x 8 out.  ws as for svd_bwd. */
int psvd_sketch_features(const float *A, const float *Z, int64_t s, float *F, int64_t batch,
                         int64_t m, int64_t n, void *ws, size_t ws_bytes, void *stream);
size_t psvd_sketch_workspace_bytes(int64_t batch, int64_t m, int64_t n, int64_t s);

/* psvd_mlp_fwd -- y = W3 relu(W2 relu(W1 f + b1) + b2) + b3 for F (nb x 8); params is
 *   one DEVICE float array [W1 64x8 | b1 64 | W2 64x64 | b2 64 | W3 1x64 | b3 1]
 *   (PSVD_MLP_NPARAMS floats).  Y: nb out. */
#define PSVD_MLP_NPARAMS (64 * 8 + 64 + 64 * 64 + 64 + 64 + 1)
int psvd_mlp_fwd(const float *params, const float *F, float *Y, int64_t nb, void *stream);

/* psvd_mlp_lower_bound -- the lower bound the learned schedule takes (opts.lower_bound):
 *   LB[i] = margin * exp(y_i), y = psvd_mlp_fwd(params, F), clamped to [1e-12, 0.999].
 *   The network predicts log sigma_min(X0); margin (> 0, from a held-out quantile of the
 *   over-prediction) makes it a lower bound for most matrices, and the conservative rerun
 *   covers the rest.  LB: DEVICE, nb floats out. */
int psvd_mlp_lower_bound(const float *params, const float *F, float *LB, int64_t nb, float margin, void *stream);

/* psvd_mlp_train_step -- one Adam step on 0.5 mean (y - target)^2 over the batch.
 *   grads (PSVD_MLP_NPARAMS floats), m1/m2 (Adam moments, same size) are DEVICE
 *   buffers; `step` is the 1-based Adam step count.  loss: DEVICE float out (may be NULL). */
int psvd_mlp_train_step(float *params, float *grads, float *m1, float *m2, const float *F,
                        const float *target, int64_t nb, float lr, int step, float *loss,
                        void *stream);
/* psvd_mlp_grad -- loss and gradients only (no parameter update). */
int psvd_mlp_grad(const float *params, const float *F, const float *target, int64_t nb,
                  float *grads, float *loss, void *stream);

/* Training helpers (all DEVICE arrays; F is nb x 8 row-major).
 * psvd_mlp_standardize -- stats[0..7] = per-feature mean, stats[8..15] = sample standard
 *   deviation (floored at 1e-6), and, if Fs is not NULL, Fs = (F - mean) / std (nb x 8).
 * psvd_mlp_fold -- makes a network trained on standardized features act on raw ones:
 *   W1 <- W1 / std (per input feature), b1 <- b1 - W1 mean (with the new W1).
 * psvd_mlp_gather -- minibatch rows Fb[i] = F[idx[i]], tb[i] = target[idx[i]], i < nb.
 * psvd_mlp_calibrate -- the learned bound's safety margin: Y = the network's predictions on F
 *   (nb floats, out), q = the `quantile` (in [0, 1]) of the over-prediction Y - target
 *   (linear interpolation between order statistics), margin[0] = exp(-max(q, 0)). */
int psvd_mlp_standardize(const float *F, int64_t nb, float *Fs, float *stats, void *stream);
int psvd_mlp_fold(float *params, const float *stats, void *stream);
int psvd_mlp_gather(const float *F, const float *target, const int *idx, int64_t nb, float *Fb,
                    float *tb, void *stream);
int psvd_mlp_calibrate(const float *params, const float *F, const float *target, int64_t nb,
                       float quantile, float *Y, float *margin, void *stream);

/* ---- QR (Appendix A.2's fallback; Section 4.1's preprocessing) ------------------
 * psvd_qr -- thin QR A = Q R of a batch of m x n matrices (m >= n), diag(R) >= 0, by blocked
 *   Householder: panels of 64 (or 32) columns factored by one thread-block cluster per
 *   matrix, trailing updates and the accumulation of Q in compact-WY form on the split-TF32
 *   tcgen05 product kernel.  A: batch x m x n (read); Q: batch x m x n out (may alias A);
 *   R: batch x n x n out, upper triangular (may be NULL).  m <= 23040. */
size_t psvd_qr_workspace_bytes(int64_t batch, int64_t m, int64_t n);
int psvd_qr(const float *A, float *Q, float *R, int64_t batch, int64_t m, int64_t n, void *ws,
            size_t ws_bytes, void *stream);

/* ---- building block ------------------------------------------------------------
 * psvd_gemm_tn -- D[b] = A[b] B[b]^T for A: batch x M x K, B: batch x N x K, D: batch x M x N
 *   (all row-major, contiguous) on the tcgen05 tensor cores; the single product kernel
 *   behind every matrix multiplication of Algorithms 1 and 4 (Gram X^T X, X p(X^T X),
 *   W^T M, W V and the backward chain).  precision: 0 = BF16 operands, 1 = TF32
 *   operands, 2 = split hi+lo TF32 (FP32-accurate).  FP32 accumulation. */
size_t psvd_gemm_workspace_bytes(int64_t batch, int64_t M, int64_t N, int64_t K);
int psvd_gemm_tn(const float *A, const float *B, float *D, int64_t batch, int64_t M, int64_t N,
                 int64_t K, int precision, void *ws, size_t ws_bytes, void *stream);

/* ---- misc ------------------------------------------------------------------ */
const char *psvd_status_string(int status);
/* Where the most recent PSVD_ERR_CUDA of this process came from (CUDA error name and
 * source location), or "" if none; a static string owned by the library. */
const char *psvd_last_error(void);
/* Number of kernels this library has launched in the calling process (all threads). */
uint64_t psvd_kernel_launch_count(void);

/* Test hook for failure detection (no counterpart in the paper): every grid barrier of the
 * cooperative kernels (the tridiagonalization, the unblocked QR) polls at most `polls` times
 * before it records PSVD_ERR_TIMEOUT and lets its CTA run on, so that every CTA returns; 0
 * restores the default (2^24 polls).  The product kernel's pipeline waits are not affected.
 * An expired wait turns the status of every psvd_svd_fwd record into PSVD_ERR_TIMEOUT (the
 * outputs of that call are then garbage).  Process-wide; takes effect at the next call. */
int psvd_debug_set_barrier_spin(uint32_t polls);

/* Measurement hooks (no counterpart in the paper; used by the benchmark's roofline).
 * psvd_profile_enable(1) makes every launch of the tcgen05 product kernel and of the
 * tridiagonalization record a pair of CUDA events on its stream (up to 8192 launches;
 * the call creates the events once), 0 turns it off.  psvd_profile_read fills
 * 4 * PSVD_PROF_CLASSES doubles: for class c -- out[4c] launches, out[4c+1] summed
 * kernel milliseconds, out[4c+2] summed algorithmic work, out[4c+3] longest launch in ms
 * -- then clears the record.  Work is flops for the product kernel (2MNK; M(M+1)K for
 * the symmetric Gram) and bytes for the tridiagonalization (its step k reads and
 * writes the (n-k-2)^2 trailing entries: sum over k of 8 (n-k-2)^2 per matrix).  Host
 * pointer; synchronizes on the recorded events. */
#define PSVD_PROF_BF16     0   /* product kernel, BF16 operands        */
#define PSVD_PROF_TF32     1   /* product kernel, TF32 operands        */
#define PSVD_PROF_TF32X3   2   /* product kernel, split-TF32 operands  */
#define PSVD_PROF_MIXED    3   /* product kernel, per-matrix precision */
#define PSVD_PROF_TRD      4   /* tridiagonalization (eigh stage 1)    */
#define PSVD_PROF_CLASSES  5
int psvd_profile_enable(int on);
int psvd_profile_read(double *out);

#ifdef __cplusplus
}
#endif
#endif /* PSVD_H */
