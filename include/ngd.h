/*
 * ngd.h -- C ABI of libngd, the GB300 (sm_103a) hot path of matrix-free natural
 * gradient descent for PINNs with a randomized Nystrom preconditioner
 * (Bioli, Marcati, Sangalli, arXiv 2505.11638).
 *
 * Conventions shared by every entry point
 *   - Pointers named "device" are CUDA device pointers owned by the caller; the
 *     library never frees them and never keeps them beyond the call, except the
 *     problem arrays X, w, target of ngd_problem_desc, which must stay valid
 *     until ngd_destroy.  Pointers named "host" are ordinary host memory.
 *   - All device work is enqueued on the context's stream.  Calls that return a
 *     host scalar (loss, iteration count, relres, ngd_step_info) synchronise that
 *     stream before returning; every other call is asynchronous.
 *   - Every call returns an ngd_status; no C++ exception crosses the ABI.
 *     ngd_last_error(ctx) gives a one-line message for the last failure.
 *     Shapes and pointers are validated on the host (NGD_ERR_INVALID_ARG) before
 *     anything is enqueued.  Device-side failures (non-SPD core, CG breakdown,
 *     non-finite values) are recorded in a device status word and reported by
 *     the next call that synchronises.
 *   - theta, v, y, g, d and every other length-p parameter-space vector are
 *     float64.  The working precision of activations, of the Jacobian and of
 *     the p x ell matrices Omega, Y and U is the context dtype (NGD_F64: double,
 *     NGD_F32: float).  Residual-space vectors (length N) are float64.
 *   - theta layout (Sec. 2.3): layer by layer, W_l row-major (n_l x n_{l-1})
 *     followed by b_l; p = sum_l (n_l n_{l-1} + n_l).
 *   - "Linearization": calls that take theta (re)linearize the context at theta
 *     (evaluate the residuals and, in stored-Jacobian mode, form J); passing
 *     theta = NULL reuses the last linearization (for repeated matvecs).
 */
#ifndef NGD_H
#define NGD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ngd_ctx ngd_ctx;

typedef enum {
  NGD_OK = 0,
  NGD_ERR_INVALID_ARG = 1,  /* bad shape, pointer, enum or option (host check) */
  NGD_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  NGD_ERR_OOM = 3,          /* workspace allocation failed */
  NGD_ERR_NOT_SPD = 4,      /* Omega^T Y_nu not positive definite (Nystrom core) */
  NGD_ERR_BREAKDOWN = 5,    /* p^T (G + mu I) p <= 0 inside CG */
  NGD_ERR_MAXIT = 6,        /* reserved: CG stopped at maxit (reported via relres, not as an error) */
  NGD_ERR_NONFINITE = 7,    /* a NaN/Inf reached a reduction */
  NGD_ERR_TIMEOUT = 8,      /* a bounded device-side wait gave up */
  NGD_ERR_UNSUPPORTED = 9   /* valid request this build cannot serve (e.g. network too wide) */
} ngd_status;

typedef enum { NGD_F64 = 0, NGD_F32 = 1 } ngd_dtype;

/* Arithmetic of the sketch GEMMs Z = J Omega and Y = J^T (w .* Z) and of the factor:
 *   F64  FP64-accurate.  In an F64 context: FP64 CUDA cores.  In an F32 context with the stored
 *        Jacobian: the tcgen05 tensor cores on an error-free split of the FP32 operands into BF16
 *        digit planes (J by rows and Omega by columns scaled by powers of two, signed base-256
 *        digits; Z split likewise); digit products of the leading levels are summed exactly in
 *        FP32 tensor memory over K-chunks of 256 and the chunk sums in double-float, leaving
 *        ~2^-46 of the term magnitudes.  Y is float64; the factor runs in double-float (FP64-
 *        accurate) with shift nu = eps_48(||Y||_F).
 *   F32  FP32 CUDA cores with FP64 cross-tile sums; Y float32; shift eps32(||Y||_F).
 *   TF32 / BF16 tcgen05 tensor cores (operands rounded, FP32 accumulation in TMEM); Y float32;
 *        shift eps_TF32 / eps_BF16 (||Y||_F).
 *   DF   FP64-accurate like F64, on the FP32 CUDA cores: exact FP32 products summed in double-float
 *        (the same accuracy class, without tensor cores).  F32 contexts only.
 * The sampled sketch (ngd_nystrom_sketch_sampled) and the matrix-free mode form the FP64-accurate
 * products in double-float for F64 and DF alike. */
typedef enum {
  NGD_SKETCH_F64 = 0, NGD_SKETCH_F32 = 1, NGD_SKETCH_TF32 = 2, NGD_SKETCH_BF16 = 3, NGD_SKETCH_DF = 4
} ngd_sketch_prec;

/* Interior residual: Poisson  r = Delta u + f  (Eq. energy_poisson);
 *                    heat     r = u_t - kappa Delta u - f, coordinate 0 = t.
 * Boundary / initial rows: r = u - g.                                          */
typedef enum { NGD_PDE_POISSON = 0, NGD_PDE_HEAT = 1 } ngd_pde;

/* Gramian matvec strategy (Sec. 4.1.2, Table tab:matvec_costs):
 *   STORED_J     "precompute Jacobian only": J (N x p) is formed once per
 *                linearization and streamed by every matvec;
 *   MATRIX_FREE  "recompute batch Jacobian on the fly": JVP kernel, then the
 *                VJP by point blocks whose Jacobian rows are recomputed;
 *   AUTO         STORED_J when J fits mem_budget, else MATRIX_FREE.          */
typedef enum { NGD_GV_AUTO = 0, NGD_GV_STORED_J = 1, NGD_GV_MATRIX_FREE = 2 } ngd_gv_mode;

typedef struct {
  int pde;                /* ngd_pde */
  double kappa;           /* heat diffusivity (ignored for Poisson) */
  int n_layers;           /* number of affine layers L+1 (>= 2), at most 8 */
  const int* widths;      /* host, n_layers+1 entries: widths[0] = d_in (<= 16), widths[n_layers] = 1,
                             hidden widths <= 512 */
  int64_t n_int, n_bnd;   /* interior rows first, then boundary rows; N = n_int + n_bnd >= 1 */
  const double* X;        /* device, N x d_in row-major collocation points */
  const double* w;        /* device, N quadrature weights (w_r phi_r of Thm. 1) */
  const double* target;   /* device, N: source f at interior rows, boundary value g at boundary rows */
  int dtype;              /* ngd_dtype: working precision */
  int gv_mode;            /* ngd_gv_mode */
  size_t mem_budget;      /* bytes the context may use for J and stored Taylor coefficients; 0 = no limit */
  void* stream;           /* cudaStream_t the context enqueues on (NULL: legacy default stream) */
} ngd_problem_desc;

/* Test matrix of the randomized Nystrom approximation (Sec. 3, Eq. nystrom_approx):
 * NGD_TEST_GAUSSIAN    standard normal entries (Philox, see ngd_nystrom_sketch), thin QR;
 * NGD_TEST_SAMPLING    ell distinct columns of the identity, drawn one after another with
 *                      probabilities proportional to diag G among those not yet drawn
 *                      ("NystromNGD Sampling", Sec. 5), see ngd_nystrom_sketch_sampled. */
typedef enum { NGD_TEST_GAUSSIAN = 0, NGD_TEST_SAMPLING = 1 } ngd_test_matrix;

/* Direction method of the NGD step:
 * NGD_PRECOND_NYSTROM  randomized Nystrom (Alg. 4: sketch of rank ell, shift, thin SVD);
 * NGD_PRECOND_RPCHOL   RPCholesky (Alg. 5): diag G, lambda_1 by four power-method steps
 *                      (start vector: the Gaussian column with counter word 2^32 - 2), mu, block
 *                      RPCholesky F of rank at most ell (rounds of rpchol_block pivots drawn i.i.d.
 *                      proportionally to the residual diagonal, stopping when its sum is below
 *                      mu p), P = F F^T + mu I.  Pivot k of round i is the winner of the race
 *                      argmin_j -ln(u_j) / d_j with u_j from Philox at counter
 *                      (j, 2^30 + i b + k, step); pivots are made unique per round.  P^{-1} is
 *                      applied in its thin-SVD form (Eq. rpchol_svdprecond), equal to the Woodbury
 *                      form of Eq. rpchol_precond; info->ell_next returns the rank found and
 *                      info->lam1 the power-method estimate.  Needs the stored Jacobian.
 * NGD_DIRECT_FULL      no preconditioner and no pCG: NGD full (Alg. 2), the explicit Gramian
 *                      G = J^T (w .* J) (FP64-accurate), lambda_1 by the same power method, mu,
 *                      the Cholesky G + mu I = L L^T and d = L^{-T} L^{-1} g.  For p < 768 the
 *                      Cholesky is FP64 throughout; from p = 768 on it is blocked (FP64 256 x 256
 *                      diagonal blocks, trailing updates FP64-accurate to ~2^-48, the precision G
 *                      is formed in).  A numerically indefinite G + mu I is retried with 8 mu,
 *                      64 mu, ..., 8^5 mu (info->mu returns the damping used), then reported as
 *                      NGD_ERR_NOT_SPD.  ell is unused; needs the stored Jacobian and about
 *                      p^2 + 256 p float64 of device memory. */
typedef enum { NGD_PRECOND_NYSTROM = 0, NGD_PRECOND_RPCHOL = 1, NGD_DIRECT_FULL = 2 } ngd_precond;

typedef struct {
  int ell;                /* Nystrom rank (sketch size), 1 <= ell <= min(p, 2048) */
  double mu;              /* damping; mu <= 0 selects mu = gamma eps lambda_hat_1 (Alg. 4) */
  double gamma;           /* gamma of the mu rule (paper default 10) */
  double rtol;            /* PCG stop: ||r_k|| <= rtol ||g|| (recurrence residual) */
  int maxit;              /* PCG iteration cap */
  int sketch;             /* ngd_sketch_prec */
  uint64_t seed;          /* Philox key of the Gaussian test matrix */
  uint64_t step;          /* Philox counter word: fresh Omega per NGD step */
  double armijo_c1;       /* sufficient-decrease constant (default 1e-4) */
  double armijo_rho;      /* backtracking factor (default 0.5) */
  int armijo_max;         /* maximum number of trial steps (default 30) */
  double mu_loss_coef;    /* c of the adaptive damping of Sec. 5, mu = max(gamma eps lambda_hat_1,
                             c L(theta)^2) when mu <= 0 (the paper's runs: 1e-4); 0: mu = gamma eps
                             lambda_hat_1 (Alg. 4) */
  int ell_max;            /* rank adaptivity of Alg. 4: 0 = off (ell_next = ell); otherwise the cap
                             l_max >= 1 of ell_next */
  int ell_delta;          /* rank increase delta_l of Alg. 4 (the paper's runs: 20), >= 0 */
  int test_matrix;        /* ngd_test_matrix of the sketch (default NGD_TEST_GAUSSIAN) */
  int precond;            /* ngd_precond (default NGD_PRECOND_NYSTROM) */
  int rpchol_block;       /* RPCholNGD: pivots per round b (the paper: 20), 1 <= b <= ell; ell is the
                             maximum rank l_max (<= 2047), rounds floor(ell / b) */
} ngd_step_opts;

typedef struct {
  double loss_before, loss_after, alpha, mu, lam1, lam_ell, nu, relres;
  int pcg_iters, armijo_trials, shift_retries, status;
  double ms_linearize, ms_sketch, ms_factor, ms_pcg, ms_linesearch; /* CUDA-event phase times */
  int ell_next;           /* rank for the next step (Alg. 4 rule; = ell when ell_max = 0):
                             min(ell + ell_delta, ell_max) if lambda_hat_ell > 10 mu, else
                             min(i + 1, ell_max) with i the first (1-based) index of lambda_hat
                             below 10 mu (ell if there is none) */
} ngd_step_info;

/* ---------------------------------------------------------------- context */

/* Create a context for one PINN problem.  Copies the description (not X/w/target,
 * which stay caller-owned and must outlive the context), validates it, sizes and
 * allocates the workspace with cudaMalloc on the current device.
 * Errors: INVALID_ARG (bad shape/pointer), UNSUPPORTED (too wide/deep), OOM, CUDA. */
ngd_status ngd_create(const ngd_problem_desc* desc, ngd_ctx** out);

/* Free the context and its workspace (synchronises its stream).  NULL is a no-op. */
void ngd_destroy(ngd_ctx* ctx);

/* Message of the last failed call on ctx ("" if none); the string is owned by ctx. */
const char* ngd_last_error(const ngd_ctx* ctx);

/* Total number of CUDA kernels this library has launched in the calling process (all
 * contexts), for instrumentation: a caller brackets a region with two reads. */
uint64_t ngd_kernel_launches(void);

/* Number of network parameters p. */
int64_t ngd_num_params(const ngd_ctx* ctx);

/* Number of collocation points N. */
int64_t ngd_num_points(const ngd_ctx* ctx);

/* Clock-cycle limit of every bounded device-side wait of the context's tensor-core kernels
 * (mbarrier waits for TMA loads, MMAs and accumulators; default 4e9, about 2 s).  A wait that
 * runs out makes the kernel stop issuing work, wait for the loads and MMAs it already issued
 * (with the default limit), store nothing, free its tensor memory and return; the call then
 * reports NGD_ERR_TIMEOUT and the context stays usable.  A caller may shorten the limit for
 * faster failure detection.  cycles >= 1, else NGD_ERR_INVALID_ARG. */
ngd_status ngd_set_wait_limit(ngd_ctx* ctx, int64_t cycles);

/* Replace the stream the context enqueues on. */
ngd_status ngd_set_stream(ngd_ctx* ctx, void* stream);

/* ---------------------------------------------------------------- residual, JVP, VJP */

/* Residual vector and loss (Sec. 2.2.1, Eq. energy_poisson; Sec. 5.1):
 * r_r as in ngd_pde, L = 1/2 sum_r w_r r_r^2, by the fused forward-Laplacian
 * (Taylor-mode) kernel.  theta: device p (float64).  r: device N or NULL.
 * loss: host or NULL; when non-NULL the call synchronises.
 * If the context may store Taylor coefficients (mem_budget), they are kept for
 * a following ngd_vjp(ctx, NULL, ...). */
ngd_status ngd_residual(ngd_ctx* ctx, const double* theta, double* r, double* loss);

/* The network's output channels at the context's points (Sec. 2.2.1 forward Laplacian): for
 * point n, out[n * (d + 2) + c] holds u_theta (c = 0), the d first derivatives (c = 1 .. d, in
 * input order; coordinate 0 is t for NGD_PDE_HEAT) and the Laplacian over the spatial
 * coordinates (c = d + 1), computed by the same kernel as ngd_residual in the context's
 * working precision and written as float64.  Used to evaluate L2 and H1 errors against a known
 * solution on a separate set of points (a context built on those points).
 * theta: device p (float64); out: device N (d + 2) float64, caller-owned.  Asynchronous; also
 * leaves the residuals and the loss in the context as ngd_residual does.
 * Errors: INVALID_ARG (NULL pointer), UNSUPPORTED (network too wide), CUDA. */
ngd_status ngd_eval(ngd_ctx* ctx, const double* theta, double* out);

/* Jacobian-vector product Jv (forward-mode tangents of the Taylor-mode forward;
 * Thm. 1 consequence, Sec. 3.2).  v: device p, out: device N. */
ngd_status ngd_jvp(ngd_ctx* ctx, const double* theta, const double* v, double* out);

/* Vector-Jacobian product J^T c, the hand-written reverse of the residual kernel
 * (Thm. 1 consequence).  theta = NULL reuses the Taylor coefficients stored by the
 * last ngd_residual when they were kept, else recomputes them.
 * cot: device N, out: device p. */
ngd_status ngd_vjp(ngd_ctx* ctx, const double* theta, const double* cot, double* out);

/* Gradient g = grad L = J^T (w .* r) (the gradient of Alg. 1), residual r (device N or NULL)
 * and loss (host or NULL, synchronises when non-NULL).  Linearizes at theta. */
ngd_status ngd_gradient(ngd_ctx* ctx, const double* theta, double* g, double* r, double* loss);

/* ---------------------------------------------------------------- Gramian */

/* Caller-supplied Jacobian for the "precompute Jacobian only" strategy (Sec. 4.1.2): replace the
 * context's stored J by J, so that G = J^T diag(w) J (Thm. 1) is the Gramian of that J in every
 * following call that reuses the linearization (theta = NULL): ngd_gramian_mv, ngd_gramian_diag,
 * ngd_nystrom_sketch(_sampled), ngd_pcg_solve and ngd_vjp.  This lets the solver run on a
 * Jacobian computed elsewhere (another residual, another network) with the context's weights w.
 * J: device, N x p row-major with leading dimension ldJ >= p, in the context dtype (float64 for
 * NGD_F64, float32 for NGD_F32); copied (the caller keeps ownership), asynchronous.  A later call
 * with a non-NULL theta re-linearizes and overwrites it.  The residuals and loss are not changed.
 * Errors: INVALID_ARG (NULL J, ldJ < p), UNSUPPORTED (the context does not store J: matrix-free
 * mode), CUDA. */
ngd_status ngd_set_jacobian(ngd_ctx* ctx, const void* J, int64_t ldJ);

/* y = (G + mu I) v with G = J^T diag(w) J (Thm. 1, Eq. G_matrixfree) by the
 * context's matvec strategy.  theta NULL reuses the last linearization.
 * v, y: device p, must not alias.  mu >= 0. */
ngd_status ngd_gramian_mv(ngd_ctx* ctx, const double* theta, const double* v, double mu, double* y);

/* ---------------------------------------------------------------- Nystrom */

/* Sketch of App. A (Alg. randomized_nystrom): the test matrix and Y = G Omega.
 * Omega_raw = randn(p, ell) from Philox4x32-10 (key = seed, counter word = step,
 * layout in the implementation notes), Omega = thin QR factor with positive
 * diag(R) (CholeskyQR2), Y = G Omega = J^T (w .* (J Omega)) in the arithmetic
 * 'prec' (the only dense contraction of the path).
 * Omega: device, p x ell column-major (leading dimension p), context dtype.  Y: same layout,
 * float64 when prec = NGD_SKETCH_F64, else the context dtype.
 * ell <= min(p, 2048).  TF32/BF16 need an F32 context and the stored Jacobian. */
ngd_status ngd_nystrom_sketch(ngd_ctx* ctx, const double* theta, int ell, uint64_t seed, uint64_t step,
                              int prec, void* Omega, void* Y);

/* Gramian times a block of vectors, Y = G V = J^T (w .* (J V)) (Thm. 1, Eq. G_matrixfree), by the
 * same products and in the same arithmetic 'prec' as the sketch step of ngd_nystrom_sketch, for a
 * test matrix V the caller chooses (Eq. nystrom_approx holds for any V of full column rank; the
 * factor of ngd_nystrom_factor wants V orthonormal).  theta NULL reuses the linearization.
 * V: device, p x ell column-major, leading dimension ldV >= p, context dtype.  Y: device, p x ell
 * column-major, leading dimension ldY >= p, float64 when prec = NGD_SKETCH_F64, else the context
 * dtype.  1 <= ell <= min(p, 2048).  Synchronises (device status).
 * Errors: as ngd_nystrom_sketch. */
ngd_status ngd_gramian_mm(ngd_ctx* ctx, const double* theta, int ell, const void* V, int64_t ldV, int prec, void* Y,
                          int64_t ldY);

/* Gramian diagonal diag(G) = sum_r w_r (d r_r / d theta)^2 elementwise (Eq. gram_diagonal), at
 * theta (NULL: the current linearization): stored J read once, or J recomputed by point blocks
 * in matrix-free mode; FP64 accumulation over row slices added in a fixed order.
 * d: device p float64, caller-owned.  Asynchronous.  Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
ngd_status ngd_gramian_diag(ngd_ctx* ctx, const double* theta, double* d);

/* The explicit Gramian G = J^T diag(w) J (Thm. 1; the matrix NGD full, Alg. 2, factors) at the
 * linearization (theta NULL reuses the last one; stored-J contexts only).  G: device, p x p
 * column-major with leading dimension ldG >= p, float64, every entry written (symmetric: the
 * lower triangle mirrored).  FP64-accurate in both dtypes: an FP32 context forms it on the tensor
 * cores from six-digit BF16 planes of the column-scaled J^T and (diag(w) J)^T (pairs of digit
 * weight sum <= 5 kept, each pair's 256-long K chunks summed exactly, ~2^-46 of the term
 * magnitudes); an FP64 context by the double-float GEMM on the lower triangle.  Workspace of the
 * FP32 form: 12 p N bytes of digit planes and up to 8 GB of split-K partials (p^2 8 bytes per 256
 * points), kept by the context.
 * Errors: INVALID_ARG (NULL G, ldG < p, no linearization), UNSUPPORTED (matrix-free context), OOM,
 * TIMEOUT (a bounded tensor-core wait ran out), CUDA. */
ngd_status ngd_gramian_full(ngd_ctx* ctx, const double* theta, double* G, int64_t ldG);

/* Randomized Nystrom sketch with the sampling test matrix (NGD_TEST_SAMPLING): diag G, then ell
 * distinct parameter indices S by an exponential race (Efraimidis & Spirakis, 2006): the ell
 * smallest keys E_j = -ln(u_j) / (diag G)_j, ties to the smaller index, u_j the 52-bit uniform of
 * Philox4x32-10 words (x0, x1) at counter (j, 2^32 - 1, step mod 2^32, step >> 32) and key
 * (seed mod 2^32, seed >> 32) (the Gaussian test matrix never uses column 2^32 - 1); this is
 * sampling without replacement proportionally to diag G.  Omega = I[:, S] (S increasing, already
 * orthonormal), Y = G Omega = G[:, S] (stored J: a gather of the sampled Jacobian columns and
 * one product J^T (w .* J[:, S])).  Outputs as ngd_nystrom_sketch, plus idx: device ell int32,
 * S in increasing order.  Synchronises.  Errors: as ngd_nystrom_sketch; INVALID_ARG also when
 * fewer than ell entries of diag G are positive. */
ngd_status ngd_nystrom_sketch_sampled(ngd_ctx* ctx, const double* theta, int ell, uint64_t seed, uint64_t step,
                                      int prec, int* idx, void* Omega, void* Y);

/* Factor of App. A (Alg. randomized_nystrom) given an orthonormal Omega and Y = G Omega:
 * nu = eps(||Y||_F) in the format of 'prec' (spacing 2^(floor(log2 x) - m) with m = 52, 23,
 * 10, 7 mantissa bits for F64, F32, TF32, BF16; m = 48 for F64 in an F32 context, whose sketch
 * and factor run in double-float), Y_nu = Y + nu Omega, C = chol(sym(Omega^T Y_nu)) in FP64,
 * B = Y_nu C^{-1}, eigen-decomposition of B^T B in FP64 (Householder tridiagonalization,
 * multisection, twisted factorization, back-transform) gives B = U Sigma V^T, lambda = max(0, Sigma^2 - nu), descending.
 * shift_scale multiplies nu (1 = the rule above; ngd_step retries with 8, 64, ..., 8^5).
 * Omega: device p x ell (context dtype); Y: device p x ell (float64 when prec = NGD_SKETCH_F64,
 * else the context dtype); U: device p x ell out, float64 when prec = NGD_SKETCH_F64, else
 * float32 (in an F32 context the preconditioner's cancellation in I - U U^T needs U in FP64 once
 * the sketch resolves G's spectrum to FP64 level); lam: device ell float64 out, nu_out: host or
 * NULL (synchronises when non-NULL).
 * NOT_SPD when C does not exist. */
ngd_status ngd_nystrom_factor(ngd_ctx* ctx, int ell, const void* Omega, const void* Y, int prec,
                              double shift_scale, void* U, double* lam, double* nu_out);

/* Nystrom preconditioner, Alg. 4 (scaled form of Eq. nystrom_inverse):
 * z = (lam_ell + mu) U (Lambda + mu I)^{-1} U^T v + (I - U U^T) v.
 * U: device p x ell of ngd_dtype u_dtype (NGD_F64, or NGD_F32 in an F32 context), lam: device
 * ell, v, z: device p (no aliasing).  Asynchronous on the context stream. */
ngd_status ngd_precond_apply(ngd_ctx* ctx, int ell, const void* U, int u_dtype, const double* lam, double mu,
                             const double* v, double* z);

/* ---------------------------------------------------------------- solver */

/* Preconditioned CG for (G + mu I) d = g (Alg. 3; textbook pCG, x0 = 0), stopping
 * when ||r_k||_2 <= rtol ||g||_2 (recurrence residual, FP64) or after maxit
 * iterations.  ell = 0 or U = NULL runs unpreconditioned CG.  mu > 0.
 * theta NULL reuses the last linearization.  U: as for ngd_precond_apply, u_dtype its
 * ngd_dtype.  g, d: device p; iters, relres: host (the call synchronises).  Returns BREAKDOWN
 * if p^T (G + mu I) p <= 0. */
ngd_status ngd_pcg_solve(ngd_ctx* ctx, const double* theta, const double* g, double mu,
                         const void* U, int u_dtype, const double* lam, int ell, double rtol, int maxit,
                         double* d, int* iters, double* relres);

/* One Nystrom-preconditioned matrix-free NGD step (Alg. 1 with Alg. 3 and Alg. 4):
 * gradient, sketch of rank opts->ell with a fresh Omega, factor (retrying with an
 * 8x, 64x, ..., 8^5x shift on NOT_SPD), mu (fixed, the Alg. 4 rule, or the adaptive
 * max(gamma eps lambda_hat_1, c L^2) of Sec. 5), pCG, Armijo backtracking along
 * theta - alpha d, update, and the rank for the next step (info->ell_next, Alg. 4).
 * A training loop passes info->ell_next as the next step's ell.  theta: device p,
 * updated in place.  info: host or NULL.  Synchronises.
 * Errors: INVALID_ARG (bad options: ell outside [1, min(p, 2048)], ell_max < 0 or above
 * that range, ell_delta < 0, ...), NOT_SPD, BREAKDOWN, NONFINITE, CUDA. */
ngd_status ngd_step(ngd_ctx* ctx, double* theta, const ngd_step_opts* opts, ngd_step_info* info);

/* Nystrom preconditioner apply that allocates nothing.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc, e.g. applications whose device
 * memory is owned by their own pool allocator, or latency-critical loops that cannot accept the
 * device-wide synchronisation a cudaMalloc may imply.  It computes the same z as
 * ngd_precond_apply, without a context:
 *   z = (lam_ell + mu) U (Lambda + mu I)^{-1} U^T v + (I - U U^T) v.
 * dtype: ngd_dtype of U (float64 or float32); U: device, p x ell column-major with leading
 * dimension ldU >= p; lam: device ell float64 (descending); v, z: device p float64, distinct;
 * mu >= 0; stream: cudaStream_t (NULL: legacy default stream).  Asynchronous.
 * Scratch: a fixed array of NGD_NOALLOC_MAX_ELL doubles (8 KB) compiled into the library and
 * held by every GPU that loads it until the process exits; ell > NGD_NOALLOC_MAX_ELL returns
 * NGD_ERR_UNSUPPORTED, other bad arguments NGD_ERR_INVALID_ARG (no message: there is no context).
 * Devices: the array's address is cached for device ordinals below NGD_NOALLOC_MAX_DEVICES (64);
 * a call with a higher ordinal current returns NGD_ERR_UNSUPPORTED.
 * The first call on a device looks up the array's device address with that device current;
 * make that first call before any stream capture starts.  The address is cached per device
 * together with the id of the CUDA context it was found in: after a device reset (or when the
 * primary context is released and created again) the next call looks it up again, so that call
 * too must come before any stream capture.  All calls share the array and it keeps the last
 * call's contents (every call overwrites the entries it reads, so nothing needs clearing); calls
 * that overlap on the GPU (e.g. on two streams) race on it and must be serialised by the caller. */
#define NGD_NOALLOC_MAX_ELL 1024
#define NGD_NOALLOC_MAX_DEVICES 64
ngd_status ngd_precond_apply_noalloc(int dtype, int64_t p, int ell, const void* U, int64_t ldU, const double* lam,
                                     double mu, const double* v, double* z, void* stream);

/* ---------------------------------------------------------------- batching form */

/* Many independent PINN problems (networks, point sets and parameters of their own; uneven
 * point counts allowed) stepped together, as in the paper's repeated-problem experiments.
 * ngd_batch_create makes one context per description (same rules as ngd_create); every context
 * enqueues on descs[0].stream, so a batch step is one ordered stream of work.
 * ngd_batch_step runs one NGD step (Alg. 1 with Alg. 3 and Alg. 4) for every problem i, with
 * the options in opts and the Philox key opts->seed + i (a distinct test matrix per problem), in
 * three stages over the problems: every problem's gradient, sketch, factor and damping; the pCG
 * solves; every problem's line search and update.  The solves that take the fused kernel (F32
 * contexts with the stored Jacobian and a Jacobian width of the first problem's kernel variant)
 * are packed several to one cooperative launch: each solve runs on a block group sized in
 * proportion to its point count (at least what its p and ell need), with barriers of its own, so
 * that the latency-bound phases of one solve overlap the row passes over the Jacobian of the
 * others; solves are grouped longest-previous-solve first.  The number of solves per launch is
 * the batch's packing (see ngd_batch_set_packing); untuned (the default), the first batch step
 * times packings of 1, 2, 4 and 8 solves per launch on its own launches and keeps the one with
 * the least time per pCG iteration; with the environment variable NGD_AUTOTUNE_CACHE naming a
 * file, the choice is read from and stored in that JSON file under a key of the SM count, p,
 * the padded Jacobian width, the problem count and ell.  info->ms_pcg of a packed solve is the
 * time of all the batch's solves.
 * thetas: host array of n device pointers (each p_i float64, updated in place); infos: host
 * array of n entries or NULL.  Synchronises.  The first failing problem stops the step; its
 * status is returned and ngd_batch_last_error names the problem.
 * Errors: as ngd_create / ngd_step; INVALID_ARG for n < 1 or a NULL argument; TIMEOUT when a
 * packed solve's block-group barrier waited longer than the context's wait limit. */
typedef struct ngd_batch ngd_batch;
ngd_status ngd_batch_create(const ngd_problem_desc* descs, int n, ngd_batch** out);
void ngd_batch_destroy(ngd_batch* batch);
int ngd_batch_size(const ngd_batch* batch);
ngd_ctx* ngd_batch_context(ngd_batch* batch, int i);   /* problem i's context (NULL if out of range) */
const char* ngd_batch_last_error(const ngd_batch* batch);
ngd_status ngd_batch_step(ngd_batch* batch, double* const* thetas, const ngd_step_opts* opts, ngd_step_info* infos);
/* Solves per cooperative launch of later batch steps: 0 = tune on the next step (see above),
 * 1 = one solve per launch on the whole GPU, k > 1 = up to k solves per launch (fewer when their
 * minimum block groups do not fit).  0 <= solves_per_launch <= 64, else INVALID_ARG. */
ngd_status ngd_batch_set_packing(ngd_batch* batch, int solves_per_launch);
int ngd_batch_packing(const ngd_batch* batch);          /* current packing (0: not tuned yet) */
int ngd_batch_solve_launches(const ngd_batch* batch);   /* packed-solve launches of the last step */

/* Default options: ell 100, mu 0 (rule), gamma 10, rtol 1e-6, maxit 500, FP64-accurate sketch
 * (NGD_SKETCH_F64) in every context (in an F32 context the TF32 / BF16 sketches force a shift of
 * their own eps that truncates the captured spectrum, so PCG needs many more iterations at small
 * mu: they are opt-in), seed 0, step 0, c1 1e-4, rho 0.5, 30 trials, mu_loss_coef 0, ell_max 0
 * (fixed rank), ell_delta 20, Gaussian test matrix, Nystrom preconditioner, rpchol_block 20. */
void ngd_default_step_opts(ngd_step_opts* opts);

#ifdef __cplusplus
}
#endif
#endif /* NGD_H */
