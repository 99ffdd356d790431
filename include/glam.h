/*
 * glam.h -- C ABI of libglam: the GD-PG penalized GLAM solver on one GB300 GPU (sm_103a).
 *
 * Method: Lund, Vincent & Hansen, "Penalized estimation in large-scale generalized linear
 * array models".  The design matrix X = X_3 (x) X_2 (x) X_1 (Sec. 2, Eq. fivenew) is never
 * formed: the linear predictor is the array transform H (Sec. 6.1, Eq. eighteen, built from
 * the rotated H-transform rho of App. A) and the gradient uses its transpose G (Eq. nineteen).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Arrays.  A paper array of size n1 x n2 x n3 is stored flattened by the vec map of App. A
 *   (Eq. index: column-major, i1 fastest), which is a C-order (n3, n2, n1) array.  The
 *   parameter array Theta (p1 x p2 x p3) is a C-order (p3, p2, p1) array.  A marginal design
 *   X_j (n_j x p_j) is stored column-major, as R stores it: element (i, k) sits at
 *   X[j][k * n_j + i] (a C-order (p_j, n_j) array).
 * Element type.  double for a GLAM_FP64 plan; float (IEEE binary32) for the GLAM_FP32,
 *   GLAM_TF32 and GLAM_BF16 plans (the precision names the arithmetic of the mode products,
 *   not the storage).  Scalars marked "double" are always double.
 * Memory.  Every array argument is a DEVICE pointer owned by the caller, unless marked HOST.
 *   The library never frees caller memory.  All workspace lives in the opaque plan, allocated
 *   by glam_plan_create and released by glam_plan_destroy.
 * Streams.  Work is enqueued on the plan's stream (glam_plan_create / glam_plan_set_stream).
 *   Calls that return only device results are asynchronous; calls that fill HOST outputs
 *   (glam_fit_path) synchronize the stream before returning.
 * Errors.  Every function returns a status (GLAM_OK = 0).  No exception crosses the ABI.
 *   On failure glam_last_error(plan) returns a message (for glam_plan_create failures, and
 *   for calls given a NULL plan, use glam_last_error(NULL): the calling thread's last error).
 * Families.  GLAM_GAUSSIAN_IDENTITY, GLAM_POISSON_LOG, GLAM_BINOMIAL_LOGIT (canonical links) and
 *   GLAM_GAMMA_LOG (Gamma with dispersion 1 and log link, not canonical; Sec. 6.4 names the four).
 *   Binomial: y_i is a proportion in [0, 1] of a_i trials (a_i the observation weight).
 * Objective.  F(theta) = f(theta) + lambda * sum_m w_m |theta_m| with f = -(1/n) l, l the
 *   weighted log-likelihood of Sec. 2, Eq. (two), n = n1 n2 n3 counting every cell (masked
 *   ones included).  Constants: Gaussian f = (1/2n) sum a_i (y_i - eta_i)^2; Poisson
 *   f = (1/n) sum a_i (exp(eta_i) - y_i eta_i) (the sum of a_i log y_i! is dropped); binomial
 *   f = (1/n) sum a_i (log(1 + exp(eta_i)) - y_i eta_i) (binomial coefficients dropped); Gamma
 *   f = (1/n) sum a_i (y_i exp(-eta_i) + eta_i) (terms in y alone dropped).
 * Observation weights W (the paper's a_i, Sec. 6.4 "Weights") are >= 0; a_i = 0 masks a cell
 *   (Sec. 4.3).  Penalty weights pen_w (omega_m) must be > 0.
 */
#ifndef GLAM_H
#define GLAM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define GLAM_OK 0
#define GLAM_EINVAL 1     /* bad argument: NULL pointer, bad dims, bad enum, unsupported combination */
#define GLAM_ENOMEM 2     /* device or host allocation failed */
#define GLAM_ECUDA 3      /* a CUDA runtime call failed; the message names it */
#define GLAM_ENONFINITE 4 /* non-finite input, or a non-finite accepted iterate (Poisson overflow) */
#define GLAM_ENOCONV 5    /* an iteration cap was reached before the KKT tolerance */
#define GLAM_ETIMEOUT 6   /* a bounded device-side wait gave up */

/* ---- families (App. B) ---- */
#define GLAM_GAUSSIAN_IDENTITY 0
#define GLAM_POISSON_LOG 1
#define GLAM_BINOMIAL_LOGIT 2
#define GLAM_GAMMA_LOG 3

/* ---- arithmetic of the mode products ---- */
#define GLAM_FP64 0
#define GLAM_FP32 1
#define GLAM_TF32 2
#define GLAM_BF16 3

typedef struct glam_plan glam_plan;

/* Grid and basis sizes.  d = 3, or d = 2 with n[2] = p[2] = 1 (then X[2] may be NULL). */
typedef struct {
  int32_t d;
  int64_t n[3]; /* n1, n2, n3: grid points per dimension */
  int64_t p[3]; /* p1, p2, p3: basis functions per dimension */
} glam_dims;

/* The quadratic model h of Sec. 3.2, Eq. (twentyfour), at an anchor Theta_k (Alg. 1, step 2-3).
 * Caller-owned device buffers, filled by glam_quad_build:
 *   V    n elements: IRLS weights w_i = a_i theta'(eta_i) (g^-1)'(eta_i) (App. B, Eq. weights,
 *        times the observation weight a_i);
 *   VZ   n elements: V (.) Z, Z the working response of Eq. (ten);
 *   b    p elements: G(V (.) Z) = X^T W z (Sec. 6.1, Eq. twentyeight);
 *   Lhat 1 double:   the Lipschitz bound max(w)/n * prod_j rho(X_j^T X_j) (Prop. 1). */
typedef struct {
  void* V;
  void* VZ;
  void* b;
  double* Lhat;
} glam_quad;

/* Options of glam_fit_path.  glam_opts_default fills the defaults given below. */
typedef struct {
  double tol;              /* KKT residual target per lambda (default 1e-6), see glam_stats.kkt */
  double lambda_min_ratio; /* auto path: lambda_min = ratio * lambda_max, in (0, 1] (default 1e-3) */
  double inner_forcing;    /* inner PG stop: max_m |x+_m - y_m| / delta <= s * lambda_max with
                              s = max(inner_floor * tol, inner_forcing * r_k), r_k the KKT residual
                              at the outer iterate (defaults 1e-2 and 0.1) */
  double inner_floor;
  double armijo_alpha0;    /* Armijo rule of Sec. 5: alpha = alpha0 * b^j (default 1) */
  double armijo_b;         /* (default 0.5) */
  double armijo_v;         /* (default 0.1) */
  int32_t max_inner;       /* inner FISTA iterations per outer iteration (default 50000) */
  int32_t max_outer;       /* outer GD iterations per lambda (default 50) */
  int32_t max_linesearch;  /* Armijo trials per outer iteration (default 30) */
  int32_t check_every;     /* inner iterations per captured CUDA graph chunk, i.e. between host
                              reads of the device stop flag (default 32, rounded up to even;
                              at most 4096) */
  int32_t iwls;            /* weights of the inner problem (the package's iwls option, Sec. 6.4):
                              GLAM_IWLS_EXACT (default) uses the IRLS weights of App. B as they are;
                              GLAM_IWLS_KRON uses their tensor-product form (Sec. 6.2, Eq.
                              kronweight): X^T W X theta = H(<X_j^T W_j X_j>, theta), so the inner
                              loop touches p-sized arrays only.  GLAM_IWLS_KRON is exact, and
                              accepted, for the families whose IRLS weight is the observation weight
                              itself (Gaussian; Gamma with log link) with an observation-weight
                              array W that is a tensor product w1 (x) w2 (x) w3 with W(0,0,0) > 0
                              (W = 1 included); otherwise glam_fit_path returns GLAM_EINVAL.
                              GLAM_IWLS_KRON1 / GLAM_IWLS_KRON2 replace the weights V of every outer
                              iteration by their geometric-mean tensor approximation (Sec. 6.2,
                              computed as glam_kron_weights does: KRON1 as printed, normalised by the
                              overall geometric mean; KRON2 with that mean restored) for any family
                              and W; the inner loop then runs on H(<X_j^T diag(v_j) X_j>, .) with the
                              exact Lipschitz constant of the approximation, while the gradient, the
                              line search and the KKT test stay exact, so the solutions are those of
                              GLAM_IWLS_EXACT (Sec. 5: any positive weights keep the fixed point) */
  int32_t penalty;         /* GLAM_PENALTY_LASSO (default): the weighted l1 penalty of Eq. (five);
                              GLAM_PENALTY_ENET / GLAM_PENALTY_RIDGE: the elastic net and ridge
                              penalties of Sec. 6.3 (below; the KKT residual is then the distance
                              of -grad f to lambda times the subdifferential of J);
                              GLAM_PENALTY_SCAD: the SCAD penalty (a = 3.7) by the multistep
                              adaptive lasso of the package (Sec. 6.4): per lambda, step 0 solves
                              the weighted lasso with pen_w, step s >= 1 the lasso with weights
                              pen_w * p'_lambda(|theta^(s-1)|) / lambda, p' the SCAD derivative
                              (lambda up to lambda, (a lambda - t)_+ / (a - 1) beyond); the
                              stats of a lambda then sum the steps' iterations and report the
                              objective and KKT residual of the last weighted problem */
  int32_t steps;           /* MSA steps per lambda for GLAM_PENALTY_SCAD (default 1, >= 1) */
  int32_t exploit_bands;   /* nonzero: the FP64 gradient passes use banded mode products, for marginal
                              designs with at most 4 consecutive nonzeros per row and nondecreasing
                              first columns (cubic B-spline bases); a specialisation, not the paper's
                              general method (which takes dense designs, Sec. 6.1).  The FP64 sums
                              skip only exact zeros, so the path is the same up to summation order.
                              glam_fit_path returns GLAM_EINVAL when a design is not banded or the
                              plan has c > 1 components (default 0) */
  int32_t reserved[2];
  double enet_alpha;       /* GLAM_PENALTY_ENET: J = sum_m w_m (|theta_m| + enet_alpha theta_m^2),
                              the elastic net of Sec. 6.3 (default 0, >= 0) */
  double wait_limit_s;     /* limit, in seconds, of every bounded device-side wait of the inner
                              loop's kernels (a copy or an MMA that should complete); a wait that
                              runs out makes glam_fit_path return GLAM_ETIMEOUT, and the plan stays
                              usable (default 2, in [0, 3600]; 0 gives up at once unless the awaited
                              data is already there, which tests the error path) */
  double nu;               /* inner step size relative to the bound L_hat (the package's nu, Sec. 6.4;
                              default 1, in [0, 1]): nu = 1 takes delta = 1/L_hat and never backtracks;
                              nu in (0, 1) starts from delta = 1/(nu L_hat), nu = 0 from delta = 1, and
                              when an inner solve diverges (its step max_m |x+_m - y_m| grows past 10
                              times its first value, or turns non-finite) the solve restarts from
                              theta_k with delta halved, but not below 1/L_hat, where it cannot
                              diverge; the divergence test runs only while delta > 1/L_hat */
} glam_opts;

#define GLAM_IWLS_EXACT 0
#define GLAM_IWLS_KRON 1
#define GLAM_IWLS_KRON1 2  /* geometric-mean tensor approximation of V, as printed (Sec. 6.2) */
#define GLAM_IWLS_KRON2 3  /* the same times the overall geometric mean of V */
#define GLAM_PENALTY_LASSO 0
#define GLAM_PENALTY_SCAD 1
#define GLAM_PENALTY_ENET 2  /* J = sum w (|theta| + alpha theta^2); prox: soft threshold, then / (1 + 2 alpha gamma) */
#define GLAM_PENALTY_RIDGE 3 /* J = sum w theta^2; prox: / (1 + 2 gamma); lambda_max is the lasso's */

/* Per-lambda record written by glam_fit_path (HOST array of nlambda entries). */
typedef struct {
  double lambda;
  double objective;        /* F at the returned Theta, FP64 */
  double kkt;              /* max_m r_m / lambda_max, FP64; r_m = |g_m + lambda w_m sign theta_m|
                              if theta_m != 0, else max(0, |g_m| - lambda w_m), g = grad f */
  double time_ms;
  int32_t outer_iters;     /* outer GD iterations (inner solves) */
  int32_t inner_iters;     /* inner PG iterations, total */
  int32_t fp64_passes;     /* FP64 gradient passes (H and G in FP64 at an outer iterate); the KKT
                              test at the start of a lambda reuses the gradient of the previous
                              lambda's solution, so a converged lambda after the first takes
                              outer_iters of them, the first lambda outer_iters + 1 */
  int32_t armijo_backtracks;
  int32_t nnz;
  int32_t status;          /* GLAM_OK or GLAM_ENOCONV / GLAM_ENONFINITE for this lambda */
  int32_t inner_restarts;  /* inner solves restarted with a halved step (opts.nu < 1) */
  int32_t reserved0;
} glam_stats;

/* Fill *opts with the defaults listed in glam_opts.  Returns GLAM_EINVAL for NULL. */
int glam_opts_default(glam_opts* opts);

/* Create a plan for one problem shape.  dims: HOST pointer (copied).  family: one of the four
 * GLAM_* families above.  precision: GLAM_FP64, GLAM_FP32, GLAM_TF32 or GLAM_BF16; it names the
 * arithmetic of the bottleneck product G(V (.) H(y)) (Sec. 6.2, Eq. twentysixnew: the inner-loop
 * product of glam_prox_step and glam_fit_path), which runs on the tensor cores for the
 * single-precision plans:
 *   GLAM_FP32  3xTF32: every operand split into two TF32 parts, three products each, FP32
 *              accumulation (about FP32 accuracy);
 *   GLAM_TF32  TF32 operands (10-bit mantissa, rounded to nearest), FP32 accumulation;
 *   GLAM_BF16  BF16 operands (8-bit mantissa, rounded to nearest), FP32 accumulation; the fit
 *              path also keeps the IRLS weights in BF16, halving the bytes the inner loop streams.
 * The 5th-generation tensor-core kernel serves shapes with n1 <= 128, n1 % 4 == 0 (% 8 for
 * BF16), n2 % 32 == 0, n2 <= 128 (GLAM_FP32) or 256, p1, p2 <= 32; outside that domain a
 * warp-level tensor-core kernel serves shapes with n1 % 32 == 0, n2 % 8 == 0, n2 <= 256,
 * p1, p2 <= 32 and 4 n1 n2 < 2^20 bytes (3xTF32 for GLAM_FP32, TF32 for GLAM_TF32 and GLAM_BF16
 * plans), and FP32 SIMT kernels every other shape.  In the single-precision plans,
 * glam_predict, glam_gradient, glam_loss and glam_quad_build take their H-transform from a
 * tcgen05 kernel in the 3xTF32 form (about FP32 accuracy) on the 5th-generation domain above
 * with n2 <= 224, from FP32 SIMT kernels elsewhere, and their G from FP32 SIMT kernels.  The
 * gradient, line-search and KKT passes of glam_fit_path run in FP64 in every plan, so the
 * product precision changes iteration counts, not the accuracy of the accepted solutions.
 * stream: a cudaStream_t (NULL = legacy default stream) on the
 * current device.  *out receives the plan.  Allocates the workspace on the current device.
 * Errors: GLAM_EINVAL (NULL argument; d not 2 or 3; an n_j or p_j below 1; d = 2 with n3 or p3
 * not 1; unknown family or precision; n1 n2 n3 or p1 p2 p3 above 2^40; n3 above 65535 or
 * n3 p2 above 65535 * 64), GLAM_ENOMEM, GLAM_ECUDA. */
int glam_plan_create(const glam_dims* dims, int family, int precision, void* stream, glam_plan** out);

/* Create a plan for the model with c components (Sec. 2, Eq. fivenew: X = [X_1 | ... | X_c], each
 * X_r = X_r3 (x) X_r2 (x) X_r1 with its own marginal designs and parameter array Theta_r):
 *   eta = sum_r H(<X_rj>, Theta_r)          (Sec. 6.1, Eq. eighteen with r = 1..c),
 *   G(U) = (G(<X_1j>, U), ..., G(<X_cj>, U))  (Eq. nineteen),
 * and, in glam_fit_path, the Prop. 1 bound L_hat = max(w)/n sum_r prod_j varrho(X_rj^T X_rj)
 * (Eq. nineteennew).  d: 2 or 3; n: the shared grid (n3 = 1 when d = 2); c in [1, 8]; p: HOST array
 * of 3c sizes, (p_r1, p_r2, p_r3) of component r at 3r (p_r3 = 1 when d = 2).  The coefficient
 * vector of such a plan is the concatenation (vec Theta_1, ..., vec Theta_c) of p = sum_r p_r1 p_r2
 * p_r3 entries, each vec in the layout of a one-component plan (p_r1 fastest), and every X
 * argument is a HOST array of 3c device pointers, X_r1, X_r2, X_r3 of component r at 3r.  Such a
 * plan serves glam_predict, glam_gradient, glam_loss and glam_fit_path (iwls GLAM_IWLS_EXACT; the
 * inner-loop product then runs as the sum of the components' mode products in the plan's
 * precision, not the fused kernels); glam_quad_build, glam_prox_step, glam_penalized_nll,
 * glam_time_inner_kernels and glam_fit_path_batched return GLAM_EINVAL for it.  c = 1 gives
 * the plan of glam_plan_create.  The other arguments and errors are those of glam_plan_create. */
int glam_plan_create_components(int d, const int64_t n[3], int c, const int64_t* p, int family, int precision,
                                void* stream, glam_plan** out);

/* Release the plan and its workspace (synchronizes its stream first).  NULL is a no-op. */
int glam_plan_destroy(glam_plan* plan);

/* Enqueue later calls on another stream of the plan's device. */
int glam_plan_set_stream(glam_plan* plan, void* stream);

/* Message of the last failure on this plan ("" if none); NULL plan: the calling thread's last
 * failure.  The string is owned by the library and valid until the next call on the plan. */
const char* glam_last_error(const glam_plan* plan);

/* eta = H(<X_j>, Theta): the linear predictor X theta of Sec. 2 computed by three chained rho
 * transforms (Sec. 6.1, Eq. eighteen; App. A).  X: HOST array of 3 device pointers (X[2] may be
 * NULL when d = 2).  Theta: p elements.  eta: n elements (written). */
int glam_predict(glam_plan* plan, const void* const X[3], const void* Theta, void* eta);

/* grad = grad f(Theta) = -(1/n) X^T u(eta(Theta)) (Sec. 2, Eq. three), u the score of App. B,
 * Eq. (four), X^T computed by G (Eq. nineteen).  Y, W: n elements.  grad: p elements (written).
 * loss_or_null: if not NULL, a DEVICE double receiving f(Theta) (FP64 accumulation). */
int glam_gradient(glam_plan* plan, const void* const X[3], const void* Theta, const void* Y,
                  const void* W, void* grad, double* loss_or_null);

/* *out = f(Theta) = -(1/n) l(eta(Theta)) (Sec. 2, Eq. two; constants as stated above), computed
 * with FP64 accumulation.  out: DEVICE double. */
int glam_loss(glam_plan* plan, const void* const X[3], const void* Theta, const void* Y,
              const void* W, double* out);

/* Build the quadratic model at Theta_k (Alg. 1 steps 2-3; Sec. 6.1 step 2 and Eq. twentyeight):
 * eta = H(Theta_k), then V, V (.) Z, b = G(V (.) Z) and Lhat (Prop. 1).  q: HOST struct of
 * caller-owned device buffers (see glam_quad). */
int glam_quad_build(glam_plan* plan, const void* const X[3], const void* Theta_k, const void* Y,
                    const void* W, const glam_quad* q);

/* One inner PG iteration of Sec. 3.2 on the model q:
 *   y = x + omega (x - x_prev);  grad h(y) = (G(V (.) H(y)) - b) / n  (Eqs. twentyfive, twentysixnew);
 *   x_next = prox_{delta lambda}(y - delta grad h(y)), the weighted soft threshold of Sec. 6.3
 *   with per-coordinate threshold delta * lambda * pen_w[m].
 * delta <= 0 means delta = 1 / *q->Lhat (read on the device).  x, x_prev, pen_w, x_next: p
 * elements; x_next must not alias x or x_prev. */
int glam_prox_step(glam_plan* plan, const void* const X[3], const glam_quad* q, const void* x,
                   const void* x_prev, double omega, double delta, double lambda, const void* pen_w,
                   void* x_next);

/* Warm-started lambda path of GD-PG (Alg. 1; lambda_max and warm starts of Sec. 6.4).
 * X, Y, W: the plan's element type, as for the other calls.
 * pen_w, Theta0, Theta_path: DOUBLE for every plan (the p-space state of the solver is FP64 in
 *   every precision: the mode products of a GLAM_FP32 plan run in FP32 on corrections only, and
 *   each outer iteration recomputes grad f and the KKT residual in FP64, so the returned Theta
 *   carries FP64 accuracy).
 * lambda: HOST array of nlambda doubles.  If lambda[0] < 0 the path is automatic,
 *   lambda_k = lambda_max * ratio^(k/(nlambda-1)) (ratio = opts->lambda_min_ratio), and the used
 *   values are written back; otherwise the given values are used in order.
 * opts: HOST, NULL for defaults.  Theta0: p doubles or NULL (start from zero).
 * Theta_path: nlambda * p doubles (written; row k is the solution at lambda[k]).
 * stats: HOST array of nlambda records or NULL.  nfit: HOST, number of completed lambdas.
 * Each lambda stops when its FP64 KKT residual is <= opts->tol.  Returns GLAM_ENOCONV (with
 * *nfit = the number of lambdas that met the tolerance, and rows up to the failing one written)
 * when an iteration cap is hit, as the paper's package does; GLAM_ENONFINITE on non-finite
 * input or a non-finite iterate; GLAM_EINVAL for a NULL argument, nlambda < 1, a NaN lambda[0],
 * a negative given lambda, or options out of range. */
int glam_fit_path(glam_plan* plan, const void* const X[3], const void* Y, const void* W,
                  const void* pen_w, int nlambda, double* lambda, const glam_opts* opts,
                  const double* Theta0, double* Theta_path, glam_stats* stats, int* nfit);

/* Geometric-mean tensor approximation of a weight array (Sec. 6.2, "tensor approximation" of the
 * weights; the iwls options "kron1" and "kron2" of Sec. 6.4): for V (n elements in the plan's
 * layout, FP64, DEVICE) writes the factors v1 (n1), v2 (n2), v3 (n3) (FP64, DEVICE) with
 *   v_j(i) = exp( mean over the cells of slice i of mode j of log V  -  mean over all cells of log V ),
 * so that V_hat(i1, i2, i3) = v1(i1) v2(i2) v3(i3) (the product form of the paper, with the
 * normalisation by the overall geometric mean V_bar); scaled != 0 multiplies v1 by V_bar, so that
 * V_hat = V whenever V is a tensor product.  Reading of the paper: the means run over the cells
 * with V > 0 (a masked cell, weight 0, has no logarithm and carries no weight), and a slice without
 * such a cell gets the factor 1.  Sums in a fixed order (the same bits on every run).  Stream-
 * ordered on the plan's stream; uses plan workspace.
 * Errors: GLAM_EINVAL (NULL argument), GLAM_ENOMEM, GLAM_ECUDA. */
int glam_kron_weights(glam_plan* plan, const double* V, int scaled, double* v1, double* v2, double* v3);

/* Penalized negative log-likelihood F(Theta) = f(Theta) + lambda sum_m pen_w[m] |theta_m| (the
 * PMLE objective of Sec. 2, Eq. five, scaled by 1/n as stated above) and its vector-Jacobian
 * product, the adjoint used by automatic differentiation:
 *   grad_Theta = g (grad f(Theta) + lambda pen_w (.) sign(Theta)),  grad f = -(1/n) G(u) with u
 *                the score of App. B, Eq. (four), at eta = H(Theta) (Eqs. three, eighteen,
 *                nineteen); sign(0) = 0 (the zero element of the subdifferential);
 *   grad_Y     = g df/dY: (1/n) a (y - eta) (Gaussian) or -(1/n) a eta (Poisson), the derivative
 *                of the loss constants stated above;
 * g = *gout (a DEVICE double, the upstream derivative of a scalar function of F) or 1 when gout
 * is NULL.  Theta, pen_w, grad_Theta: p elements; Y, W, grad_Y: n elements (plan element type).
 * F: DEVICE double or NULL; grad_Theta, grad_Y: written when not NULL (at least one output must
 * be requested).  lambda >= 0.  Asynchronous; FP64 accumulation for F.
 * Errors: GLAM_EINVAL (NULL inputs, no output, bad lambda), GLAM_ECUDA. */
int glam_penalized_nll(glam_plan* plan, const void* const X[3], const void* Theta, const void* Y,
                       const void* W, double lambda, const void* pen_w, const double* gout,
                       double* F, void* grad_Theta, void* grad_Y);

/* One problem of a batch: the arguments of glam_fit_path for one plan (same meaning, layout and
 * ownership), plus its two outputs. */
typedef struct {
  const void* X[3];
  const void* Y;
  const void* W;
  const void* pen_w;       /* DOUBLE, p elements */
  int32_t nlambda;
  double* lambda;          /* HOST, nlambda (in/out as in glam_fit_path) */
  const double* Theta0;    /* p doubles or NULL */
  double* Theta_path;      /* nlambda * p doubles (written) */
  glam_stats* stats;       /* HOST, nlambda records, or NULL */
  int32_t nfit;            /* out: completed lambdas */
  int32_t status;          /* out: the status glam_fit_path returned for this problem */
} glam_batch_item;

/* Many independent penalized GLAM fits (cross-validation folds, bootstrap replicates, separate
 * data sets; each a warm-started lambda path of Alg. 1 / Sec. 6.4) run concurrently on one GPU:
 * item i is fitted with plans[i], whose shape, family and precision it must match, by up to
 * max_threads host worker threads (max_threads <= 0: one per item, at most the number of host
 * cores), each fit on its plan's private stream, so the small kernels of different fits overlap
 * on the device.  plans: HOST array of nitems distinct plans (a plan serves one fit at a time).
 * items: HOST array of nitems records (outputs nfit and status written).  opts: HOST, NULL for
 * defaults, shared by every item.  Returns when every fit has finished: GLAM_OK if every item's
 * status is GLAM_OK, else the status of the lowest-numbered failing item (its message:
 * glam_last_error(plans[i])).  Errors: GLAM_EINVAL (NULL arrays, nitems < 0, a repeated plan;
 * message from glam_last_error(NULL)). */
int glam_fit_path_batched(int nitems, glam_plan* const* plans, glam_batch_item* items,
                          const glam_opts* opts, int max_threads);

/* ---- allocation-free entry point (the paper has no counterpart) ----
 *
 * f(eta) = (1/n) sum_i a_i l_i(eta_i, y_i), the loss of glam_loss (constants as stated at the
 * top of this header) computed from a caller-supplied linear predictor eta instead of Theta,
 * for callers that cannot allocate device memory where they need it: code running while a
 * stream is captured into a CUDA graph, hosts that hand out every byte of device memory from
 * their own pool, real-time paths where an allocation could block.  It calls no cudaMalloc,
 * cudaFree or allocating library routine and needs no plan: its reduction scratch (1024 FP64
 * block partials and a completion counter, 8448 bytes) is a fixed __device__ array inside
 * libglam, which every GPU that loads the library holds until the process exits.
 *   family: any of the four families; precision: GLAM_FP64 (double arrays) or GLAM_FP32 (float
 *   arrays); n: cells, 1 <= n <= 2^40 (the cell limit of a plan; larger n returns GLAM_EINVAL);
 *   eta, Y, W: n elements (DEVICE); out: one DEVICE double (written); stream: cudaStream_t.
 * Each cell's term is computed exactly as glam_loss computes it, including the clamp of eta
 * before the exponential (at 80 in FP32, 700 in FP64), so that a large eta gives a finite term
 * and a masked cell (a_i = 0) contributes zero; a NaN or infinite input gives a NaN result.
 * Every term is added in FP64, with a fixed summation order (same bits on every call).
 * Asynchronous on `stream`.  The first call on a device looks up the scratch address with
 * cudaGetSymbolAddress (a runtime query, not an allocation) and keeps it; every call clears the
 * counter with cudaMemsetAsync on `stream`.
 * All calls share
 * the one scratch array: calls whose kernels overlap on the GPU race on it and must be
 * serialized (one stream).
 * Errors: GLAM_EINVAL (message from glam_last_error(NULL)), GLAM_ECUDA. */
int glam_loss_eta_noalloc(int family, int precision, int64_t n, const void* eta, const void* Y,
                          const void* W, double* out, void* stream);

/* ---- diagnostics (tracing hooks of this library; the paper has no counterpart) ---- */

/* Number of kernels this process has launched through libglam so far (each replay of a captured
 * CUDA graph adds its kernel nodes).  Never fails. */
int64_t glam_launch_count(void);

/* Time the kernels of one inner PG iteration of glam_fit_path, as the fit launches them, on the
 * plan's stream with CUDA events: ms[0] the fused per-slab G(V (.) H(.)) kernel, which also forms
 * the first H stage X_3 d of the correction d (0 if the shape uses the unfused chain); ms[1] the
 * separate mode-3 product of the unfused chain (0 when the fused kernel is used); ms[2] the
 * mode-3 adjoint product: the split GEMM, or, where the fit path fuses it with the proximal step
 * (FP32 and TF32 plans whose p2 p1 and n3 are multiples of 4), that one kernel; ms[3] the
 * proximal step (0 when it is part of ms[2]).  Each kernel runs 2 + reps times back to
 * back (the tcgen05 kernel as programmatic dependent launches, as the fit path launches it, so
 * that a launch's start overlaps the end of the one before); ms (HOST, 4 doubles) receives the
 * mean of the last reps launches in milliseconds.  Uses
 * q->V as the weights and the plan's FP64 state of the last fit (values do not change the work).
 * Synchronizes the plan's stream. */
int glam_time_inner_kernels(glam_plan* plan, const void* const X[3], const glam_quad* q, int reps,
                            double* ms);

#ifdef __cplusplus
}
#endif

#endif /* GLAM_H */
