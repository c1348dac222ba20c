/*
 * dcg.h -- C ABI of the GB300 deflated-CG library.
 *
 * Method: de Roos & Hennig, "Krylov Subspace Recycling for Fast Iterative
 * Least-Squares in Machine Learning" (arXiv 1706.00241).
 *   - Eq. 1: a sequence of SPD systems A^(i) x^(i) = b^(i).
 *   - Algorithm 1 (Sec. 2.2): Deflated-CG(k, ell)(A, b, x_{-1}, W, (AW), tol).
 *   - Sec. 2.3, Eq. 7: harmonic projection G u = theta F u, F = (AZ)^T Z,
 *     G = (AZ)^T AZ, Z = [W, P_ell]; the next W is Z U for k chosen u.
 *     Optionally the orthogonal projection Z^T A Z u = theta Z^T Z u (Sec. 2.3).
 *   - Sec. 3: the RBF kernel k(x_i, x_j) = s^2 exp(-|x_i - x_j|^2 / (2 l^2)).
 *
 * Conventions for every entry point:
 *   - Device pointers are CUDA device addresses on the device that was current
 *     when the context was created. Host pointers are ordinary host memory.
 *     Which one an argument is, is stated per argument ("device" / "host").
 *   - Vectors are float32, length n, contiguous. Matrices of vectors (W, the
 *     stored directions) are column-major n x c with leading dimension n.
 *   - Dense operators are row-major float32 with leading dimension lda
 *     (lda >= n, lda % 4 == 0, base address 16-byte aligned).
 *   - "stream" is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream. All device work of a context is ordered on its stream.
 *   - Ownership: buffers passed in stay owned by the caller. Operator buffers
 *     are borrowed until the next dcg_set_operator_* call or dcg_destroy; the
 *     caller keeps them alive and unchanged during dcg_solve.
 *   - Errors: every call returns a dcg_status; nothing aborts or exits. A
 *     context-level message is kept for dcg_last_error(). After an error
 *     inside dcg_solve, x holds the last iterate.
 *   - Thread safety: a context must not be used by two host threads at once.
 */
#ifndef DCG_H
#define DCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum dcg_status {
  DCG_OK = 0,
  DCG_ERR_INVALID_ARG = 1,       /* bad size, pointer, alignment or enum      */
  DCG_ERR_NOMEM = 2,             /* device allocation failed                  */
  DCG_ERR_CUDA = 3,              /* a CUDA runtime call failed                */
  DCG_ERR_BREAKDOWN = 4,         /* p^T A p <= 0 or not finite: A not SPD     */
  DCG_ERR_SUBSPACE_SINGULAR = 5, /* E = W^T A W or F not positive definite    */
  DCG_ERR_MAXITER = 6,           /* max_iter reached before tol               */
  DCG_ERR_TIMEOUT = 7,           /* a bounded device-side wait gave up        */
  DCG_ERR_STATE = 8,             /* call out of order (e.g. no operator set)  */
  DCG_ERR_UNSUPPORTED = 9,       /* configuration this build does not handle  */
  DCG_ERR_STAGNATION = 10        /* the true residual stopped decreasing above
                                    tol (tol below the attainable accuracy);
                                    x is the last iterate, relres_true its
                                    residual                                   */
} dcg_status;

typedef enum dcg_window {         /* which directions feed the next W (Algorithm 1) */
  DCG_WINDOW_FIRST = 0,           /* p_0 .. p_{ell-1}, as the paper stores        */
  DCG_WINDOW_LAST = 1             /* the final ell directions of the solve        */
} dcg_window;

typedef enum dcg_select {         /* which (harmonic) Ritz values are kept (Sec. 2.3) */
  DCG_SELECT_LARGEST = 0,
  DCG_SELECT_SMALLEST = 1
} dcg_select;

typedef enum dcg_extraction {     /* how the next W is drawn from Z = [W, P] (Sec. 2.3) */
  DCG_EXTRACT_HARMONIC = 0,       /* harmonic projection, G u = theta F u (Eq. 7)    */
  DCG_EXTRACT_RITZ = 1            /* orthogonal projection,
                                     Z^T A Z u = theta Z^T Z u (the equation before
                                     Eq. 7)                                          */
} dcg_extraction;

typedef enum dcg_fg_form {        /* how the harmonic pencil's F, G are formed (Sec. 2.3) */
  DCG_FG_EXPLICIT = 0,            /* Gram products over Z = [W, P] and AZ = [AW, AP]:
                                     two tall passes over n x (k + ell) per update  */
  DCG_FG_SPARSE = 1               /* Saad et al.'s sparse forms from scalars the solve
                                     records per stored direction p_j: d_j, alpha_j,
                                     |r_j|^2, |r_{j+1}|^2, (AW)^T r_j, (AW)^T r_{j+1},
                                     with E and (AW)^T AW: F = diag(E, d_j),
                                     G tridiagonal in the P block. Exact in exact
                                     arithmetic (A-conjugacy, orthogonal residuals);
                                     in float32 it neglects what those identities lose.
                                     An update takes the Gram products instead when
                                     a replacement (reading R13) fell inside the
                                     window (it breaks the coupling of the two
                                     directions around it) or the solve had no W
                                     (plain CG: once a Ritz value converges the
                                     float32 directions lose orthogonality and the
                                     tridiagonal model holds ghost copies of it);
                                     dcg_get_pencil_form tells which. Harmonic
                                     extraction only.                               */
} dcg_fg_form;

typedef enum dcg_xformat {        /* element format of X for the matrix-free operator */
  DCG_X_FP32 = 0,                 /* X kept in float32 (the operator is K(X)): the
                                     iteration's tiles are split TF32 (x = hi + lo,
                                     three TF32 products, ~2^-21), the true
                                     residual uses the float32 points             */
  DCG_X_BF16 = 1,                 /* X rounded to bfloat16; exact BF16 products    */
  DCG_X_TF32 = 2                  /* X rounded to TF32; one TF32 product           */
} dcg_xformat;

typedef struct dcg_config {
  int64_t n;            /* system size                                           */
  int32_t k;            /* deflation vectors carried between systems (k >= 0)    */
  int32_t ell;          /* directions stored per solve for extraction (ell >= 0) */
  int32_t window;       /* dcg_window                                            */
  int32_t select;       /* dcg_select                                            */
  int32_t refine_every; /* m: replace r by b - A x every m iterations; 0 = never
                           (the final true-residual confirmation always runs)    */
  int32_t max_iter;     /* iteration cap per solve (> 0)                         */
  int32_t warm_start;   /* 0: x_{-1} = 0 and the input x is ignored; 1: x is x_{-1} */
  int32_t reproject;    /* 1: take mu from (AW)^T (beta p + r) every iteration   */
  int32_t record_history; /* 1: keep |r_j| / |b| per iteration (dcg_get_history) */
  int32_t host_loop;    /* 0: the solve runs as one CUDA graph with conditional
                           nodes (default). 1: the same kernels in the same order,
                           launched from the host with one state read per
                           iteration (slower; for profilers that cannot see
                           kernels inside conditional graphs, and for debugging) */
  int32_t extraction;   /* dcg_extraction (0 = harmonic, the paper's choice)     */
  int32_t fg_form;      /* dcg_fg_form (0 = explicit Gram products)              */
  int32_t reserved[4];  /* must be zero                                          */
  double tol;           /* relative residual target |b - A x| <= tol |b|         */
} dcg_config;

typedef struct dcg_solve_info {
  int32_t status;          /* dcg_status of the solve                             */
  int32_t iters;           /* CG iterations (one A p each)                        */
  int32_t matvecs_loop;    /* = iters                                             */
  int32_t matvecs_setup;   /* columns of the start-of-solve product A [x_{-1} | W] */
  int32_t matvecs_check;   /* true-residual evaluations (confirmation + refinement) */
  int32_t k_used;          /* deflation vectors used in this solve                */
  int32_t stored;          /* directions stored for the next extraction           */
  int32_t reserved;
  double relres_recursive; /* |r_j| / |b| of the recursion at exit                */
  double relres_true;      /* |b - A x| / |b|, compensated accumulation (see dcg_solve) */
  double ms_total;         /* device time of the whole solve (CUDA events)        */
  double ms_setup;         /* start-of-solve product, E and its factor, x_0, p_0  */
} dcg_solve_info;

typedef struct dcg_ctx dcg_ctx;

/* ------------------------------------------------------------------------ */
/* Status strings                                                            */
/* ------------------------------------------------------------------------ */

/* Static description of a status code. Never NULL. */
const char* dcg_status_string(dcg_status s);

/* Last error message of a context (empty string if none); ctx may be NULL,
 * in which case the message of the calling host thread's last failed call
 * made without a context (dcg_create, dcg_form_rbf_dense,
 * dcg_matvec_dense_noalloc) is returned. The pointer stays valid until the
 * next call on the context (or, for NULL, the thread's next such call). */
const char* dcg_last_error(const dcg_ctx* ctx);

/* ------------------------------------------------------------------------ */
/* Context                                                                   */
/* ------------------------------------------------------------------------ */

/* dcg_create: a solver for def-CG(k, ell) (Algorithm 1) on systems of size n.
 *   cfg    host, read once.
 *   stream cudaStream_t (void*) on which all work of the context runs.
 *   out    host; receives the context.
 * Allocates on the current device: W, AW (n x k), the direction store P, AP
 * (n x ell), x, r, p, A p, b and small float64 workspaces. W starts empty
 * (k_active = 0), so the first solve is plain CG (Fig. 1 caption).
 * Errors: INVALID_ARG (n < 1, k < 0, ell < 0, k > n, ell > n, max_iter < 1,
 * tol <= 0, k > 0 with ell + k < k, reserved nonzero), NOMEM, CUDA,
 * UNSUPPORTED (k > 96 or ell > 128: limits of the small dense kernels; or n
 * above what the fused iteration kernel covers with one CTA per SM, 32 passes
 * of 128 rows per CTA: 622592 on a 152-SM GB300). */
dcg_status dcg_create(const dcg_config* cfg, void* stream, dcg_ctx** out);

/* Frees everything the context owns. NULL is allowed. Synchronizes its stream. */
dcg_status dcg_destroy(dcg_ctx* ctx);

/* ------------------------------------------------------------------------ */
/* Operators (L0 of the method: A applied as A v)                            */
/* ------------------------------------------------------------------------ */

/* Stored dense operator: A (device, row-major float32, n x n, leading
 * dimension lda, lda % 4 == 0, 16-byte aligned) is borrowed. Call again after
 * changing A's contents: the next solve then recomputes A W (Algorithm 1
 * takes AW as an input; it is stale once A changes).
 * Errors: INVALID_ARG (NULL, misaligned, lda < n or lda % 4 != 0), CUDA. */
dcg_status dcg_set_operator_dense(dcg_ctx* ctx, const float* A, int64_t lda);

/* Symmetric stored operator given by its upper triangle: as
 * dcg_set_operator_dense, but the operator is the symmetric matrix whose
 * entries A[i*lda + j], j >= i, are read (the strictly lower triangle is never
 * read by the matvec). The matvec of the solve then streams about half of the
 * 4 n^2 bytes: tiles on or right of the diagonal, each contributing A_ij p_j
 * to q_i and, right of the diagonal blocks, A_ij p_i to q_j (the stored
 * operator of Eq. 1 is symmetric positive definite, as Algorithm 1 assumes).
 * The true residual (convergence test and replacement) reads the full
 * matrix, so A must be exactly symmetric (dcg_form_rbf_dense writes it so).
 * Scratch: (8 ceil(n / 2048) + ceil(n / 128)) n floats of partial sums,
 * allocated by the first call on a context (24 MB at n = 16384).
 * Errors: INVALID_ARG (NULL, misaligned, lda < n or lda % 4 != 0), NOMEM, CUDA. */
dcg_status dcg_set_operator_dense_sym(dcg_ctx* ctx, const float* A, int64_t lda);

/* Matrix-free RBF operator A = K + noise I, K_ij = signal_var *
 * exp(-|x_i - x_j|^2 / (2 lengthscale^2)) (Sec. 3 kernel).
 *   X        device, row-major float32 n x d (row i is x_i); copied into the
 *            context's own padded buffer in the requested format, so X is
 *            not borrowed.
 *   d        1 <= d <= 61 (BF16), 29 (TF32) or 9 (FP32: 3 d split-TF32
 *            coordinates): a tile row holds the coordinates and three pieces
 *            of -|x_j|^2 / 2 in 128 bytes, so that the tensor-core product
 *            x_i . x_j - |x_j|^2 / 2 gives each entry's exponent with one FMA.
 *   xformat  dcg_xformat; fixes how X_I X_J^T tiles are formed on the tensor
 *            cores (the operator is the one defined by the rounded X).
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
dcg_status dcg_set_operator_rbf(dcg_ctx* ctx, const float* X, int32_t d, int32_t xformat,
                                double lengthscale, double signal_var, double noise);

/* Change only the RBF hyperparameters of the current matrix-free operator
 * (the lengthscale path of a sequence). Marks A W stale. Errors: STATE. */
dcg_status dcg_set_rbf_params(dcg_ctx* ctx, double lengthscale, double signal_var, double noise);

/* Hyperparameter derivative forms of the current matrix-free operator, for
 * the gradient of a Gaussian-process objective whose solves run through
 * dcg_solve. The paper does not differentiate; the kernel is the Sec. 3 RBF
 * kernel K_ij = s2 exp(-D_ij / (2 l^2)), D_ij = |x_i - x_j|^2 (x as rounded
 * by dcg_set_operator_rbf), and A = K + noise I, so
 *   dA/dl = K .* D / l^3,  dA/ds2 = K / s2,  dA/dnoise = I.
 * For each column pair (u_p, v_p):
 *   out[3p]     = u_p^T (dA/dl) v_p
 *   out[3p + 1] = u_p^T (dA/ds2) v_p
 *   out[3p + 2] = u_p^T (dA/dnoise) v_p = u_p^T v_p
 * computed in one pass over the n^2 kernel entries (float32 entries, float64
 * accumulation across tiles and rows).
 *   U, V    device, column-major n x npairs float32 (leading dimension n).
 *   npairs  1 <= npairs <= 64.
 *   out     host, 3 * npairs doubles.
 * Synchronises the context's stream. Errors: STATE (no matrix-free operator),
 * INVALID_ARG, NOMEM (first call allocates its reduction scratch), CUDA. */
dcg_status dcg_rbf_dtheta(dcg_ctx* ctx, const float* U, const float* V, int32_t npairs, double* out);

/* Forms a stored RBF operator (A1): A[i*lda + j] = signal_var *
 * exp(-|x_i - x_j|^2 / (2 l^2)) + noise * [i == j], float32, computed from X
 * (device, row-major float32 n x d) with float32 difference-form distances.
 * A: device, n x lda. No context needed; runs on `stream`.
 * The squared distance is a float32 sum over the d coordinates (relative
 * error up to d u, u = 2^-24, and typically sqrt(d) u).
 * Errors: INVALID_ARG (X or A NULL, n outside [1, 2^30], lda < n, d outside
 * [1, 4096], lengthscale <= 0, a non-finite parameter), CUDA. The message is
 * kept for dcg_last_error(NULL). */
dcg_status dcg_form_rbf_dense(const float* X, int64_t n, int32_t d, double lengthscale,
                              double signal_var, double noise, float* A, int64_t lda,
                              void* stream);

/* ------------------------------------------------------------------------ */
/* Solve (Algorithm 1)                                                       */
/* ------------------------------------------------------------------------ */

/* dcg_solve: runs Deflated-CG(k, ell)(A, b, x_{-1}, W, AW, tol).
 *   b    device, n floats (read).
 *   x    device, n doubles; in: x_{-1} if cfg.warm_start, else ignored;
 *        out: the solution (or the last iterate on error). The iterate is
 *        accumulated in float64 (x_{j+1} = x_j + alpha_j p_j with float32 p_j):
 *        a float32 iterate cannot represent a solution below the residual floor
 *        ~ eps32 |A| |x| / |b|, which exceeds 1e-6 on ill-conditioned systems.
 *   info host, may be NULL.
 * Steps (all on the device, one host synchronisation at the end):
 *   A W (stored operator: one pass over A; matrix-free: one pass per 8
 *   columns of W, with the tensor-core entries of the loop's matvec, so that
 *   the deflation matches the iteration's operator); r_{-1} = b - A x_{-1}
 *   (warm start only); E = W^T (AW) in
 *   float64 and its Cholesky factor; x_0 = x_{-1} + W E^{-1} W^T r_{-1}
 *   (the initial projection); p_0 = r_0 - W mu_0 (the first direction); then
 *   the iteration with its direction store as a
 *   CUDA graph with a device-side while node. Stops when |r_j| <= tol |b|,
 *   confirmed by a true residual b - A x evaluated with compensated (twice
 *   float32 precision, Ogita-Rump-Oishi Dot2) accumulation and summed in
 *   float64; if it is above tol |b| it replaces r and the loop continues.
 *   The last ell (or first ell) directions p_j and A p_j are kept for
 *   dcg_update_subspace.
 * Returns the solve status (also in info->status): OK, MAXITER, BREAKDOWN,
 * SUBSPACE_SINGULAR, TIMEOUT, STATE (no operator), INVALID_ARG, CUDA. */
dcg_status dcg_solve(dcg_ctx* ctx, const float* b, double* x, dcg_solve_info* info);

/* dcg_solve_multi: nrhs independent solves A x_c = b_c (c < nrhs), each the
 * Deflated-CG(k)(A, b_c, x_{-1,c}, W, AW, tol) of dcg_solve (Algorithm 1,
 * Sec. 2.2) with the context's W, run in lockstep: every iteration forms one
 * block product A [p_c1 p_c2 ...] over the systems still running (matrix-free
 * operator: one pass over the kernel entries for all of them, each entry
 * formed once and contracted with every system's direction on the tensor
 * cores; stored operator: one read of A), then each system takes
 * its own step, its convergence checks, refinements and final true residual
 * exactly as dcg_solve does. Systems leave the block as they converge. The
 * iterates are those of dcg_solve up to the rounding of the block product.
 *   B      device, nrhs x n floats, row c = b_c (read).
 *   X      device, nrhs x n doubles, row c = x_c; in: x_{-1,c} if
 *          cfg.warm_start, else ignored; out: the solutions.
 *   infos  host, nrhs entries, may be NULL; infos[c] as dcg_solve's info.
 *   1 <= nrhs <= DCG_MAX_RHS. The first call with a larger nrhs than before
 *   allocates the per-system workspace (about 5 n floats and 3 n doubles per
 *   system) on the context's device.
 * Stores no directions and records no history; dcg_update_subspace after it
 * returns DCG_ERR_STATE until the next dcg_solve. The iteration is driven
 * from the host (one state read per iteration), whatever cfg.host_loop says.
 * Returns OK if every system returned OK, else the first other status in
 * system order (MAXITER, BREAKDOWN, SUBSPACE_SINGULAR, TIMEOUT, STAGNATION);
 * STATE (no operator), INVALID_ARG, CUDA as dcg_solve; NOMEM if the
 * per-system workspace cannot be allocated. */
#define DCG_MAX_RHS 32
dcg_status dcg_solve_multi(dcg_ctx* ctx, int nrhs, const float* B, double* X, dcg_solve_info* infos);

/* dcg_update_subspace: harmonic-Ritz extraction (Sec. 2.3, Eq. 7) from the
 * last solve: Z = [W, P], AZ = [AW, AP], F = Z^T AZ (symmetrised),
 * G = AZ^T AZ (float64 sums), G u = theta F u solved in float32 after scaling
 * the pencil to unit diagonal (pivoted Cholesky of F, directions dependent at
 * float32 dropped), keep min(k, cols(Z)) values (largest or smallest per
 * cfg.select), W <- Z U with unit columns whose largest-magnitude entry is
 * positive. With cfg.extraction = DCG_EXTRACT_RITZ the pencil is the
 * orthogonal projection instead: F = Z^T Z, G = Z^T AZ (symmetrised), the
 * rest unchanged. Waits for the result on the host.
 *   k_new host, may be NULL; receives the new number of columns of W.
 * Errors: STATE (no completed solve since the last update), SUBSPACE_SINGULAR
 * (F not positive definite even after dropping directions), CUDA. */
dcg_status dcg_update_subspace(dcg_ctx* ctx, int32_t* k_new);

/* dcg_update_subspace_async: the same extraction, enqueued on the context's
 * stream without waiting, so that the caller can overlap it with other work
 * (for example forming the next operator on another stream: the update reads
 * W, AW and the stored directions, not A). The update is then pending: the
 * next call of dcg_solve, dcg_update_subspace(_async), dcg_get_subspace,
 * dcg_set_subspace, dcg_get_ritz_values or dcg_sync waits for it first and,
 * if it failed, returns its error (SUBSPACE_SINGULAR or CUDA) instead of doing
 * its own work; W is then unchanged. Errors here: STATE (no completed solve
 * since the last update), CUDA (enqueueing failed). */
dcg_status dcg_update_subspace_async(dcg_ctx* ctx);

/* (Harmonic) Ritz values of the last update, descending (float64, host): the
 * kept ones are float64 Rayleigh quotients of the pencil (dcg_get_pencil) at
 * the float32 eigenvectors; the others come from the float32 eigen-solve.
 *   theta host, capacity cap; m host: number of values (cols(Z)). */
dcg_status dcg_get_ritz_values(dcg_ctx* ctx, double* theta, int32_t cap, int32_t* m);

/* The float64 pencil (F, G) of the last update, row-major m x m each, m =
 * columns of Z = [W, P] (F = (AZ)^T Z and G = (AZ)^T AZ for the harmonic
 * extraction of Eq. 7; Z^T Z and Z^T A Z for the orthogonal one). The
 * eigen-solve runs in float32 on the scaled pencil and the kept values are
 * then the float64 Rayleigh quotients of this pencil at the float32 vectors,
 * so dcg_get_ritz_values can be checked against a float64 solve of (F, G).
 *   F, G   host, capacity cap doubles each (cap >= m * m), or NULL to query m.
 *   m      host, may be NULL. */
dcg_status dcg_get_pencil(dcg_ctx* ctx, double* F, double* G, int32_t cap, int32_t* m);

/* How the last update formed its pencil (a dcg_fg_form, host): with
 * cfg.fg_form = DCG_FG_SPARSE it is DCG_FG_EXPLICIT when a residual
 * replacement (reading R13) fell inside the window of stored directions, when
 * the solve had no W (see DCG_FG_SPARSE), and for an update that extracted
 * nothing. Errors: INVALID_ARG (NULL), or the pending update's. */
dcg_status dcg_get_pencil_form(dcg_ctx* ctx, int32_t* form);

/* Prior knowledge for the next solve or a checkpoint restore (Fig. 1 caption):
 * W device, column-major n x k (0 <= k <= cfg.k), copied. */
dcg_status dcg_set_subspace(dcg_ctx* ctx, const float* W, int32_t k);

/* Copies the current W (device, column-major n x k_active) into W (device,
 * capacity n x cfg.k) and its column count into *k (host). */
dcg_status dcg_get_subspace(dcg_ctx* ctx, float* W, int32_t* k);

/* Residual history |r_j| / |b|, j = 0..iters, of the last solve when
 * cfg.record_history is set. relres: host, capacity cap; count: host. */
dcg_status dcg_get_history(dcg_ctx* ctx, double* relres, int32_t cap, int32_t* count);

/* ------------------------------------------------------------------------ */
/* The Sec. 3 experiment: Newton steps of the Laplace approximation          */
/* ------------------------------------------------------------------------ */

/* dcg_laplace_system: the linear system of one Newton step for the mode of
 * the Laplace approximation in binary GP classification (Sec. 3, Eq. obj and
 * Eq. linsys), logistic likelihood p(y_i | f_i) = sigma(y_i f_i):
 *   pi = sigma(f), H = diag(pi (1 - pi)), s = H^{1/2} (elementwise, float64),
 *   c = H f + grad log p(y | f) = H f + (y + 1)/2 - pi,
 *   A = I + diag(s) K diag(s),   b = diag(s) K c.
 * A is written in one pass over K (entries (s_i s_j) K_ij, exactly symmetric
 * when K is), so it can be given to dcg_set_operator_dense_sym; K c uses the
 * stored-operator GEMV. The eigenvalues of A lie in [1, 1 + lambda_max(K)/4].
 *   K      device, row-major float32 n x n, leading dimension ldk (ldk >= n,
 *          ldk % 4 == 0, 16-byte aligned): the kernel matrix, read.
 *   y      device, n floats, labels -1 or +1.     f  device, n doubles.
 *   A      device, row-major float32 n x lda (lda >= n, lda % 4 == 0,
 *          16-byte aligned), written.
 *   b      device, n floats; c device, n doubles; s device, n floats: written.
 * Runs on the context's stream without synchronising; the context's own
 * operator and subspace are not touched. The first call allocates 2 n floats
 * of scratch. Errors: INVALID_ARG, NOMEM, CUDA. */
dcg_status dcg_laplace_system(dcg_ctx* ctx, const float* K, int64_t ldk, const float* y, const double* f, float* A,
                              int64_t lda, float* b, double* c, float* s);

/* dcg_laplace_update: the Newton update from the solution x of A x = b:
 *   a = c - s x (float64),  f = K a (stored-operator GEMV, float32 sums),
 *   Psi = log p(y | f) - 1/2 f^T a (float64 sums; Eq. obj without the terms
 *   that do not depend on f, since K^{-1} f = a).
 *   K, y as for dcg_laplace_system; c, s its outputs; x device n doubles.
 *   f, a   device, n doubles, written.
 *   psi    host, may be NULL; receives Psi (the call then synchronises).
 * The Newton loop stops when Psi rises by less than 1 (Sec. 3).
 * Errors: INVALID_ARG, NOMEM, CUDA. */
dcg_status dcg_laplace_update(dcg_ctx* ctx, const float* K, int64_t ldk, const float* y, const double* c,
                              const float* s, const double* x, double* f, double* a, double* psi);

/* ------------------------------------------------------------------------ */
/* Single steps of the hot path, for testing and measurement                 */
/* ------------------------------------------------------------------------ */

/* One operator application q = A p with the fused product p^T q (the
 * denominator d_j = p_j^T A p_j of Algorithm 1).
 *   p, q device n floats; pAp host, may be NULL (then no synchronisation).
 * Errors: STATE (no operator), INVALID_ARG, CUDA. */
dcg_status dcg_matvec(dcg_ctx* ctx, const float* p, float* q, double* pAp);

/* True residual r = b - A x of the current operator: the quantity of the
 * solve's stopping test (the relative |b - A x| / |b| of the Sec. 3
 * experiments) and of its residual replacement. Stored operator: Dot2
 * compensated sums over A with x split as a float32 pair. Matrix-free
 * operator: exact-form entries (Gram-form distances summed onto a fixed grid,
 * a table-driven float32-pair exponential) and Dot2 sums.
 *   b device n floats; x device n doubles; r device n floats (written).
 *   rnorm2 host, may be NULL: |r|^2 summed in float64.
 *   err host, may be NULL: for the matrix-free operator the estimated error
 *     of |r| from the entries' rounding (probabilistic model; the solve
 *     accepts convergence only when |r| + err <= tol |b|); 0 for the stored
 *     operator.
 * Uses the context's iterate buffers (a later dcg_solve overwrites them
 * anyway). Synchronises the context's stream.
 * Errors: STATE (no operator), INVALID_ARG, CUDA. */
dcg_status dcg_residual(dcg_ctx* ctx, const float* b, const double* x, float* r, double* rnorm2, double* err);

/* Multi-vector product Y = A V (the start-of-solve product AW of Algorithm 1,
 * needed by its initial projection): one pass over a stored A; for the matrix-free operator the
 * exact-form entries (as in its true residual), one pass per 16 columns.
 *   V device, column-major n x c; Y device, column-major n x c; 1 <= c <= 129. */
dcg_status dcg_apply_block(dcg_ctx* ctx, const float* V, int32_t c, float* Y);

/* Synchronises the context's stream. */
dcg_status dcg_sync(dcg_ctx* ctx);

/* Throughput of the exponential on the special-function units (ex2.approx),
 * the pipe that binds the matrix-free matvec for small d (one exponential per
 * kernel entry): a short probe kernel on `stream` (independent chains,
 * 2048 threads per SM), best of two timed runs after a warm-up. The paper has
 * no counterpart; the benchmark reports the matrix-free kernels against it.
 *   per_second         host: exponentials per second on the current device.
 *   per_clock_per_sm   host, may be NULL: the same per SM and clock cycle at
 *                      the device's maximum SM clock.
 * Allocates and frees a small device buffer; synchronises `stream`.
 * Errors: INVALID_ARG, CUDA (message for dcg_last_error(NULL)). */
dcg_status dcg_measure_ex2_rate(void* stream, double* per_second, double* per_clock_per_sm);

/* Failure-handling test hook (no counterpart in the paper): arms the next
 * dcg_solve of this context so that, in its first iteration, CTA 0 of the
 * fused iteration kernel withholds its arrival at the grid barrier that
 * separates the per-CTA partial sums from their reduction, and every CTA's
 * bounded wait there gives up after `polls` polls (1 <= polls <= 2^22, about
 * 32 ns or more each) instead of the normal limit. That solve then ends with
 * DCG_ERR_TIMEOUT; dcg_last_error() names the wait that gave up, x holds the
 * iterate as the kernels left it, and no GPU fault or hang is involved (the
 * wait returns; no copy is left in flight). The hook is
 * disarmed by that solve, and later solves on the context run normally.
 * Errors: INVALID_ARG (polls out of range), STATE (no operator set). */
dcg_status dcg_debug_arm_barrier_timeout(dcg_ctx* ctx, int32_t polls);

/* ------------------------------------------------------------------------ */
/* Context-free matvec on fixed scratch (no device allocation)               */
/* ------------------------------------------------------------------------ */

/* q = A p and p^T q for a dense stored operator, without a context and
 * without allocating device memory: the same kernel, grid and reduction order
 * as dcg_matvec (results are bit-identical), with the reduction scratch in
 * a fixed array inside the library. The paper has no counterpart. It serves
 * callers that hold no dcg context
 * and may not allocate at the point of the call: code working inside another
 * framework's device-memory budget (its caching allocator owns the free
 * memory, so a cudaMalloc here could fail or fragment it), and loops that
 * cannot afford the device-wide synchronisation that cudaMalloc and cudaFree
 * may imply.
 *   A      device, row-major float32 n x n with leading dimension lda
 *          (lda >= n, lda % 4 == 0), 16-byte aligned. Read only.
 *   n      1 <= n <= 2^30.
 *   p      device, n floats, 16-byte aligned. Read only.
 *   q      device, n floats. Written.
 *   pAp    device, one double receiving p^T q, or NULL.
 *   stream cudaStream_t as void*; everything runs on it, nothing synchronises.
 * Scratch: a 4352-byte array in the library, per device: an arrival counter
 * and a timeout word (both cleared to zero on `stream` before every launch)
 * and one double partial per CTA for at most 512 CTAs. The grid is min(ceil(n / 8), number of SMs);
 * a device that would need more than 512 CTAs is rejected with UNSUPPORTED.
 * The scratch address is looked up once per device (cudaGetSymbolAddress with
 * that device current); make the first call on each device before any stream
 * capture begins. All calls on a device share the scratch: calls that overlap
 * in time (different streams, or host threads without ordering between them)
 * race on it and give wrong results, so order them, e.g. on one stream.
 * Bounded waits: every wait of the kernel gives up after a fixed number of
 * polls instead of hanging. The call returns before the kernel runs, so such
 * a failure cannot be returned as a status: the CTAs that gave up write NaN
 * into their whole band of rows of q, and *pAp (when given) receives NaN. A
 * finite *pAp means every row of q was computed; without pAp, check q.
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA; the message is kept for
 * dcg_last_error(NULL). */
dcg_status dcg_matvec_dense_noalloc(const float* A, int64_t n, int64_t lda, const float* p, float* q,
                                    double* pAp, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DCG_H */
