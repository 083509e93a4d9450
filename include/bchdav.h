/*
 * bchdav.h -- C ABI of the GB300 block Chebyshev-Davidson eigensolver.
 *
 * Problem (Eqs. (1)-(2) of the paper): for the symmetric normalized Laplacian
 * A = I - D^{-1/2} S D^{-1/2} of an undirected graph with N nodes, find the k
 * smallest eigenvalues 0 <= lambda_1 <= ... <= lambda_k <= 2 and eigenvectors
 * V (N x k) with A V = V Lambda_k.  The method is Algorithm 2 (block
 * Chebyshev-Davidson with inner-outer restart) with the Chebyshev filter of
 * Algorithm 3 and the analytic spectrum bounds [0, 2].
 *
 * Conventions shared by every entry point:
 *  - All array arguments are DEVICE pointers unless stated otherwise.  Dense
 *    blocks are row-major: element (i, j) of an N x w block with leading
 *    dimension ld sits at p[i * ld + j], ld >= w.
 *  - The caller owns every array it passes in; the library owns its workspace
 *    (kept in the handle) and the CSR arrays returned by bchdav_build_laplacian.
 *  - Work is ordered on the handle's CUDA stream.  Functions that must decide
 *    on data (bchdav_solve, bchdav_orthonormalize, bchdav_build_laplacian)
 *    synchronise that stream before returning; the others only enqueue.
 *  - Errors are returned as bchdav_status, never thrown; bchdav_last_error()
 *    gives a message.  Invalid sizes give BCHDAV_ERR_ARG and no work is
 *    enqueued.  A CUDA failure gives BCHDAV_ERR_CUDA.
 *  - Nothing here allocates memory visible to the caller except
 *    bchdav_build_laplacian.
 */
#ifndef BCHDAV_H
#define BCHDAV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BCHDAV_OK = 0,
  BCHDAV_NOT_CONVERGED = 1,   /* itmax reached; the first info.n_converged pairs are valid */
  BCHDAV_ERR_ARG = -1,        /* invalid size, pointer or parameter */
  BCHDAV_ERR_CSR = -2,        /* CSR structure invalid (row pointers, column range/order) */
  BCHDAV_ERR_OOM = -3,        /* workspace allocation failed */
  BCHDAV_ERR_CUDA = -4,       /* a CUDA call or kernel launch failed */
  BCHDAV_ERR_NONFINITE = -5,  /* NaN or Inf appeared in the iteration */
  BCHDAV_ERR_TIMEOUT = -6     /* a bounded device-side wait gave up */
} bchdav_status;

typedef enum {
  BCHDAV_PREC_FP64 = 0,   /* every step in float64 */
  BCHDAV_PREC_MIXED = 1   /* filter SpMM and recurrence in float32, the rest float64 */
} bchdav_precision;

typedef struct bchdav_handle_s* bchdav_handle;

/* The matrix A in CSR form (device arrays).  Rows ascending, column indices
 * ascending and in [0, n) within each row, nnz = rowptr[n] < 2^31.
 * val (float64) is required.  val_f32 is optional: when NULL and the mixed
 * path is requested, the solver rounds val to float32 into its workspace. */
typedef struct {
  int32_t n;
  int64_t nnz;
  const int32_t* rowptr;   /* n + 1 */
  const int32_t* colidx;   /* nnz */
  const double* val;       /* nnz */
  const float* val_f32;    /* nnz or NULL */
} bchdav_csr;

/* Step 1 of Algorithm 2: the spectrum bounds of the filter (Sec. 2).  The first low_nwb is
 * lowb + (upperb - lowb) k / N in every mode. */
typedef enum {
  BCHDAV_BOUNDS_NORMALIZED = 0,  /* lowb = 0, upperb = 2: the normalized Laplacian (Eq. (1)) */
  BCHDAV_BOUNDS_GIVEN = 1,       /* opts.lowb, opts.upperb */
  BCHDAV_BOUNDS_LANCZOS = 2      /* k-step Lanczos estimate (bchdav_lanczos_bounds), seed = opts.seed */
} bchdav_bounds;

/* Optional parameters of bchdav_solve; zero-initialise for the defaults. */
typedef struct {
  int32_t dim_max;          /* 0: min(max(act_max + 2b, k + 30), N)  (Sec. 4 defaults) */
  int32_t itmax;            /* 0: 1000 outer iterations */
  int32_t precision;        /* bchdav_precision */
  int32_t dense_path;       /* Steps 6, 8 and 11: 0 (default): float64-accurate products from
                               bf16 digit slices on tcgen05 (tensor-memory level sums); 1: plain
                               float64 FMA kernels; 2: the same slice products on the legacy
                               warp-level mma.sync (kept for comparison) */
  uint64_t seed;            /* seed of the random vectors the method draws (Philox4x32-10) */
  const double* v_init;     /* optional N x k_init initial block (Algorithm 2, V_init) */
  int32_t k_init;
  int32_t ld_v_init;
  int32_t record_history;   /* nonzero: keep per-iteration counters (bchdav_history) */
  int32_t bounds;           /* bchdav_bounds: where Step 1's lowb and upperb come from */
  double lowb, upperb;      /* BCHDAV_BOUNDS_GIVEN: the bounds (lowb < upperb) */
  int32_t lanczos_steps;    /* BCHDAV_BOUNDS_LANCZOS: steps of the estimate (0: 20; <= 64) */
  int32_t reserved3;
} bchdav_opts;

/* Results and per-component device time of one solve. */
typedef struct {
  int32_t iters;            /* outer iterations of Algorithm 2 */
  int32_t n_converged;      /* locked pairs (>= k on success) */
  int32_t n_spmm;           /* SpMM launches with A (filter + W + residual) */
  int32_t n_replaced;       /* vectors replaced by random ones in Step 6 */
  double max_rel_resid;     /* max_j ||A v_j - lambda_j v_j|| / ||v_j|| over the returned pairs */
  double ms_total;
  double ms_filter, ms_orth, ms_spmm_w, ms_h, ms_eig, ms_rot, ms_resid, ms_other;
  double filter_bytes;      /* algorithmic bytes moved by all filter SpMM steps */
  double filter_ms_kernels; /* device time of those steps alone (CUDA events) */
  int64_t n_kernel_launches;/* kernels this library launched during the solve */
  int32_t status;           /* the solve's return status (set by bchdav_solve_batched) */
  int32_t reserved2;
  double lowb, upperb;      /* the bounds Step 1 used */
} bchdav_info;

/* One record per outer iteration when opts.record_history is set. */
typedef struct {
  int32_t it, k_c, e_c, k_act, k_sub, k_old, n_rep;
  int32_t k_orth;           /* basis width Step 6 orthogonalised against (k_sub before Step 7) */
  double low_nwb;
  double max_resid;         /* max relative residual of the k_b tested pairs */
  double min_resid;         /* min relative residual of the k_b tested pairs */
} bchdav_iter_record;

/* ---- handle ------------------------------------------------------------- */

/* Create a handle bound to the current CUDA device and the given stream
 * (cudaStream_t, NULL = legacy default stream). */
bchdav_status bchdav_create(bchdav_handle* h, void* cuda_stream);
bchdav_status bchdav_destroy(bchdav_handle h);
bchdav_status bchdav_set_stream(bchdav_handle h, void* cuda_stream);
const char* bchdav_status_string(bchdav_status s);
/* NULL handle: the message of the last failed call without a handle on this host thread. */
const char* bchdav_last_error(bchdav_handle h);
/* Cap the device workspace the handle may hold (bytes; 0, the default, removes the cap).  A
 * call whose workspace would grow past the cap returns BCHDAV_ERR_OOM, exactly as when
 * cudaMalloc fails: nothing already held is freed and the handle stays usable (raise the cap,
 * or call bchdav_release_workspace, and call again).  It bounds what one handle takes on a
 * device shared with other work.  Not a paper concept. */
bchdav_status bchdav_set_memory_limit(bchdav_handle h, uint64_t bytes);
/* Device workspace the handle holds now, in bytes. */
uint64_t bchdav_workspace_bytes(bchdav_handle h);

/* ---- Eq. (1): the symmetric normalized Laplacian ------------------------ */

/* Build A = I - D^{-1/2} S D^{-1/2} from n_edges undirected edges
 * (src[e], dst[e]) given as DEVICE int32 arrays.  Self loops are dropped,
 * both orientations and repeats count once (S is 0/1).  Output is canonical
 * CSR: columns ascending, diagonal stored explicitly as 1.0, off-diagonal
 * -(r_i * r_j) with r_i = 1/sqrt(d_i) (IEEE), a degree-0 row holding only its
 * diagonal; val_f32 is the round-to-nearest float of val.  The arrays of *out
 * are allocated by the library and released with bchdav_free_csr.  Returns
 * BCHDAV_ERR_ARG for an endpoint outside [0, n). */
bchdav_status bchdav_build_laplacian(bchdav_handle h, int32_t n, int64_t n_edges,
                                     const int32_t* src, const int32_t* dst, bchdav_csr* out);
bchdav_status bchdav_free_csr(bchdav_handle h, bchdav_csr* csr);

/* The graph matrices the library assembles.  The combinatorial Laplacian L = D - S has the
 * same pattern as Eq. (1), off-diagonal -1.0 and diagonal d_i (0.0 for an isolated node); its
 * spectrum lies in [0, 2 max d_i], and its bounds for Algorithm 2 come from
 * BCHDAV_BOUNDS_LANCZOS or BCHDAV_BOUNDS_GIVEN. */
typedef enum {
  BCHDAV_LAPLACIAN_NORMALIZED = 0,     /* Eq. (1) */
  BCHDAV_LAPLACIAN_COMBINATORIAL = 1   /* D - S */
} bchdav_laplacian_kind;

/* bchdav_build_laplacian for the matrix of the given kind (same arguments, layout, ownership
 * and errors; an unknown kind gives BCHDAV_ERR_ARG). */
bchdav_status bchdav_build_laplacian_kind(bchdav_handle h, int32_t n, int64_t n_edges,
                                          const int32_t* src, const int32_t* dst, int32_t kind,
                                          bchdav_csr* out);

/* Copy the arrays of csr into caller-owned device arrays (n + 1 and nnz
 * entries; val_f32 may be NULL to skip it), ordered on the handle's stream and
 * complete when the call returns. */
bchdav_status bchdav_copy_csr(bchdav_handle h, const bchdav_csr* csr, int32_t* rowptr,
                              int32_t* colidx, double* val, float* val_f32);

/* Check a caller-built CSR on the device (row pointers monotone, columns in
 * range and strictly ascending per row).  BCHDAV_ERR_CSR when it is not. */
bchdav_status bchdav_check_csr(bchdav_handle h, const bchdav_csr* A);

/* ---- Sec. 2: spectrum bounds when they are not analytic -------------------- */

/* k-step Lanczos estimate of the bounds of the symmetric matrix A (any CSR: both triangles
 * stored).  Start vector v_1 = u/||u||, u_i uniform in [-1/2, 1/2) from Philox4x32-10 stream 3,
 * vector 0, the given seed; steps w = A v_j - beta_{j-1} v_{j-1}, alpha_j = v_j . w,
 * w -= alpha_j v_j, beta_j = ||w||, v_{j+1} = w / beta_j, no reorthogonalisation; an exactly
 * zero beta_j ends it after step j.  With theta the eigenvalues of the tridiagonal T:
 * *lowb = theta_min and *upperb = theta_max + beta_last (the residual norm of the Lanczos
 * relation; Zhou and Li's estimator).  lowb, upperb, alpha, beta (steps doubles each, may be
 * NULL) and steps_done (may be NULL) are HOST pointers.  1 <= steps <= min(64, N), else
 * BCHDAV_ERR_ARG.  Synchronises the handle's stream. */
bchdav_status bchdav_lanczos_bounds(bchdav_handle h, const bchdav_csr* A, int32_t steps,
                                    uint64_t seed, double* lowb, double* upperb, double* alpha,
                                    double* beta, int32_t* steps_done);

/* ---- Algorithm 2 ---------------------------------------------------------- */

/* k smallest eigenpairs of A by block Chebyshev-Davidson (Algorithm 2) with
 * block size b (k_b), filter degree m, active-space limit act_max (0 = the
 * default max(5b, 30)) and convergence tolerance tol on the relative residual
 * ||A v - lambda v|| / ||v||.  evals: k doubles, ascending (device).  evecs:
 * N x k row-major, ld = k (device).  info may be NULL.  Requires 1 <= k <= N,
 * b >= 1, m >= 1, 2b <= act_max and max(dim_max, k + 2b) <= N.
 * Returns BCHDAV_NOT_CONVERGED (with the pairs locked so far, sorted, in the
 * leading info->n_converged slots) when itmax is reached, BCHDAV_ERR_NONFINITE
 * (before any iteration) when opts->v_init holds a NaN or an infinity, and
 * BCHDAV_ERR_OOM when the workspace cannot be allocated (or would pass the
 * handle's bchdav_set_memory_limit cap); the handle stays usable after both. */
bchdav_status bchdav_solve(bchdav_handle h, const bchdav_csr* A, int32_t k, int32_t b, int32_t m,
                           int32_t act_max, double tol, const bchdav_opts* opts,
                           double* evals, double* evecs, bchdav_info* info);

/* Same as bchdav_solve with HOST arrays for the CSR, V_init and the results:
 * copies in, solves, copies out, all inside the call (the end-to-end path). */
bchdav_status bchdav_solve_host(bchdav_handle h, int32_t n, int64_t nnz, const int32_t* rowptr,
                                const int32_t* colidx, const double* val, int32_t k, int32_t b,
                                int32_t m, int32_t act_max, double tol, const bchdav_opts* opts,
                                double* evals_host, double* evecs_host, bchdav_info* info);

/* Many independent problems (the paper solves one; running many side by side is an
 * extension of Algorithm 2, not a step of it).  Graph i is solved as by bchdav_solve with
 * k[i], b[i], m[i], act_max[i] (0 = default), the shared tol and opts, except that
 * opts->v_init is ignored and graph i draws its start block with seed opts->seed + i.
 * evals[i] (k[i] doubles) and evecs[i] (N_i x k[i], ld = k[i]) are device arrays.
 * The graphs run on a pool of worker handles, each with its own stream, taking graphs
 * largest-first (nnz * b); the call returns when all are done.  infos[i] (status included)
 * and per_graph_ms[i] (wall time of graph i's own solve) may be NULL arrays.  Returns
 * BCHDAV_OK when every graph converged, else the first error, else BCHDAV_NOT_CONVERGED. */
bchdav_status bchdav_solve_batched(bchdav_handle h, int32_t n_graphs, const bchdav_csr* As,
                                   const int32_t* k, const int32_t* b, const int32_t* m,
                                   const int32_t* act_max, double tol, const bchdav_opts* opts,
                                   double* const* evals, double* const* evecs,
                                   bchdav_info* infos, float* per_graph_ms);

/* Free every device and pinned buffer the handle holds (the next call allocates again). */
bchdav_status bchdav_release_workspace(bchdav_handle h);

/* Kernels this library has launched in the process so far (all handles). */
int64_t bchdav_launch_count(void);

/* Number of concurrent solves of bchdav_solve_batched (default 8, 1..64). */
bchdav_status bchdav_set_batch_workers(bchdav_handle h, int32_t n_workers);

/* Per-iteration records of the last solve of this handle (opts.record_history). */
int32_t bchdav_history(bchdav_handle h, bchdav_iter_record* out, int32_t max_records);

/* ---- single steps (each is one step of Algorithm 2 / 3) -------------------- */

/* Algorithm 3: Y = p_m(A) X with p_m(x) = T_m((x - c)/e) / T_m((a0 - c)/e),
 * c = (a + upb)/2, e = (upb - a)/2, computed by the scaled three-term
 * recurrence.  X, Y: N x b, leading dimensions ldx, ldy (distinct buffers).
 * precision = BCHDAV_PREC_MIXED runs the recurrence in float32 (A->val_f32
 * required); X and Y stay float64 and are rounded on entry / widened on exit. */
bchdav_status bchdav_filter(bchdav_handle h, const bchdav_csr* A, const double* X, int32_t ldx,
                            int32_t b, int32_t m, double a, double upb, double a0,
                            int32_t precision, double* Y, int32_t ldy);

/* Plain SpMM Y = A X (Eq. (6)), float64.  X: N x b (ldx), Y: N x b (ldy). */
bchdav_status bchdav_spmm(bchdav_handle h, const bchdav_csr* A, const double* X, int32_t ldx,
                          int32_t b, double* Y, int32_t ldy);

/* The same product as the mixed path computes it in Steps 7 and 12 of Algorithm 2: A's values
 * and X's entries as unevaluated sums of two floats (hi + lo; hi of the values = A->val_f32,
 * required), an exact float product and sum per term, float64 in and out.  Relative error per
 * entry about 2^-46 of sum_j |a_ij x_j|.  X, Y: device, N x b (ldx, ldy), X != Y; b a multiple
 * of 4 and at most 128, and no row longer than the SpMM segment length (otherwise
 * BCHDAV_ERR_ARG: the mixed path then uses the float64 product). */
bchdav_status bchdav_spmm_dd(bchdav_handle h, const bchdav_csr* A, const double* X, int32_t ldx,
                             int32_t b, double* Y, int32_t ldy);

/* Step 6: orthonormalise the N x b block X (in place, ldx) against the k
 * orthonormal columns of V (ldv) and among themselves: two classical
 * Gram-Schmidt passes against V, then column-by-column Gram-Schmidt with a
 * second pass inside the block; a column whose remaining norm is <= tau_dep
 * times its original norm (or zero) is replaced by Philox random vector
 * number *rep_counter (seed, stream 1) and the block is redone.  *rep_counter
 * is advanced by the number of replacements, *n_replaced receives it. */
bchdav_status bchdav_orthonormalize(bchdav_handle h, int32_t n, const double* V, int32_t ldv,
                                    int32_t k, double* X, int32_t ldx, int32_t b, uint64_t seed,
                                    double tau_dep, int64_t* rep_counter, int32_t* n_replaced);

/* Steps 6 and 8: out (ka x kb, row-major, ld = kb) = A^T B for the N x ka block A (lda)
 * and the N x kb block B (ldb), by the float64-accurate slice product on tcgen05 (dense_path
 * 0), plain float64 FMAs (dense_path 1) or the slice product on warp-level mma (dense_path 2).
 * Deterministic (fixed reduction order).  BCHDAV_ERR_TIMEOUT if a bounded device wait of the
 * tcgen05 kernel expired (nothing faults; the handle stays usable).  Synchronises the stream
 * on dense_path 0. */
bchdav_status bchdav_gram(bchdav_handle h, int32_t n, const double* A, int32_t lda, int32_t ka,
                          const double* B, int32_t ldb, int32_t kb, double* out,
                          int32_t dense_path);

/* Step 11: V(:, 0:nb) = V(:, 0:k) Y in place (V: n x k, ldv; Y: k x nb, ld_y; nb <= k),
 * the subspace rotation, with the products of bchdav_gram's dense_path (0: tcgen05, 1: float64
 * FMAs, 2: warp-level mma; the tensor-core paths need k <= 448).  BCHDAV_ERR_TIMEOUT as for
 * bchdav_gram. */
bchdav_status bchdav_rotate(bchdav_handle h, int32_t n, double* V, int32_t ldv, int32_t k,
                            const double* Y, int32_t ld_y, int32_t nb, int32_t dense_path);

/* Step 9 (Algorithm 2): H Y = Y D for the symmetric n x n float64 matrix H (ld_h; only the
 * upper triangle is read).  D: n eigenvalues ascending; Y: n x n, column j the eigenvector of
 * D[j] (row-major, ld_y).  All on the device, float64-accurate by one of three routes:
 *  - n <= 64: a float32 decomposition (Householder, multisection, inverse iteration) refined
 *    in float64 by the Ogita-Aishima iteration, in one thread-block cluster;
 *  - 64 < n <= 448: Householder tridiagonalisation in one cluster, multisection and inverse
 *    iteration on the tridiagonal matrix, one Newton-Schulz step;
 *  - n > 448, and whenever a route flags its result on the device (a cluster of eigenvalues it
 *    cannot resolve, a refinement that did not settle, a non-finite H): parallel cyclic Jacobi
 *    on a cooperative grid.
 * The routes give the same eigenpairs to rounding (vectors of a repeated eigenvalue: any
 * orthonormal basis of its space).  n outside [1, 1024] returns BCHDAV_ERR_ARG.  Synchronises
 * the handle's stream (it reads the convergence status). */
bchdav_status bchdav_eigh(bchdav_handle h, int32_t n, const double* H, int32_t ld_h, double* D,
                          double* Y, int32_t ld_y);

/* ---- learned start block (an extension feeding Algorithm 2's V_init) ----------
 * The paper takes an optional block of initial vectors and filters it progressively, best
 * Rayleigh quotient first (Sec. 3, progressive filtering; Algorithm 2, Step 17).  These calls
 * run a three-layer message-passing network on Ahat = I - A that proposes such a block:
 *   X0 = [sqrt(deg)/8, log(1 + deg)/8, R],  S_l = (Ahat H_{l-1}) W_l + H_{l-1} U_l + b_l,
 *   H_l = relu(S_l), Z = H_3 Wo  (N x k),
 * trained to align span(Z) with solver eigenvectors U: loss = 1 - tr(G^{-1} P^T P) / k with
 * G = Z^T Z + rho I, rho = ridge tr(Z^T Z) / k, P = U^T Z.  theta: float32 device vector of
 * bchdav_gnn_n_params values in the order W_1, U_1, b_1, W_2, U_2, b_2, W_3, U_3, b_3, Wo
 * (row-major fan_in x fan_out).  R: N x d_r float32 device features.  A needs val_f32.
 * Shapes: d_r + 2 and width multiples of 4 and at most 64; 1 <= k <= 64. */
int64_t bchdav_gnn_n_params(int32_t d_r, int32_t width, int32_t k);
/* Z (N x k float32, device) = network output. */
bchdav_status bchdav_gnn_forward(bchdav_handle h, const bchdav_csr* A, const float* R,
                                 int32_t d_r, const float* theta, int32_t width, int32_t k,
                                 float* Z);
/* loss (host or device double) and its gradient (device, n_params floats) against U (N x k
 * float64, ld k, device); Z (may be NULL) receives the output. Synchronises the stream. */
bchdav_status bchdav_gnn_loss_grad(bchdav_handle h, const bchdav_csr* A, const float* R,
                                   int32_t d_r, const float* theta, int32_t width, int32_t k,
                                   const double* U, double ridge, float* grad, double* loss,
                                   float* Z);
/* steps x n_graphs Adam updates (lr, beta1 = 0.9, beta2 = 0.999, eps = 1e-8; one update per
 * graph, graphs in order) of theta in place; loss_history (host, may be NULL) receives the
 * loss before each update, row-major steps x n_graphs. */
bchdav_status bchdav_gnn_train(bchdav_handle h, int32_t n_graphs, const bchdav_csr* As,
                               const float* const* R, int32_t d_r, const double* const* U,
                               int32_t width, int32_t k, float* theta, int32_t steps, double lr,
                               double ridge, double* loss_history);
/* V0 (N x k float64, ld k, device): orthonormal basis of span(Z) rotated to Ritz vectors,
 * Rayleigh quotients ascending in ritz (k, device) -- the V_init of bchdav_solve. */
bchdav_status bchdav_gnn_start_block(bchdav_handle h, const bchdav_csr* A, const float* R,
                                     int32_t d_r, const float* theta, int32_t width, int32_t k,
                                     double* V0, double* ritz);

/* ---- Algorithm 1, Steps 4-5: spectral clustering of the eigenvectors ------ */

/* The paper's Algorithm 1 normalises each row of the eigenvector block (Step 4) and
 * clusters the rows (Step 5), naming k-means as one method; it fixes neither the variant nor
 * its arithmetic.  These calls implement Lloyd's k-means with farthest-first seeding in a
 * fixed arithmetic, so that labels, seeds and centroids are bit-reproducible and independent
 * of the launch shape:
 *   features   X(i, d) = float32(V(i, d) / sqrt(s_i)), s_i the float64 sum over d in order of
 *              V(i, d)^2 (separate multiply and add); a zero row stays zero;
 *   distance   acc = 0; acc = acc + (x_d - c_d)^2 over d in order, float32, no fused
 *              multiply-add;
 *   seeding    s_0 = first; s_j = the node with the largest min_{l<j} dist(X_i, X_{s_l}),
 *              the lowest index on ties (farthest-first traversal);
 *   assignment the nearest float32(C_j), the lowest j on ties;
 *   update     C_j = float64(Q_j) / count_j * 2^-36 with Q_j the 64-bit integer sum of
 *              round-half-even(X_i * 2^36) over the members (order-independent; exact while
 *              |X| <= 1 and n < 2^27); a cluster without members keeps its centroid;
 *   rounds     the first assignment is round 1, each update + assignment one more; stop
 *              when an assignment changes no label or after max_rounds rounds.
 * Features are stored transposed: Xt is dim x n, row-major, leading dimension ldx >= n
 * (element (d, i) at Xt[d * ldx + i]).  Limits: 1 <= n < 2^27, 1 <= dim <= 512,
 * 1 <= n_clusters <= n; otherwise BCHDAV_ERR_ARG and nothing is enqueued. */

/* Step 4: V is n x dim row-major (ld ldv >= dim, float64), e.g. the evecs of bchdav_solve;
 * writes Xt.  Enqueue only. */
bchdav_status bchdav_row_normalize(bchdav_handle h, int32_t n, int32_t dim, const double* V,
                                   int64_t ldv, float* Xt, int64_t ldx);

/* Farthest-first seeds: seeds[0..n_clusters-1] (device int32) from the node `first` in
 * [0, n).  Enqueue only (n_clusters - 1 passes over Xt). */
bchdav_status bchdav_kmeans_seed(bchdav_handle h, int32_t n, int32_t dim, const float* Xt,
                                 int64_t ldx, int32_t n_clusters, int32_t first, int32_t* seeds);

/* Step 5: Lloyd's k-means from the nodes seeds[] (device int32, each in [0, n); a seed
 * outside that range gives BCHDAV_ERR_ARG after the call's work has drained).  labels: n
 * int32 (device); centroids: n_clusters x dim row-major float64 (device, may be NULL), the
 * centroids of the final assignment; rounds: HOST int32 (may be NULL).  Synchronises the
 * handle's stream once per round (the stopping test). */
bchdav_status bchdav_kmeans(bchdav_handle h, int32_t n, int32_t dim, const float* Xt,
                            int64_t ldx, int32_t n_clusters, const int32_t* seeds,
                            int32_t max_rounds, int32_t* labels, double* centroids,
                            int32_t* rounds);

/* Steps 4 and 5 in one call: features of V into the handle's workspace, farthest-first seeds
 * from `first`, Lloyd's k-means.  seeds (device, n_clusters int32) and centroids may be
 * NULL. */
bchdav_status bchdav_spectral_cluster(bchdav_handle h, int32_t n, int32_t dim, const double* V,
                                      int64_t ldv, int32_t n_clusters, int32_t first,
                                      int32_t max_rounds, int32_t* labels, double* centroids,
                                      int32_t* seeds, int32_t* rounds);

/* ---- allocation-free variant (no counterpart in the paper) --------------- */

/* bchdav_eigh for callers that cannot allocate device memory when they call
 * it (for example while another runtime owns all device memory through its
 * own pool, or on a latency-critical path that must not pay the device-wide
 * synchronisation of cudaMalloc/cudaFree).  It uses no handle and calls no
 * cudaMalloc, cudaFree or other allocating routine: its scratch is a fixed
 * array inside the library (about 384 KiB per GPU, held until the process
 * exits).  Same arguments as bchdav_eigh, plus the CUDA stream (cudaStream_t,
 * NULL = legacy default stream) the work is ordered on; the call synchronises
 * that stream before returning.  It always runs one thread block's Householder
 * tridiagonalisation and implicit-shift QL (bchdav_eigh takes the routes listed
 * above instead), so its results equal bchdav_eigh's to rounding, not bit for
 * bit, and it is slower than bchdav_eigh (about 0.25 ms at n = 8, 2.7 ms at
 * n = 32 on GB300, where float64 chains wait ~64 cycles per operation).
 *  - n must be <= 128; larger n returns BCHDAV_ERR_ARG (message via
 *    bchdav_last_error(NULL)).
 *  - The first call on a device looks up the scratch array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - All calls share the one scratch array: calls whose work overlaps on the
 *    GPU (different streams, different host threads) race and give wrong
 *    results.  Serialise them. */
bchdav_status bchdav_eigh_noalloc(int32_t n, const double* H, int32_t ld_h, double* D, double* Y,
                                  int32_t ld_y, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* BCHDAV_H */
