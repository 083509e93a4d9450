// Launchers of the device kernels (one translation unit per family).
#pragma once
#include "common.cuh"

namespace bchdav {

// Exclusive scan of int counts (+ add_one each) into int64 offsets out[0..n] (laplacian.cu);
// tile_sums holds ceil(n / 2048) + 1 values.
cudaError_t exclusive_scan(cudaStream_t st, int n, const int* in, int add_one, long long* out,
                           long long* tile_sums);
inline int scan_tile_count(int n) { return (n + 2047) / 2048 + 1; }

// ---------------- SpMM family (spmm.cu) ----------------
// Rows with more than kLongRow nonzeros are cut into segments of kLongRow nonzeros, each
// reduced by its own CTA into pseg (n_seg x b, in the SpMM's value type) before the row
// kernel adds them up in segment order.
constexpr int kLongRow = 1024;
struct SpmmLong {
  long long n_seg = 0;                 // 0: no long rows (the row kernel does every row)
  const long long* seg_off = nullptr;  // n + 1: row r owns segments [seg_off[r], seg_off[r+1])
  const int* seg_row = nullptr;        // n_seg: row of each segment
  void* pseg = nullptr;                // n_seg * b values of workspace
};
// Builds seg_off / seg_row for rowptr (one host synchronisation to read the segment count).
// cnt_work: n ints; tile_sums: scan_tile_count(n) values; seg_row capacity seg_cap.
cudaError_t build_spmm_long(cudaStream_t st, int n, const int* rowptr, int* cnt_work,
                            long long* seg_off, long long* tile_sums, int* seg_row,
                            long long seg_cap, long long* host_total, long long* n_seg);
long long spmm_long_seg_cap(long long nnz);

// Y = alpha * (A X) + beta * X + gamma * Z + diag(delta) R, row by row (Eq. (6)
// with the epilogue of Algorithm 3).  Z may be NULL (gamma ignored); R may be
// NULL (delta, one coefficient per column on the device, ignored).
template <typename T>
cudaError_t launch_spmm_axpby(cudaStream_t st, int n, const int* rowptr, const int* colidx,
                              const T* val, const T* X, int ldx, int b, T* Y, int ldy,
                              const T* Z, int ldz, T alpha, T beta, T gamma,
                              const T* R = nullptr, int ldr = 0, const T* delta = nullptr,
                              const SpmmLong* lg = nullptr, int threads = 256);

// Residual of Step 12: R = A V - V diag(d) into Rout (n x b, ldr >= b; required), then
// per-CTA partial sums of r_j^2 and v_j^2 in partial[cta * 2b + {j, b + j}]; the CTA count
// is returned in *n_parts.  negd: b doubles of device scratch.
cudaError_t launch_spmm_resid(cudaStream_t st, int n, const int* rowptr, const int* colidx,
                              const double* val, const double* V, int ldv, int b,
                              const double* d, double* partial, int* n_parts, double* Rout,
                              int ldr, double* negd, const SpmmLong* lg = nullptr);
int spmm_resid_max_parts(int n, int b);
// Double-float products for the mixed path (A's values as float hi + lo: vh = the float32
// copy, vl = launch_split_dd_vec of the float64 values): Y = alpha A X + diag(delta) R and the
// Step-12 residual, with float64 blocks in and out.  b a multiple of 4 (<= 128), no long rows;
// scratch holds spmm_dd_scratch_floats(n, b) floats.
bool spmm_dd_supported(int b, const SpmmLong* lg);
size_t spmm_dd_scratch_floats(int n, int b);
cudaError_t launch_split_dd_vec(cudaStream_t st, long long n, const double* v, float* lo);
cudaError_t launch_spmm_dd(cudaStream_t st, int n, const int* rowptr, const int* colidx,
                           const float* vh, const float* vl, const double* X, int ldx, int b,
                           double* Y, int ldy, double alpha, const double* R, int ldr,
                           const double* delta, float* scratch);
cudaError_t launch_spmm_resid_dd(cudaStream_t st, int n, const int* rowptr, const int* colidx,
                                 const float* vh, const float* vl, const double* V, int ldv,
                                 int b, const double* d, double* partial, int* n_parts,
                                 double* Rout, int ldr, double* negd, float* scratch);

// ---------------- dense family (dense.cu) ----------------
// partial[c] = A(rows of chunk c, 0:ka)^T B(rows of chunk c, 0:kb); ka*kb outputs.
cudaError_t launch_gemm_tn_partial(cudaStream_t st, int n, const double* A, int lda, int ka,
                                   const double* B, int ldb, int kb, double* partial,
                                   int n_chunks);
int gemm_tn_chunks(int n);
// out[i] = scale * sum_c partial[c * count + i] (fixed order).
cudaError_t launch_reduce_partials(cudaStream_t st, const double* partial, int n_chunks, int count,
                                   double* out, double scale);
// C(:, 0:nb) -= A(:, 0:k) B (k x nb, ldb) ; A and C distinct.
cudaError_t launch_gemm_nn_sub(cudaStream_t st, int n, const double* A, int lda, int k,
                               const double* B, int ldb, int nb, double* C, int ldc);
// A(:, 0:nb) = A(:, 0:k) B  in place (nb <= k), row tiles staged in shared memory.
// X(:, 0:b) <- X(:, 0:b) U in place for U upper triangular (b <= 64).
cudaError_t launch_gemm_tri_inplace(cudaStream_t st, int n, double* X, int ldx, int b,
                                    const double* U, int ldu);
cudaError_t launch_gemm_nn_inplace(cudaStream_t st, int n, double* A, int lda, int k,
                                   const double* B, int ldb, int nb);
// Column sums of squares of X (N x b): per-CTA partials, count b.
cudaError_t launch_col_sumsq_partial(cudaStream_t st, int n, const double* X, int ldx, int b,
                                     double* partial, int n_chunks);
cudaError_t launch_copy_block(cudaStream_t st, int n, int w, const double* src, int lds,
                              double* dst, int ldd);
// dst(:, j) = src(:, perm[j]) for j < w (perm on the device).
// X(:, 0:count) = X(:, shift:shift+count) in place (warp per row, chunked left to right).
cudaError_t launch_shift_cols_left(cudaStream_t st, int n, double* X, int ldx, int count, int shift);
cudaError_t launch_gather_cols(cudaStream_t st, int n, int w, const double* src, int lds,
                               const int* perm, double* dst, int ldd);
cudaError_t launch_f64_to_f32(cudaStream_t st, int n, int w, const double* src, int lds,
                              float* dst, int ldd);
cudaError_t launch_f32_to_f64(cudaStream_t st, int n, int w, const float* src, int lds,
                              double* dst, int ldd);
// Mixed-precision filter inputs: column j of Z0/R32 (float, ldo) takes
// float(X(:, j)) / 0 when src[j] < 0, else 0 / float(R(:, src[j])).
cudaError_t launch_mixed_inputs(cudaStream_t st, int n, int b, const double* X, int ldx,
                                const double* R, int ldr, const int* src, float* Z0, float* R32,
                                int ldo);
cudaError_t launch_f64_to_f32_vec(cudaStream_t st, long long count, const double* src, float* dst);
// Column `col` of X := Philox random vector `vec` of `stream`.
cudaError_t launch_fill_random_col(cudaStream_t st, int n, double* X, int ldx, int col,
                                   uint64_t seed, uint32_t stream, uint32_t vec);
// H(0:k_act, k_act-b:k_act) = G (k_act x b), mirrored, new diagonal block symmetrised.
cudaError_t launch_h_update(cudaStream_t st, double* H, int ldh, const double* G, int k_act, int b);
// H = diag(d[0:k]) (ldh x ldh cleared up to k).
cudaError_t launch_h_diag(cudaStream_t st, double* H, int ldh, const double* d, int k, int clear);
// Cholesky G = R^T R of a small Gram matrix and R^{-1} (see dense.cu for the flag rules).
// With colscale (b doubles, output): G is first equilibrated by exact powers of two,
// G' = D G D with D_jj = colscale[j] ~ 1 / sqrt(G_jj), and R^{-1} is that of G' (so that
// (X D) R'^{-1} = X R^{-1}).
cudaError_t launch_chol_inv(cudaStream_t st, int b, const double* G, const double* norm0,
                            double rel_min, double dep, double* Rinv, int* flag,
                            double* colscale = nullptr);
// Non-finite check: flag |= any(!isfinite(x)).
cudaError_t launch_check_finite(cudaStream_t st, int n, int w, const double* X, int ldx, int* flag);

// ---------------- float64-accurate tensor-core products (ozaki.cu) ----------------
// C = A B (subtract: C -= A B) for A N x K row-major, B K x nb, K <= 448; C may alias A
// (A is read only through its slices).  work: ozaki_nn_work_bytes(n, K, nb) bytes.
cudaError_t launch_ozaki_nn(cudaStream_t st, int n, const double* A, int lda, int K,
                            const double* B, int ldb, int nb, double* C, int ldc, bool subtract,
                            void* work);
size_t ozaki_nn_work_bytes(int n, int K, int nb);
bool ozaki_nn_supported(int K);
// out (ka x kb, row-major) = A^T B for A N x ka, B N x kb (any N: the reduction is cut
// into pieces of 1024 rows whose float32 sums are exact, folded in float64).
// tc_err non-NULL: the products run on tcgen05 (launch_tc_gram), which sets *tc_err when one
// of its bounded waits expired.
cudaError_t launch_ozaki_tn(cudaStream_t st, int n, const double* A, int lda, int ka,
                            const double* B, int ldb, int kb, double* out, void* work,
                            int* tc_err = nullptr);
size_t ozaki_tn_work_bytes(int n, int ka, int kb);
// Building blocks with caller-kept slices ("planes": 8 bf16 digit planes plus exponents).
int oz_chunks(int Np);   // 1024-row exponent chunks of a Gram operand with Np rows
size_t oz_planes_bytes(size_t rows, size_t kp);
int oz_pad_k(int k);      // k padded to the k step (16)
int oz_pad_rows(int m);   // rows padded to the row tile (64)
int oz_pad_cols(int n);   // columns padded to the column tile (32)
// colscale (optional, K doubles, exact powers of two): slices of A diag(colscale).  slices: the
// leading planes written (a product that reads fewer slices needs only those).
cudaError_t oz_slice_rows(cudaStream_t st, int n, const double* A, int lda, int K, int Kp,
                          void* planes, int* E, const double* colscale = nullptr, int slices = 8);
cudaError_t oz_slice_cols_t(cudaStream_t st, int n, const double* A, int lda, int w, int Np, int cap,
                            int c_off, void* planes, int* E);
cudaError_t oz_gram_from_planes(cudaStream_t st, int Np, const void* PA, const int* EA, int capA,
                                int a0, int ka, const void* PB, const int* EB, int capB, int kb,
                                double* out, double* partial, int slices = 8);
cudaError_t oz_nn_from_planes(cudaStream_t st, int n, int K, int Kp, const void* PA, const int* EA,
                              const double* B, int ldb, int nb, double* C, int ldc, bool subtract,
                              void* bwork, int slices = 8);
// The same product C = / -= A B from A's row planes on the tcgen05 tensor cores (tc05.cu):
// B (K x nb) is split here into planes of round_up(nb, 32 or 64) columns in bwork; err (device
// int, may be NULL) is set when a bounded wait inside the kernel expires.
cudaError_t oz_nn_from_planes_tc(cudaStream_t st, int n, int K, int Kp, const void* PA,
                                 const int* EA, const double* B, int ldb, int nb, double* C,
                                 int ldc, bool subtract, void* bwork, int slices, int* err);
// Gram product A^T B of transposed column planes on tcgen05 (tc05.cu); same operands as
// oz_gram_from_planes, plus err (device int, set when a bounded wait expired).
cudaError_t launch_tc_gram(cudaStream_t st, int Np, const void* PA, const int* EA, int capA, int a0,
                           int ka, const void* PB, const int* EB, int capB, int kb, double* out,
                           double* partial, int slices, int* err);
cudaError_t launch_tc_slice_nn(cudaStream_t st, int n, int nb, int Kp, const void* PA,
                               const int* EA, const void* PB, int nbp, const int* EB, double* C,
                               int ldc, bool subtract, int slices, int* err);
size_t oz_bwork_bytes(int K, int nb);

// ---------------- orthonormalisation (orth.cu) ----------------
// Column-by-column classical Gram-Schmidt with two passes inside the block,
// starting at column j0; stops at the first column found dependent and
// reports it in *dep (-1 if none).  Cooperative launch; grid_cap > 0 bounds its block count
// (a one-block grid never waits for blocks that are not resident, whatever else runs).
cudaError_t launch_inblock_gs(cudaStream_t st, int n, double* X, int ldx, int b, int j0,
                              const double* norm0, double tau_dep, double* scratch, int* dep,
                              double* final_norms, int grid_cap = 0);
size_t inblock_gs_scratch_doubles(int b);

// ---------------- eigensolver (eig.cu) ----------------
// Symmetric eigendecomposition of the n x n matrix H (upper triangle read).
cudaError_t launch_eigh(cudaStream_t st, int n, const double* H, int ldh, double* D, double* Y,
                        int ldy, double* work, int* status);
size_t eigh_work_doubles(int n);
// Same result by the small route (n <= kEsMaxN), the tridiagonal route (n <= kTrdMaxN) or
// parallel cyclic Jacobi over many SMs, which also replaces a route's result that the route
// flags; launch_eigh for n <= 32 where the device cannot run the small route's cluster.  work
// holds eigh_fast_work_doubles(n) doubles.
// aux, ev1, ev2 (optional, all or none): a second stream and two events on which the
// tridiagonal route accumulates Q beside the eigenvalue and eigenvector kernels.
cudaError_t launch_eigh_fast(cudaStream_t st, int n, const double* H, int ldh, double* D, double* Y,
                             int ldy, double* work, int* status, int grid_cap = 0,
                             cudaStream_t aux = nullptr, cudaEvent_t ev1 = nullptr,
                             cudaEvent_t ev2 = nullptr);
size_t eigh_fast_work_doubles(int n);
// Tridiagonal route of launch_eigh_fast for 32 < n <= kTrdMaxN (one thread-block cluster
// reduces H; eigenvalues and vectors of T on the whole GPU).  work holds trd_work_doubles(n)
// doubles.  *run_jacobi receives the device word that is nonzero when the result must be
// replaced by the Jacobi route.  cudaErrorNotSupported: the device cannot run the cluster.
constexpr int kTrdMaxN = 448;
size_t trd_work_doubles(int n);
cudaError_t launch_trd_eigh(cudaStream_t st, int n, const double* H, int ldh, double* D,
                            double* Y, int ldy, double* work, int** run_jacobi,
                            cudaStream_t aux = nullptr, cudaEvent_t ev_reduced = nullptr,
                            cudaEvent_t ev_q = nullptr);
// Small route of launch_eigh_fast for n <= kEsMaxN (eigs.cu): a float32 decomposition refined
// in float64 by one thread-block cluster.  work holds eig_small_work_doubles() doubles;
// *run_jacobi as for the tridiagonal route.  eig_small_available(): the device runs the cluster.
constexpr int kEsMaxN = 64;
size_t eig_small_work_doubles();
bool eig_small_available();
cudaError_t launch_eig_small(cudaStream_t st, int n, const double* H, int ldh, double* D,
                             double* Y, int ldy, double* work, int** run_jacobi);

// ---------------- Laplacian assembly (laplacian.cu) ----------------
struct LapWork;
}  // namespace bchdav
