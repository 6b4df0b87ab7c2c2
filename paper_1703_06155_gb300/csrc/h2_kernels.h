// Device-side building blocks of libh2 and the task descriptors the host
// planner fills for them.  Every batched kernel takes a flat array of tasks
// (and, where output is tiled, a flat array of tiles), so one launch covers
// all clusters of a colour class / level.  Sizes are exact (the host reads the
// ranks back after each colour's basis update), so no kernel sees a dynamic
// shape.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace h2k {

// Interleaved complex numbers, the storage of every complex arena.
struct __align__(16) cd { double re, im; };
struct __align__(8) cf { float re, im; };

enum Op : int { OP_N = 0, OP_T = 1, OP_C = 2 /* conj */, OP_H = 3 /* conj-transpose */ };
enum Prec : int { P64 = 0, P32 = 1 };

// ---- batched sum-GEMM:  C = alpha * sum_p op(A_p) op(B_p) + beta * C -----
struct GemmPair {
  const void* A;
  const void* B;
  int lda, ldb, K, opA, opB;
};
struct GemmTask {
  void* C;
  int ldc, M, N;
  int p0, np;       // pairs [p0, p0+np)
  double alpha, beta;
  int nk;           // split-K chunks (1: direct)
  int64_t ws_off;   // split-K workspace offset (accumulator complex elements)
  int ksz;          // split-K chunk length in the concatenated K of the pairs
  int herm;         // 1: C is Hermitian, only tiles tm <= tn are computed and
                    // gemm_mirror fills the rest
};
struct GemmTile { int task, tm, tn, kc; };

// ---- in-place apply of a small square matrix to a panel -------------------
//  left : X[r_lo:p, 0:w] = op(A)[r_lo:p, 0:p] * X[0:p, 0:w]
//  right: X[0:h, c_lo:p] = X[0:h, 0:p] * op(A)[0:p, c_lo:p]
struct ApplyTask {
  const void* A;
  void* X;
  int lda, ldx;
  int p;       // order of A
  int w;       // left: columns of X; right: rows of X
  int lo;      // first output row (left) / column (right)
  int opA;
};
struct ApplyTile { int task, t0; };  // t0: first column (left) / row (right)

// ---- batched 2-D copy / accumulate ---------------------------------------
//  dst[0:rows, 0:cols] (=|+=) alpha * op(src) ; src NULL -> zero fill
struct CopyTask {
  const void* src;
  void* dst;
  int lds, ldd, rows, cols;
  int srows, scols;        // source extent; entries outside it read as zero
  int src_prec, dst_prec;  // Prec of each side (complex64 or complex128)
  int mode;                // 0 assign, 1 accumulate, 2 identity (src unused)
  int transpose;           // 1: dst = src^T (src is cols x rows)
  double alpha;
};

// ---- Householder complement of an orthonormal basis ----------------------
//  B (n x k, FP64) -> Vp (n x (n-k)), orthonormal, orthogonal to B.
struct HhTask {
  const cd* B;
  cd* W;      // n x k scratch
  cd* Vp;     // n x (n-k) output (ld n)
  int n, k;
};

// ---- Hermitian Jacobi eigen-decomposition (FP64) -------------------------
//  A (p x p, ld p) is destroyed; U (p x p) gets eigenvectors sorted by
//  decreasing eigenvalue, lam the eigenvalues (decreasing).
struct EigTask {
  cd* A;
  cd* U;
  double* lam;
  int p;
  int* sweeps;  // may be NULL: number of sweeps used
  // Jacobi: off-diagonal entries at or below tol_rel * eps2 * (snorm2 + *trM)
  // are not rotated (trM NULL: no such floor)
  const double* trM;
  double snorm2, eps2, tol_rel;
};

// ---- partial-pivoting LU of one m x m block + explicit triangular inverses
struct LuTask {
  void* A;        // m x m in place (ld lda)
  void* Linv;     // m x m out: L^{-1} P (ld m)
  void* Uinv;     // m x m out: U^{-1}   (ld m)
  int* piv;       // m out: piv[r] = original row now at r
  int lda, m;
  void* scratch;  // m x m work space of the inversion
};

// ---- Step 0 rank selection: r = #{lambda_j > eps^2 (snorm2 + trace(M))} ---
struct SelTask {
  const double* trM;  // trace of the fill-in Gram M (sum of ||F||_F^2)
  const double* lam;  // p eigenvalues, decreasing
  int* out;           // r
  int n, p;
  double snorm2, eps2;
};

// ---- sum of squared Frobenius norms of a list of blocks (trace of M) ------
struct FrobBlock {
  const void* A;
  int lda, rows, cols;
};
struct FrobTask {
  int b0, nb;   // blocks [b0, b0 + nb)
  double* out;
};

// ---- Step 0 subspace: pivoted Cholesky of G' down to thr/(10p), Householder
//  QR of the pivoted columns; Q = I - Y T Y^H, first r' columns Qx.
struct PcholTask {
  cd* G;          // p x p Gram in complement coordinates (ld p), preserved
  const double* trM;  // trace of the fill-in Gram M (-> nu^2)
  cd* L;          // p x p scratch; on exit Y (p x r', unit lower trapezoidal)
  cd* T;          // r' x r' upper triangular (ld r') -- sized p x p by caller
  int* rout;      // r'
  int p, n;
  double snorm2, eps2;
  cd* W;          // p x p scratch (Y^H Y)
  cd* R;          // NULL, or r' x r' (ld r'): the upper triangle receives R of L = Q [R; 0]
  int dfqr;       // 1: Householder QR and Y^H Y in double-float on the FP32 pipe
};

// ---- blocked LU of the final block: one tall panel with partial pivoting --
//  A[row0:row0+nrows, col0:col0+kb] factorized in place, ipiv[j] = absolute
//  row swapped with row0+j, Linv = (unit lower L11)^{-1}, Uinv = U11^{-1}.
struct PanelTask {
  void* A;
  void* Linv;
  void* Uinv;
  int* ipiv;
  int lda, row0, col0, nrows, kb;
};

// ---- far-field sample Gram of the H^2 construction ------------------------
//  G = Z(rows, F) Z(rows, F)^H over the tree-order column ranges F; only the
//  tiles with tm <= tn (upper triangle) are written.
struct KGramTask {
  const int64_t* rows;    // nr tree positions
  const int64_t* ranges;  // nranges (start, count) pairs of tree positions
  cd* G;                  // nr x nr (ld nr)
  int nr, nranges;
};
struct KGramTile { int task, tm, tn; };

// ---- launches (all on `s`, return cudaGetLastError()) ---------------------
// Element precision of A, B (inputs) and C (output), and the precision the
// products are accumulated in.
// split-K: tasks with nk > 1 write partial tiles to `ws` (accumulator
// precision), then gemm_reduce sums them in a fixed order into C.
// shape: output tile 0 = 64 x 64, 1 = 64 x 16, 2 = 32 x 32, 3 = 32 x 16, 4 = 16 x 16,
// 5 = 64 x 8, 6 = 64 x 4 (5 and 6 not with emul), 7 = 64 x 128 (tensor = 2
// complex64 products only)
// (gemm_tile_m / gemm_tile_n).  pina >= 0: precision of the A operands when
// it differs from B's (pin); supported: A complex128 with B complex64, FP64
// accumulation into complex128 or FP32 accumulation into complex64.
// tensor = 1: complex64 64 x 64 products on warp-level TF32 MMAs (3xTF32);
// tensor = 2: the same on tcgen05 MMAs with TMEM accumulators (3xTF32);
// emul = 1: complex64 operands with FP64 accumulation run on the FP32 pipe
// (exact products summed in double-float, flushed to FP64 per K slice);
// emul = 2: complex128 operands and output, products in double-float on the
// FP32 pipe (operands split into two FP32 parts)
cudaError_t gemm(const GemmTask* d_tasks, const GemmPair* d_pairs,
                 const GemmTile* d_tiles, int ntiles, int pin, int pout,
                 int pacc, void* ws, cudaStream_t s, int shape = 0,
                 int pina = -1, int tensor = 0, int emul = 0);
cudaError_t gemm_reduce(const GemmTask* d_tasks, int ntasks, int maxmn,
                        int pout, int pacc, const void* ws, cudaStream_t s);
// C[i, j] = conj(C[j, i]) for the entries of bm x bm tiles below the diagonal
cudaError_t gemm_mirror(const GemmTask* d_tasks, int ntasks, int maxmn,
                        int pout, int bm, cudaStream_t s);
int gemm_tile_m(int shape);
// tiles of the tcgen05 path that gave up waiting for their MMAs (NaN output);
// ~0u when the counter cannot be read
unsigned int gemm_umma_timeouts();
int gemm_tile_n(int shape);

cudaError_t apply_left(const ApplyTask* d_tasks, const ApplyTile* d_tiles,
                       int ntiles, int prec, int maxp, int tw, cudaStream_t s);
cudaError_t apply_right(const ApplyTask* d_tasks, const ApplyTile* d_tiles,
                        int ntiles, int prec, int maxp, int th, cudaStream_t s);
int apply_tile_width(int prec, int maxp);

// ctas_per_task CTAs (1..32) share each task's columns
cudaError_t copy2d(const CopyTask* d_tasks, int ntasks, cudaStream_t s, int ctas_per_task = 4);

cudaError_t householder_complement(const HhTask* d_tasks, int ntasks,
                                   cudaStream_t s);
cudaError_t jacobi_eig(const EigTask* d_tasks, int ntasks, int maxp,
                       int* d_status, cudaStream_t s);
// the same decomposition, one thread-block cluster of `csize` CTAs per task
int64_t jacobi_cluster_scratch(int maxp);  // doubles per task
cudaError_t jacobi_eig_cluster(const EigTask* d_tasks, int ntasks, int maxp,
                               int csize, double* d_scratch, int* d_status,
                               cudaStream_t s, int* csize_used = nullptr);
// the same decomposition by Householder tridiagonalization, implicit QL with
// accumulated rotations and back-transformation (orders <= heev_max_order())
int heev_max_order();
// the Step-0 truncation from the Cholesky factor: one-sided Jacobi SVD of R
// (EigTask.A = R, r' x r' upper triangular, ld r') in double-float on the
// FP32 pipe; lam = squared singular values (decreasing), U = left singular
// vectors.  Orders <= osj_max_order(); scratch in bytes per task.
int osj_max_order();
int64_t osj_cluster_scratch(int maxp);
int osj_cluster_size(int ntasks, int maxp, int cmax);
cudaError_t osj_eig_cluster(const EigTask* d_tasks, int ntasks, int maxp, int csize, void* d_scratch, int* d_status,
                            cudaStream_t s, int* csize_used = nullptr);
int64_t heev_cluster_scratch(int maxp);  // doubles per task
int heev_cluster_size(int ntasks, int maxp, int cmax);
cudaError_t heev_cluster(const EigTask* d_tasks, int ntasks, int maxp, int csize, double* d_scratch, int* d_status,
                         cudaStream_t s, int* csize_used = nullptr);
// Step 3 partial LU with pivoting (one CTA per task), then explicit L^{-1} P
// and U^{-1} (two CTAs per task, in a second launch); maxm = the largest m of
// the tasks (<= 4096)
cudaError_t lu_blocked(const LuTask* d_tasks, int ntasks, int maxm, int prec,
                       int* d_status, cudaStream_t s);
cudaError_t select_rank(const SelTask* d_tasks, int ntasks, cudaStream_t s);
// one thread-block cluster of up to cmax (<= 16) CTAs per task
cudaError_t pchol_wy(const PcholTask* d_tasks, int ntasks, int maxp, int cmax, cudaStream_t s,
                     int* csize_used = nullptr);
// one CTA per task
// maxrows / maxkb: the largest panel of the launch; launches whose largest
// panel fits in 200 KB factorize their panels in shared memory
cudaError_t lu_panel(const PanelTask* d_tasks, int ntasks, int prec, int maxrows, int maxkb, int* d_status,
                     cudaStream_t s);
// the row interchanges of several panels, each on its own column range
struct SwapTask {
  void* A;
  const int* ipiv;
  int lda, row0, kb, c0, c1, reverse;
};
cudaError_t swap_rows_batch(const SwapTask* d_tasks, int ntasks, int prec, cudaStream_t s);
// apply the row interchanges ipiv[0:kb] (rows row0+j <-> ipiv[j]) to the
// columns [c0, c1) of A (ld lda), in order (forward) or reversed
cudaError_t swap_rows(void* A, int lda, const int* ipiv, int row0, int kb,
                      int c0, int c1, int prec, int reverse, cudaStream_t s);

// pts / sq in tree order; w = s k^2 h^3 / (4 pi)
cudaError_t kernel_gram(const KGramTask* d_tasks, const KGramTile* d_tiles,
                        int ntiles, const double* d_pts, const double* d_sq,
                        double k, double w, cudaStream_t s);

// A[i, i] = v for i < n (other entries untouched)
cudaError_t set_diag(void* A, int lda, int n, int prec, double v, cudaStream_t s);

// Vector helpers: y[perm-gathered] etc.
//  gather : out[p + col*N] = scale(in[perm[p] + col*ldi]) * in[...]
cudaError_t permute_scale(const void* in, void* out, const int64_t* d_perm,
                          const double* d_scale, int64_t N, int nrhs,
                          int in_prec, int out_prec, int inverse, int conj,
                          cudaStream_t s);
// column-wise squared norms (FP64) of an N x nrhs complex128 matrix
cudaError_t col_norms2(const cd* x, int64_t N, int nrhs, double* d_out,
                       cudaStream_t s);
// y = a - b   (complex128, N x nrhs contiguous)
cudaError_t axpby(const cd* a, const cd* b, cd* y, int64_t n, double alpha,
                  double beta, cudaStream_t s);
// FrobTask.out = sum of ||block||_F^2 (blocks complex128 or complex64);
// d_part: nblocks doubles of scratch
cudaError_t frob2(const FrobTask* d_tasks, int ntasks, const FrobBlock* d_blocks, int nblocks, double* d_part,
                  int prec, cudaStream_t s);
// grad[i] (=|+=) alpha / sqchi[i]^2 * sum_c Re(x[i,c] conj(mu[i,c] - g[i,c]))
// (g may be null); all in the caller's (global) order
cudaError_t grad_chi(const cd* x, const cd* mu, const cd* g, const double* sqchi,
                     int64_t N, int nrhs, double alpha, double* grad,
                     int accumulate, cudaStream_t s);
// convert complex128 <-> complex64 (contiguous)
cudaError_t convert(const void* in, int in_prec, void* out, int out_prec,
                    int64_t n, cudaStream_t s);

}  // namespace h2k
