/*
 * h2.h - C ABI of libh2, a GB300 (sm_103a) implementation of the
 * accuracy-controlled direct solver for general H^2 matrices of
 * Ma & Jiao (2017): level-by-level factorization with cluster-basis update
 * from the fill-ins, its explicit inverse, forward / backward substitution,
 * and the H^2 matrix-vector product.
 *
 * Conventions shared by every entry point
 *   - Complex numbers are interleaved (re, im) pairs: complex128 = 2 doubles.
 *   - Vectors are N x nrhs, column-major, in the GLOBAL point order that the
 *     caller used for the points (the library applies its tree permutation).
 *   - Every call returns an h2_status; nothing throws across the ABI.  After
 *     an error, h2_last_error(ctx) holds a message; a context whose
 *     factorization failed stays valid for h2_matvec, h2_stats and
 *     h2_destroy (its factors are dropped).
 *   - Device pointers must be CUDA device (or managed) memory of the current
 *     device unless the H2_HOST flag says they are host memory.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  All
 *     work of a call is enqueued on it; calls return after it finished.
 *   - The caller owns every buffer it passes in; the library copies what it
 *     keeps.  The context owns all of its device arenas.
 */
#ifndef H2_H
#define H2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct h2_ctx h2_ctx;

typedef enum {
  H2_OK = 0,
  H2_EINVAL = -1,     /* bad argument (sizes, NULL, flags)                  */
  H2_ENOMEM = -2,     /* device or host allocation failed, or arena cap hit */
  H2_ESINGULAR = -3,  /* zero pivot in a partial LU or in the final LU      */
  H2_ENOCONV = -4,    /* refinement did not reach the tolerance             */
  H2_ETIMEOUT = -5,   /* a bounded device-side wait ran out                 */
  H2_ECUDA = -6,      /* a CUDA runtime call failed                         */
  H2_EINTERNAL = -7,  /* broken internal invariant (message says which)     */
  H2_ESTATE = -8      /* call out of order (e.g. solve before factorize)    */
} h2_status;

/* Precision of the factorization bulk (Steps 2-3, fill-ins, factors, solve).
 * Rank decisions (Step 0-1: Gram, eigen-decomposition, complement) and the
 * H^2 matvec always run in FP64. */
typedef enum { H2_FP64 = 0, H2_MIXED = 1 /* complex64 bulk */ } h2_prec;

/* Elimination order inside a level (Sec. III: "from the left to the right
 * across all the clusters"). COLORED processes the colour classes of the
 * near-field graph in increasing colour, each class as one batch. */
typedef enum { H2_ORDER_COLORED = 0, H2_ORDER_NATURAL = 1 } h2_order;

/* Flags of h2_solve / h2_matvec. */
#define H2_ADJOINT 1u      /* solve A^H x = b / multiply by A^H              */
#define H2_REFINE 2u       /* iterative refinement against the FP64 matvec   */
#define H2_USE_INVERSE 4u  /* apply the explicit inverse of h2_invert        */
#define H2_HOST 8u         /* b / x (or x / y) are HOST pointers             */

typedef struct {
  int leafsize;          /* cluster tree leaf size (default 64)             */
  double eta;            /* admissibility ||c_t-c_s|| >= eta (r_t+r_s) (1.0) */
  double sign;           /* s in A = I + s K D_chi (default +1)             */
  int ordering;          /* h2_order (default H2_ORDER_COLORED)             */
  int proxy_min;         /* construction of h2_build: 0 (default) samples
                            each cluster's whole far field (O(N^2) kernel
                            evaluations); > 0 samples the far-field points
                            within proxy_radius * r_t of the cluster centre
                            plus proxy points on two spheres (radii R and
                            0.8 R, R = proxy_radius * r_t), at least
                            proxy_min per sphere (O(N k^2))                */
  double proxy_radius;   /* proxy sphere radius / cluster radius (3.0)      */
  size_t arena_cap_bytes;/* 0 = unlimited; else H2_ENOMEM beyond it         */
  int host_only;         /* 1: h2_build keeps the representation on the host
                            only (no GPU needed); such a context allows
                            h2_export, h2_stats and h2_destroy only         */
  int profile;           /* 1: bracket every kernel launch with CUDA events
                            on the call's stream and report per-kernel-class
                            launches, device time and algorithmic flops in
                            h2_stats ("kernels"); 2: the same, kept apart
                            per tree level ("tag@l"); 0 (default): off      */
  int apply_path;        /* Step 2 and panel applications (Alg. 3, Alg. 4):
                            0 (default) automatic (currently 2), 1 in-place
                            kernel (one CTA per column / row strip), 2
                            batched GEMM into a workspace, then copied back */
  int solve_graph;       /* 1: the forward / backward sweeps of repeated
                            solves (same vectors, nrhs, direction, factors)
                            are captured once into a CUDA graph and replayed;
                            0 (default): launched one by one              */
  int split_target;      /* batched GEMM: split the K range of long products
                            until a launch has about this many CTAs
                            (0 = default, 8 per SM)                         */
  int cluster_max;       /* Step 0: most CTAs in the thread-block cluster of
                            one subspace / eigen problem (1..16; 0 = 16)    */
  int tile_policy;       /* batched GEMM tile shape: 0 (default) least padded
                            work per launch; 1 64 x 64 (64 x 16 when every
                            output has <= 16 columns)                      */
  int tensor_cores;      /* complex64 64 x 64 GEMM tiles of the mixed bulk:
                            2 (default): tcgen05 MMAs with the accumulator
                            in tensor memory; 1: warp-level TF32 MMAs; both
                            split each operand into TF32 hi + lo parts
                            (FP32 accuracy); 0: FP32 FMA pipe             */
  int gram_emulation;    /* Step-0 Grams of complex64 operands (FP64
                            accumulation): 1 (default) on the FP32 pipe, as
                            exact products summed in double-float and
                            flushed to FP64 every 8 terms; 0: FP64 FMAs   */
  int eig_solver;        /* Step-0 eigen-decomposition (eq. 17): 0
                            cyclic Jacobi of the Ritz matrix; 1
                            Householder reduction of the Ritz matrix to
                            real tridiagonal form + implicit QL with
                            accumulated rotations (orders up to 452,
                            Jacobi above); 2 (default) one-sided Jacobi
                            SVD of the
                            Cholesky factor R (squared singular values =
                            eigenvalues of L L^H, within trace(E) of those
                            of G'), double-float on the FP32 pipe (orders
                            up to 327, Jacobi above)                      */
  int stop_level;        /* early stop (Sec. III-C, last paragraph): 0
                            (default) factorize levels L .. l0; s > l0:
                            levels L .. s only, the remaining matrix of all
                            level-s pairs (couplings of ancestor blocks
                            expressed in the level-s bases) is the final
                            dense block; clamped to [l0, L]                 */
  double proxy_margin;   /* proxy construction: a proxy point is placed only
                            within this angle (radians, default 0.3) of the
                            angular extent of some far-field node outside
                            the proxy sphere, as seen from the cluster centre */
  int matvec_emulation;  /* products of the FP64 H^2 matvec: 1 (default)
                            in double-float on the FP32 pipe (operands split
                            into two FP32 parts, ~1e-13 relative error) for
                            the residuals of refined solves with tol >=
                            1e-11, FP64 FMAs elsewhere; 2: also h2_matvec;
                            0: FP64 FMAs everywhere                        */
  int ldlt;              /* elimination form: 2 (default) block LDL^T for
                            FP64 factorizations of a complex-symmetric
                            matrix, block LU for mixed-precision ones; 1
                            block LDL^T for both precisions; 0 block LU
                            always (eq. 34, both panels L^-1 P Z_i'c and
                            Z_ci' U^-1 kept).  LDL^T needs Z^T = Z (always
                            for h2_build, for h2_load when every block
                            equals the transpose of its mirror); a batch
                            uses it when all its instances qualify.  With
                            a complex64 bulk its rounding error is larger
                            than LU's (1.4x at 262,144 unknowns; at
                            884,736 unknowns, eps 1e-4, the refinement did
                            not converge), hence the default.
                            LDL^T keeps one block of each off-diagonal
                            pair, the raw block row Z_i'c and the pivoted
                            LU of F = Z_i'i' as the factor (F^-1 applied
                            as U^-1 L^-1 P), and forms the Schur updates of
                            one triangle of the target pairs: the same
                            Step-0 decisions and solution
                            as LU in exact arithmetic with about half the
                            near-field factor memory; h2_stats "ldlt"
                            reports the form of the last factorization    */
} h2_opts;

/* Fill `o` with the defaults listed above. */
void h2_default_opts(h2_opts* o);

/*
 * h2_build - H^2 representation of the scalar volume-integral-equation
 * matrix A = I + s K D_chi on the points (Sec. II, eqs. 1-3; the paper
 * builds its H^2 matrices with its refs. [14],[15], not described there):
 *   K_ij = k^2 h^3 exp(-j k r_ij)/(4 pi r_ij) (i != j),
 *   K_ii = (1 + j k a) exp(-j k a) - 1,  a = (3/(4 pi))^(1/3) h.
 * The library factorizes the complex-symmetric Z = D^{1/2} A D^{-1/2}
 * (chi_i > 0 required) and maps A x = b onto Z (D^{1/2} x) = D^{1/2} b.
 *
 *   pts     HOST, N x 3 row-major doubles (x, y, z per point)
 *   k, h    wavenumber and cell size
 *   chi     HOST, chi_len doubles: chi_len == N (per cell) or 1 (uniform)
 *   eps     construction accuracy (relative, per cluster sample)
 *   opts    NULL = defaults
 *   stream  cudaStream_t for the uploads
 *   out     receives the new context (NULL on error)
 */
h2_status h2_build(const double* pts, int64_t N, double k, double h,
                   const double* chi, int64_t chi_len, double eps,
                   const h2_opts* opts, void* stream, h2_ctx** out);

/*
 * h2_load - import an explicit H^2 matrix (e.g. from another constructor).
 * All arrays are HOST memory; complex arrays are complex128, column-major.
 *   N, L, l0     size, leaf depth, first level with admissible blocks; the
 *                cluster tree is complete: level l has 2^l clusters, cluster
 *                c has children 2c, 2c+1; leaves are contiguous in tree order
 *   perm         N int64: perm[p] = global index of tree position p
 *   leaf_size    2^L int64 point counts of the leaves
 *   rank         ranks k_c of all clusters at levels l0..L, level-major
 *                (level l0 first), 2^l entries per level
 *   V            leaf bases, concatenated: leaf c is size_c x k_c
 *   T            stacked transfers of levels l0..L-1 (level-major, cluster
 *                order): (k_2c + k_2c+1) x k_c each
 *   n_adm        admissible pair counts per level l0..L (L-l0+1 entries)
 *   adm          pairs (t, s) per level, concatenated, 2 int64 each
 *   S            couplings k_t x k_s in the same order (Z_ts = V_t S V_s^T)
 *   n_near       number of dense leaf blocks; near: pairs (t, s), 2 int64
 *   D            dense blocks size_t x size_s in the same order
 *   dscale       N doubles (global order) or NULL: the context represents
 *                A = diag(dscale)^{-1} Z diag(dscale) (NULL = identity)
 * The pairs must partition the matrix (every entry in exactly one block).
 */
h2_status h2_load(int64_t N, int L, int l0, const int64_t* perm,
                  const int64_t* leaf_size, const int64_t* rank,
                  const double* V, const double* T, const int64_t* n_adm,
                  const int64_t* adm, const double* S, int64_t n_near,
                  const int64_t* near, const double* D, const double* dscale,
                  const h2_opts* opts, void* stream, h2_ctx** out);

/*
 * h2_factorize - Algorithm 1 of the paper (Steps 0-3 per cluster, eqs.
 * 4-33; coupling / transfer update and merge per level; LU of the final
 * block), giving Z = LU in the product form of eq. (34).  The partial-LU
 * diagonal blocks and the final block are also inverted explicitly (the
 * solves apply those inverses, cf. eq. 35).
 *   eps_fill  truncation of the fill-in basis update, eqs. (17)/(26)
 *   prec      h2_prec
 * Replaces any earlier factorization of the context.  H2_ESINGULAR on a zero
 * pivot.  Runs on the context's build stream.
 */
h2_status h2_factorize(h2_ctx* ctx, double eps_fill, int prec);

/*
 * h2_invert - explicit factor-form inverse of eq. (35): on top of the
 * diagonal and final-block inverses formed by h2_factorize, pre-multiplies
 * the U panels, so that H2_USE_INVERSE solves use matrix-vector products
 * only.
 * Requires a factorization (H2_ESTATE otherwise).
 */
h2_status h2_invert(h2_ctx* ctx);

/*
 * h2_solve - x = A^{-1} b by forward substitution (Algorithm 5, eqs. 36-39),
 * the final block, and backward substitution (Algorithm 6, eqs. 40-42).
 *   b, x       N x nrhs complex128, column-major, global order; x may alias b
 *   flags      H2_ADJOINT (x = A^{-H} b, the adjoint traversal of the same
 *              factors), H2_REFINE, H2_USE_INVERSE, H2_HOST
 *   tol        H2_REFINE: stop at ||b - A x|| / ||b|| <= tol (per column max)
 *   max_iter   H2_REFINE: maximum correction steps
 *   iters      out (may be NULL): refinement steps taken
 *   resid      out (may be NULL): final relative residual (max over columns)
 * H2_ENOCONV if refinement stops above tol (x holds the last iterate).
 */
h2_status h2_solve(h2_ctx* ctx, const void* b, void* x, int nrhs,
                   unsigned flags, double tol, int max_iter, int* iters,
                   double* resid, void* stream);

/*
 * h2_matvec - y = A x (or A^H x with H2_ADJOINT) with the H^2 representation
 * in FP64: upward pass through the nested bases (eq. 3), couplings (eq. 2),
 * downward pass and the dense near field.  x, y: N x nrhs complex128,
 * column-major, global order; must not alias.
 */
h2_status h2_matvec(h2_ctx* ctx, const void* x, void* y, int nrhs,
                    unsigned flags, void* stream);

/*
 * h2_matvec_noalloc - the product of h2_matvec (y = A x, or y = A^H x with
 * H2_ADJOINT) for callers that must not allocate device memory during the
 * call: for example a host thread in a real-time loop, or code whose device
 * memory is fully reserved up front, which can only call into a context set
 * up earlier.  The paper has no counterpart; this is a runtime variant of
 * h2_matvec.
 *   x, y      DEVICE, N x nrhs complex128, column-major, global order; must
 *             not alias (host buffers are not accepted)
 *   flags     0 or H2_ADJOINT
 * All temporaries (permuted vectors, level coefficients, task descriptors)
 * live in one static device array of 32 MiB that every GPU which loads the
 * library's module holds until the process exits.  Sizes whose temporaries
 * exceed it (about 2 N nrhs + 2 (sum of ranks) nrhs complex128 plus the task
 * lists) are rejected with H2_EINVAL and a message before any work is
 * enqueued.  The call makes no cudaMalloc, cudaFree or other allocating call.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress).  Under CUDA's lazy module loading (the default
 * since CUDA 12.2) that lookup also loads the module that holds the array,
 * so the 32 MiB are reserved on that device at this first call: make it
 * during set-up, before device memory is reserved up front, and before any
 * stream capture.  x or y in host memory: H2_EINVAL.  A stream that is being
 * captured: H2_ESTATE, nothing enqueued.  All calls share the array, which
 * keeps the last call's contents (every entry a call reads it writes
 * first), so calls that overlap on the GPU (other streams, other threads)
 * race: serialize them.
 */
h2_status h2_matvec_noalloc(h2_ctx* ctx, const void* x, void* y, int nrhs,
                            unsigned flags, void* stream);

/*
 * h2_factorize_batch - h2_factorize (Algorithm 1) of `count` independent
 * instances at once.  The paper factorizes one matrix; this runs the same
 * per-level work of several matrices in the same launches: for each
 * level-from-leaf index d (d = 0 at every instance's leaves) and each colour
 * class b, Steps 0-3 of all instances that have that level and class form
 * one batch (one launch per kernel), the merges of level d share launches,
 * and the final blocks are factorized together.  Instances of different
 * depth join as their levels come up.  Results equal those of h2_factorize
 * of each instance up to the summation order of the batched products.
 *   ctxs      count distinct contexts (not host_only), each built or loaded
 *   eps_fill  prec: as h2_factorize, the same for all instances
 * Runs on ctxs[0]'s stream; the host waits for it.  On error every
 * instance's factorization is invalid and ctxs[0] holds the message.
 */
h2_status h2_factorize_batch(h2_ctx* const* ctxs, int count, double eps_fill,
                             int prec);

/*
 * h2_solve_batch - h2_solve of `count` factorized instances with one
 * right-hand-side block each (all nrhs wide): the forward / backward sweeps
 * (Algorithms 5-6), the final blocks and, with H2_REFINE, the FP64 H^2
 * matvecs of the refinement run as one launch per stage for all instances.
 *   b[q], x[q]  DEVICE, N_q x nrhs complex128, column-major, global order of
 *               instance q; x[q] may alias b[q]
 *   flags       H2_ADJOINT, H2_REFINE, H2_USE_INVERSE (no H2_HOST)
 *   tol         H2_REFINE: stop when every instance's residual (max over
 *               its columns of ||b - A x|| / ||b||) is <= tol
 *   iters,resid out (may be NULL): refinement steps, largest final residual
 * H2_ENOCONV if refinement stops above tol.  Runs on `stream`; the host
 * waits for it.  Messages go to ctxs[0].
 */
h2_status h2_solve_batch(h2_ctx* const* ctxs, int count, const void* const* b,
                         void* const* x, int nrhs, unsigned flags, double tol,
                         int max_iter, int* iters, double* resid,
                         void* stream);

/*
 * h2_grad_chi - per-cell derivative of a real objective L through the solution
 * map x = A(chi)^{-1} b of the volume-integral system A = I + s K D_chi (the
 * matrix the paper's solver factors, with chi the per-cell contrast of the
 * column scaling).  The paper has no counterpart: this is the adjoint
 * (reverse-mode) derivative of its solve.  With g = dL/dx in the
 * conjugate-Wirtinger convention (dL = Re sum conj(g) dx) and mu = A^{-H} g
 * from h2_solve(..., H2_ADJOINT, ...) on the same factors,
 *   grad[i] (=|+=) alpha / chi_i * sum_c Re( x[i,c] * conj(mu[i,c] - g[i,c]) )
 * (dA/dchi_i = s K e_i e_i^T and A^H mu = g).  chi_i is the context's contrast
 * (dscale_i^2 of h2_load; the chi of h2_build).
 *   x, mu, g  DEVICE, N x nrhs complex128, column-major, global order; g may
 *             be NULL (taken as 0: the form 2 Re(x conj(lambda)) / chi of an
 *             objective whose chi-dependence outside the solve has been
 *             folded into lambda, alpha = 2)
 *   grad      DEVICE, N doubles, global order, caller-allocated
 *   flags     0, or H2_GRAD_ACCUMULATE to add into grad
 * Runs asynchronously on `stream` (one kernel, no synchronisation).
 */
#define H2_GRAD_ACCUMULATE 1u
h2_status h2_grad_chi(h2_ctx* ctx, const void* x, const void* mu,
                      const void* g, int nrhs, double alpha, double* grad,
                      unsigned flags, void* stream);

/*
 * h2_set_opts - change the run-time tunables of a context (apply_path,
 * solve_graph, split_target, cluster_max, tile_policy, tensor_cores,
 * gram_emulation, eig_solver, stop_level, matvec_emulation, ldlt, profile) without
 * rebuilding it; the other fields of *opts are ignored.  They take effect at
 * the next h2_factorize / h2_solve (captured solve graphs are retired).  No
 * counterpart in the paper: used by the autotuner.
 */
h2_status h2_set_opts(h2_ctx* ctx, const h2_opts* opts);

/*
 * h2_set_chi - new contrast chi on an existing context (the column scaling
 * D_chi of A = I + s K D_chi; Sec. II's matrix with the workload's contrast):
 * Z = D^{1/2} A D^{-1/2} becomes Z' = I + E (Z - I) E, E = diag(sqrt(chi' /
 * chi)).  The H^2 form is updated exactly (dense blocks scaled, the scaled
 * cluster bases re-orthonormalised leaf to root so they stay nested, eq. 3,
 * couplings multiplied by the triangular factors, eq. 2): ranks and the block
 * partition are unchanged, no new approximation is made, cost O(N k^2) host
 * work plus one upload.  Valid for matrices of that form (h2_build; h2_load
 * with dscale = sqrt(chi)).  The factorization and explicit inverse are
 * invalidated: call h2_factorize again before solving.
 *   chi       HOST, chi_len doubles (N, or 1 = uniform), finite and > 0
 * H2_EINVAL for a bad chi (the context is unchanged).
 */
h2_status h2_set_chi(h2_ctx* ctx, const double* chi, int64_t chi_len);

/*
 * h2_level_ranks - cluster ranks of tree level `level` (l0 <= level <= L) in
 * the last factorization: k0[i] the incoming rank k_i and kt[i] the rank
 * after the Step-0 basis update (eqs. 17-18), i = 0 .. 2^level - 1 (HOST
 * arrays of n >= 2^level entries; either may be NULL).  H2_ESTATE without a
 * valid factorization, H2_EINVAL for another level or a short array.
 */
h2_status h2_level_ranks(const h2_ctx* ctx, int level, int* k0, int* kt, int64_t n);

/*
 * h2_export - copy the H^2 representation out in the h2_load layout (HOST
 * arrays, caller-allocated).  Call h2_export_sizes first: it returns the
 * element counts (complex entries for V, T, S, D; pairs for adm / near).
 */
h2_status h2_export_sizes(const h2_ctx* ctx, int64_t* N, int* L, int* l0,
                          int64_t* nV, int64_t* nT, int64_t* nS,
                          int64_t* n_adm_total, int64_t* n_near, int64_t* nD);
h2_status h2_export(const h2_ctx* ctx, int64_t* perm, int64_t* leaf_size,
                    int64_t* rank, double* V, double* T, int64_t* n_adm,
                    int64_t* adm, double* S, int64_t* near, double* D,
                    double* dscale);

/*
 * h2_stats - JSON object with per-level sizes, ranks before / after the
 * basis update, block counts (near, admissible, fill-in, pushed), colours,
 * algorithmic flops and bytes, kernel launches, device bytes and timings of
 * the last factorization / solve.  Returns H2_EINVAL if `cap` is too small
 * (the JSON is truncated); `cap` >= 64 KiB is always enough.
 */
h2_status h2_stats(const h2_ctx* ctx, char* json, size_t cap);

/* Last error message of the context ("" if none); valid until next call. */
const char* h2_last_error(const h2_ctx* ctx);

/* Message for a status code. */
const char* h2_status_string(int status);

/* Frees the context and all of its device memory. NULL is a no-op. */
void h2_destroy(h2_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* H2_H */
