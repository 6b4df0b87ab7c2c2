// Partial LU of the leading m x m block of a near-field diagonal block with
// row pivoting (Step 3, eqs. 9-11 and Algorithm 4; pivot = largest |z| in
// the column, ties to the lowest row), followed by the explicit L^{-1} P and
// U^{-1} that the panels, the Schur updates' operands and the solve apply.
//
// One thread-block cluster per task, blocked:
//   * panels of nb columns are factorized in shared memory by the cluster's
//     first CTA (pivot search by warp shuffles, one row swap, scaling, rank-1
//     update per column);
//   * the row swaps are then applied to the other columns, U12 = L11^{-1} A12
//     with the inverse of the 32 x 32 diagonal block (formed in shared
//     memory), and the trailing block is updated, these by all CTAs of the
//     cluster over 64-column / 64 x 64 tiles with a CTA-wide tiled GEMM
//     (32-deep K slices staged in shared memory, 4 x 4 complex micro-tiles);
//   * in two more launches (one CTA per task, L or U and 32-column block) the
//     inverses of the diagonal blocks, then every column block of L^{-1} and
//     U^{-1} by block forward / back substitution with the same GEMM;
//     L^{-1} P is L^{-1} with its columns permuted.
// A zero pivot sets status bit 1 and the CTA returns.
#include <cooperative_groups.h>

#include <algorithm>

#include "h2_kernels.h"

namespace cg = cooperative_groups;

namespace h2k {
namespace {

constexpr int NT = 256;
constexpr int NBMAX = 32;            // widest panel
constexpr int TM = 64, TN = 64, TK = 32;

template <class E> struct RealOf;
template <> struct RealOf<cd> { using T = double; };
template <> struct RealOf<cf> { using T = float; };

template <class R>
struct GemmSmem {
  R ar[TK][TM], ai[TK][TM], br[TK][TN], bi[TK][TN];
};

template <class E, class R>
__device__ __forceinline__ void cmul_sub(E& acc, const E a, const E b) {
  acc.re = (decltype(acc.re))((R)acc.re - ((R)a.re * (R)b.re - (R)a.im * (R)b.im));
  acc.im = (decltype(acc.im))((R)acc.im - ((R)a.re * (R)b.im + (R)a.im * (R)b.re));
}

// C[0:M, 0:N] (=|+=) alpha * A[0:M, 0:K] B[0:K, 0:N], column-major, whole CTA.
// Every thread must call it (it synchronizes).  C must not overlap A; it may
// be B itself when M <= TM and K <= TK (each output tile then stages all of
// its B columns in shared memory before it writes them).
template <class E, class R>
__device__ void cta_gemm(E* C, int ldc, const E* A, int lda, const E* B, int ldb, int M, int N, int K, R alpha,
                         bool overwrite, GemmSmem<R>& s) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int n0 = 0; n0 < N; n0 += TN)
    for (int m0 = 0; m0 < M; m0 += TM) {
      R cr[4][4], ci[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cr[i][j] = ci[i][j] = (R)0;
      for (int k0 = 0; k0 < K; k0 += TK) {
        for (int l = tid; l < TM * TK; l += NT) {
          const int i = l % TM, k = l / TM;
          R re = 0, im = 0;
          if (m0 + i < M && k0 + k < K) {
            const E v = A[(size_t)(m0 + i) + (size_t)(k0 + k) * lda];
            re = (R)v.re;
            im = (R)v.im;
          }
          s.ar[k][i] = re;
          s.ai[k][i] = im;
        }
        for (int l = tid; l < TK * TN; l += NT) {
          const int k = l % TK, j = l / TK;
          R re = 0, im = 0;
          if (n0 + j < N && k0 + k < K) {
            const E v = B[(size_t)(k0 + k) + (size_t)(n0 + j) * ldb];
            re = (R)v.re;
            im = (R)v.im;
          }
          s.br[k][j] = re;
          s.bi[k][j] = im;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < TK; ++k) {
          R ar[4], ai[4], br[4], bi[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) { ar[i] = s.ar[k][ty + 16 * i]; ai[i] = s.ai[k][ty + 16 * i]; }
#pragma unroll
          for (int j = 0; j < 4; ++j) { br[j] = s.br[k][tx + 16 * j]; bi[j] = s.bi[k][tx + 16 * j]; }
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              cr[i][j] = fma(ar[i], br[j], fma(-ai[i], bi[j], cr[i][j]));
              ci[i][j] = fma(ar[i], bi[j], fma(ai[i], br[j], ci[i][j]));
            }
        }
        __syncthreads();
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int n = n0 + tx + 16 * j;
          if (n >= N) continue;
          E* p = C + (size_t)m + (size_t)n * ldc;
          E v;
          if (overwrite) {
            v.re = (decltype(v.re))(alpha * cr[i][j]);
            v.im = (decltype(v.im))(alpha * ci[i][j]);
          } else {
            v = *p;
            v.re = (decltype(v.re))((R)v.re + alpha * cr[i][j]);
            v.im = (decltype(v.im))((R)v.im + alpha * ci[i][j]);
          }
          *p = v;
        }
      }
    }
}

// largest |z|^2 over the block, ties to the lowest index; result in (wv[0], wi[0])
template <class R>
__device__ void cta_argmax(R v, int i, R* wv, int* wi) {
  for (int o = 16; o > 0; o >>= 1) {
    const R ov = __shfl_down_sync(0xffffffffu, v, o);
    const int oi = __shfl_down_sync(0xffffffffu, i, o);
    if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
  }
  if ((threadIdx.x & 31) == 0) { wv[threadIdx.x >> 5] = v; wi[threadIdx.x >> 5] = i; }
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < NT / 32 ? wv[threadIdx.x] : (R)-1;
    i = threadIdx.x < NT / 32 ? wi[threadIdx.x] : 0x7fffffff;
    for (int o = 16; o > 0; o >>= 1) {
      const R ov = __shfl_down_sync(0xffffffffu, v, o);
      const int oi = __shfl_down_sync(0xffffffffu, i, o);
      if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
    }
    if (threadIdx.x == 0) { wv[0] = v; wi[0] = i; }
  }
  __syncthreads();
}

// Ds = inverse of the unit lower (upper = false) or upper (upper = true)
// triangle of the ib x ib block Ls (both ld NBMAX, shared memory); one column
// per thread.  The caller synchronizes before and after.
template <class E, class R>
__device__ void diag_inverse(const E* Ls, int ib, E* Ds, bool upper) {
  const int c = threadIdx.x;
  if (c >= ib) return;
  if (!upper) {
    for (int r = 0; r < ib; ++r) {
      E v;
      v.re = (r == c) ? 1 : 0;
      v.im = 0;
      for (int q = c; q < r; ++q) cmul_sub<E, R>(v, Ls[r + q * NBMAX], Ds[q + c * NBMAX]);
      Ds[r + c * NBMAX] = v;
    }
  } else {
    for (int r = ib - 1; r >= 0; --r) {
      E v;
      v.re = (r == c) ? 1 : 0;
      v.im = 0;
      if (r <= c) {
        for (int q = r + 1; q <= c; ++q) cmul_sub<E, R>(v, Ls[r + q * NBMAX], Ds[q + c * NBMAX]);
        const E d = Ls[r + r * NBMAX];
        const R dd = (R)d.re * (R)d.re + (R)d.im * (R)d.im;
        const R ir = (R)d.re / dd, ii = -(R)d.im / dd;
        const R vr = (R)v.re * ir - (R)v.im * ii, vi = (R)v.re * ii + (R)v.im * ir;
        v.re = vr;
        v.im = vi;
      }
      Ds[r + c * NBMAX] = v;
    }
  }
}

// cluster-wide barrier: arrive with release, wait with acquire (cluster scope)
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// One thread-block cluster of C CTAs per task.  Per panel of nb columns:
//   1. CTA 0 factorizes the panel in its shared memory (pivot search, swap,
//      scaling, rank-1 updates) and writes it back; its pivots and a failure
//      flag stay in its shared memory;
//   2. after a cluster barrier every CTA reads the pivots through distributed
//      shared memory and, for the 64-column tiles it owns (tile q belongs to
//      CTA q mod C), applies the row swaps and forms U12 = L11^{-1} A12 (L11^{-1}
//      computed by each CTA from the panel);
//   3. after a cluster barrier the 64 x 64 tiles of A22 -= L21 U12 are dealt
//      round-robin over the CTAs; a third barrier precedes the next panel.
template <class E>
__global__ void __launch_bounds__(NT) k_lu_cl(const LuTask* __restrict__ tasks, int nb, int maxm, int* status) {
  using R = typename RealOf<E>::T;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  extern __shared__ __align__(16) unsigned char smraw[];
  GemmSmem<R>& gs = *reinterpret_cast<GemmSmem<R>*>(smraw);
  E* Ls = reinterpret_cast<E*>(smraw + sizeof(GemmSmem<R>));  // NBMAX x NBMAX, ld NBMAX
  E* Ds = Ls + NBMAX * NBMAX;                                  // NBMAX x NBMAX, ld NBMAX
  E* Pn = Ds + NBMAX * NBMAX;                                  // panel, (m - j0) x nb (CTA 0)
  int* perm = reinterpret_cast<int*>(Pn + (size_t)maxm * nb);  // m (CTA 0)
  const LuTask t = tasks[blockIdx.x / C];
  const int m = t.m, ld = t.lda;
  __shared__ R wv[NT / 32];
  __shared__ int wi[NT / 32];
  __shared__ int spiv[NBMAX], lpiv[NBMAX];
  __shared__ int fail;
  const int tid = threadIdx.x;
  E* A = (E*)t.A;
  if (rank == 0) {
    for (int i = tid; i < m; i += NT) perm[i] = i;
    if (tid == 0) fail = 0;
  }
  __syncthreads();
  int* spiv0 = cl.map_shared_rank(spiv, 0);
  int* fail0 = cl.map_shared_rank(&fail, 0);

  for (int j0 = 0; j0 < m; j0 += nb) {
    const int jb = min(nb, m - j0), pl = m - j0;
    // ------------------------------------------------ 1. panel (CTA 0)
    if (rank == 0) {
      for (int idx = tid; idx < pl * jb; idx += NT) {
        const int r = idx % pl, c = idx / pl;
        Pn[idx] = A[(size_t)(j0 + r) + (size_t)(j0 + c) * ld];
      }
      __syncthreads();
      for (int jj = 0; jj < jb; ++jj) {
        R best = -1;
        int bi = 0x7fffffff;
        for (int r = jj + tid; r < pl; r += NT) {
          const E v = Pn[r + jj * pl];
          const R a = (R)v.re * (R)v.re + (R)v.im * (R)v.im;
          if (a > best) { best = a; bi = r; }
        }
        cta_argmax<R>(best, bi, wv, wi);
        const int pr = wi[0];
        const R pv = wv[0];
        __syncthreads();
        if (!(pv > (R)0)) {
          if (tid == 0) {
            fail = 1;
            if (status) atomicMax(status, 1);
          }
          break;
        }
        if (tid == 0) {
          spiv[jj] = pr;
          if (pr != jj) {
            const int x = perm[j0 + jj];
            perm[j0 + jj] = perm[j0 + pr];
            perm[j0 + pr] = x;
          }
        }
        if (pr != jj && tid < jb) {
          const E a = Pn[jj + tid * pl];
          Pn[jj + tid * pl] = Pn[pr + tid * pl];
          Pn[pr + tid * pl] = a;
        }
        __syncthreads();
        const E d = Pn[jj + jj * pl];
        const R dd = (R)d.re * (R)d.re + (R)d.im * (R)d.im;
        const R ir = (R)d.re / dd, ii = -(R)d.im / dd;
        for (int r = jj + 1 + tid; r < pl; r += NT) {
          E v = Pn[r + jj * pl];
          const R vr = (R)v.re * ir - (R)v.im * ii, vi = (R)v.re * ii + (R)v.im * ir;
          v.re = vr;
          v.im = vi;
          Pn[r + jj * pl] = v;
        }
        __syncthreads();
        const int rem = pl - jj - 1, pc = jb - jj - 1;
        for (int idx = tid; idx < rem * pc; idx += NT) {
          const int r = jj + 1 + idx % rem, c = jj + 1 + idx / rem;
          E v = Pn[r + c * pl];
          cmul_sub<E, R>(v, Pn[r + jj * pl], Pn[jj + c * pl]);
          Pn[r + c * pl] = v;
        }
        __syncthreads();
      }
      __syncthreads();
      if (!fail)
        for (int idx = tid; idx < pl * jb; idx += NT) {
          const int r = idx % pl, c = idx / pl;
          A[(size_t)(j0 + r) + (size_t)(j0 + c) * ld] = Pn[idx];
        }
    }
    cluster_barrier();
    if (*fail0) break;
    // ----------------------- 2. swaps and U12 on the own 64-column tiles
    if (tid < jb) lpiv[tid] = spiv0[tid];
    __syncthreads();
    const int rest = m - j0 - jb;
    const int ntile = (m + 63) / 64;
    for (int q = rank; q < ntile; q += C) {
      const int c0 = q * 64, c1 = min(m, c0 + 64);
      for (int c = c0 + tid; c < c1; c += NT) {
        if (c >= j0 && c < j0 + jb) continue;
        E* x = A + (size_t)c * ld;
        for (int u = 0; u < jb; ++u) {
          const int pr = lpiv[u];
          if (pr == u) continue;
          const E a = x[j0 + u];
          x[j0 + u] = x[j0 + pr];
          x[j0 + pr] = a;
        }
      }
    }
    if (rest > 0) {
      for (int idx = tid; idx < jb * jb; idx += NT)
        Ls[(idx % jb) + (idx / jb) * NBMAX] = A[(size_t)(j0 + idx % jb) + (size_t)(j0 + idx / jb) * ld];
      __syncthreads();
      diag_inverse<E, R>(Ls, jb, Ds, false);
      __syncthreads();
      // U12 = L11^{-1} A12 (unit lower L11), in place, own tiles of the
      // columns j0 + jb .. m (the swaps above touched the same columns)
      const int cb = j0 + jb;
      for (int q = rank; q < ntile; q += C) {
        const int c0 = max(q * 64, cb), c1 = min(m, q * 64 + 64);
        if (c0 >= c1) continue;
        cta_gemm<E, R>(A + (size_t)j0 + (size_t)c0 * ld, ld, Ds, NBMAX, A + (size_t)j0 + (size_t)c0 * ld, ld, jb,
                       c1 - c0, jb, (R)1, true, gs);
        __syncthreads();
      }
    }
    cluster_barrier();
    // ------------------------------------ 3. A22 -= L21 U12, dealt by tiles
    if (rest > 0) {
      const int cb = j0 + jb;
      const int nt = (rest + 63) / 64;
      for (int q = rank; q < nt * nt; q += C) {
        const int tm = q % nt, tn = q / nt;
        const int r0 = cb + tm * 64, c0 = cb + tn * 64;
        cta_gemm<E, R>(A + (size_t)r0 + (size_t)c0 * ld, ld, A + (size_t)r0 + (size_t)j0 * ld, ld,
                       A + (size_t)j0 + (size_t)c0 * ld, ld, min(64, m - r0), min(64, m - c0), jb, (R)-1, false, gs);
        __syncthreads();
      }
    }
    cluster_barrier();
  }
  if (rank == 0 && !fail)
    for (int i = tid; i < m; i += NT) t.piv[i] = perm[i];
  // no CTA leaves while another may still read CTA 0's shared memory
  cluster_barrier();
}

// The explicit inverses from the packed LU of k_lu_cl, in two launches over
// (task, L or U, 32-column block J):
//   1. k_lu_dinv: the inverse of the diagonal block J of the unit lower L or
//      of U, into the diagonal block of X (the L^{-1} scratch) or of U^{-1};
//   2. k_lu_inv_cols: the rest of column block J, independently of the other
//      blocks -- L^{-1} E_J by forward substitution over the block rows below
//      J, X[I, J] = -D_I L[I, J0:I0] X[J0:I0, J] (D_I = L_II^{-1} from launch
//      1); U^{-1} E_J by back substitution over the block rows above J,
//      Y[I, J] = -D_I U[I, I1:J1] Y[I1:J1, J] (D_I = U_II^{-1}); then the
//      columns of L^{-1} go to their permuted places in L^{-1} P.
// Every CTA writes only its own column block (launch 2 reads the diagonal
// blocks of the others, written by launch 1).
template <class E>
__global__ void __launch_bounds__(NT) k_lu_dinv(const LuTask* __restrict__ tasks, int maxblk) {
  using R = typename RealOf<E>::T;
  __shared__ E Ls[NBMAX * NBMAX], Ds[NBMAX * NBMAX];
  const LuTask t = tasks[blockIdx.x / (2 * maxblk)];
  const int rest = blockIdx.x % (2 * maxblk);
  const bool upper = (rest & 1) != 0;
  const int J = rest >> 1, m = t.m, ld = t.lda;
  const int J0 = J * NBMAX;
  if (J0 >= m) return;
  const int jb = min(NBMAX, m - J0);
  const E* A = (const E*)t.A;
  for (int idx = threadIdx.x; idx < jb * jb; idx += NT) {
    const int r = idx % jb, c = idx / jb;
    Ls[r + c * NBMAX] = A[(size_t)(J0 + r) + (size_t)(J0 + c) * ld];
  }
  __syncthreads();
  diag_inverse<E, R>(Ls, jb, Ds, upper);
  __syncthreads();
  E* Y = upper ? (E*)t.Uinv : (E*)t.scratch;
  for (int idx = threadIdx.x; idx < jb * jb; idx += NT) {
    const int r = idx % jb, c = idx / jb;
    Y[(size_t)(J0 + r) + (size_t)(J0 + c) * m] = Ds[r + c * NBMAX];
  }
}

template <class E>
__global__ void __launch_bounds__(NT) k_lu_inv_cols(const LuTask* __restrict__ tasks, int maxblk) {
  using R = typename RealOf<E>::T;
  extern __shared__ __align__(16) unsigned char smraw[];
  GemmSmem<R>& gs = *reinterpret_cast<GemmSmem<R>*>(smraw);
  E* Ds = reinterpret_cast<E*>(smraw + sizeof(GemmSmem<R>));  // NBMAX x NBMAX, ld NBMAX
  const LuTask t = tasks[blockIdx.x / (2 * maxblk)];
  const int rest = blockIdx.x % (2 * maxblk);
  const bool upper = (rest & 1) != 0;
  const int J = rest >> 1, m = t.m, ld = t.lda;
  const int J0 = J * NBMAX;
  if (J0 >= m) return;
  const int jb = min(NBMAX, m - J0), J1 = J0 + jb;
  const int tid = threadIdx.x;
  const E* A = (const E*)t.A;
  E zero;
  zero.re = 0;
  zero.im = 0;
  auto load_d = [&](const E* Y, int I0, int ib) {
    for (int idx = tid; idx < ib * ib; idx += NT) {
      const int r = idx % ib, c = idx / ib;
      Ds[r + c * NBMAX] = Y[(size_t)(I0 + r) + (size_t)(I0 + c) * m];
    }
    __syncthreads();
  };
  if (!upper) {
    E* X = (E*)t.scratch;  // L^{-1}, m x m
    for (int idx = tid; idx < J0 * jb; idx += NT) X[(size_t)(idx % J0) + (size_t)(J0 + idx / J0) * m] = zero;
    __syncthreads();
    for (int I0 = J1; I0 < m; I0 += NBMAX) {
      const int ib = min(NBMAX, m - I0);
      cta_gemm<E, R>(X + I0 + (size_t)J0 * m, m, A + I0 + (size_t)J0 * ld, ld, X + J0 + (size_t)J0 * m, m, ib, jb,
                     I0 - J0, (R)-1, true, gs);
      __syncthreads();
      load_d(X, I0, ib);
      cta_gemm<E, R>(X + I0 + (size_t)J0 * m, m, Ds, NBMAX, X + I0 + (size_t)J0 * m, m, ib, jb, ib, (R)1, true, gs);
      __syncthreads();
    }
    // L^{-1} P: column r of L^{-1} is column piv[r] of the result (every
    // thread's rows of the block, zeroed or computed, are written by now)
    __syncthreads();
    E* Lp = (E*)t.Linv;
    for (int idx = tid; idx < m * jb; idx += NT) {
      const int i = idx % m, r = J0 + idx / m;
      Lp[(size_t)i + (size_t)t.piv[r] * m] = X[(size_t)i + (size_t)r * m];
    }
    return;
  }
  E* Y = (E*)t.Uinv;
  for (int idx = tid; idx < (m - J1) * jb; idx += NT)
    Y[(size_t)(J1 + idx % (m - J1)) + (size_t)(J0 + idx / (m - J1)) * m] = zero;
  __syncthreads();
  for (int bI = J - 1; bI >= 0; --bI) {
    const int I0 = bI * NBMAX, I1 = I0 + NBMAX;
    cta_gemm<E, R>(Y + I0 + (size_t)J0 * m, m, A + I0 + (size_t)I1 * ld, ld, Y + I1 + (size_t)J0 * m, m, NBMAX, jb,
                   J1 - I1, (R)-1, true, gs);
    __syncthreads();
    load_d(Y, I0, NBMAX);
    cta_gemm<E, R>(Y + I0 + (size_t)J0 * m, m, Ds, NBMAX, Y + I0 + (size_t)J0 * m, m, NBMAX, jb, NBMAX, (R)1, true,
                   gs);
    __syncthreads();
  }
}

template <class E>
size_t lu_smem(int maxm, int nb) {
  using R = typename RealOf<E>::T;
  return sizeof(GemmSmem<R>) + 2 * (size_t)NBMAX * NBMAX * sizeof(E) + (size_t)maxm * nb * sizeof(E) +
         (size_t)maxm * sizeof(int) + 16;
}

template <class E>
size_t lu_inv_smem() {
  using R = typename RealOf<E>::T;
  return sizeof(GemmSmem<R>) + (size_t)NBMAX * NBMAX * sizeof(E) + 16;
}

template <class E>
cudaError_t launch_lu(const LuTask* d, int n, int maxm, int* st, cudaStream_t s) {
  // panel width: as wide as the shared-memory budget allows (at most 32)
  constexpr size_t kPanelBytes = 104 * 1024;
  int nb = (int)std::min<size_t>(NBMAX, kPanelBytes / ((size_t)std::max(maxm, 1) * sizeof(E)));
  if (nb < 1) return cudaErrorInvalidValue;
  const size_t sm = lu_smem<E>(maxm, nb);
  if (sm > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_lu_cl<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  // CTAs per task: about one per 64 x 64 tile of the first trailing update,
  // at most 16, and the launch's clusters within the 152 SMs
  const int tiles = (maxm + 63) / 64;
  int csize = std::max(1, std::min(std::min(16, tiles * tiles), 152 / std::max(n, 1)));
  if (csize > 8) {
    cudaFuncSetAttribute(k_lu_cl<E>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t q = {};
    q.gridDim = dim3(csize, 1, 1);
    q.blockDim = dim3(NT, 1, 1);
    q.dynamicSmemBytes = sm;
    cudaLaunchAttribute qa[1];
    qa[0].id = cudaLaunchAttributeClusterDimension;
    qa[0].val.clusterDim.x = csize;
    qa[0].val.clusterDim.y = 1;
    qa[0].val.clusterDim.z = 1;
    q.attrs = qa;
    q.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, k_lu_cl<E>, &q) != cudaSuccess || ncl < 1) {
      cudaGetLastError();
      csize = 8;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n * csize, 1, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, k_lu_cl<E>, d, nb, maxm, st);
  if (e != cudaSuccess) return e;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int maxblk = (maxm + NBMAX - 1) / NBMAX;
  k_lu_dinv<E><<<2 * maxblk * n, NT, 0, s>>>(d, maxblk);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smi = lu_inv_smem<E>();
  cudaFuncSetAttribute(k_lu_inv_cols<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smi);
  k_lu_inv_cols<E><<<2 * maxblk * n, NT, smi, s>>>(d, maxblk);
  return cudaGetLastError();
}

}  // namespace

cudaError_t lu_blocked(const LuTask* d, int n, int maxm, int prec, int* st, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (maxm > 4096) return cudaErrorInvalidValue;
  return prec == P64 ? launch_lu<cd>(d, n, maxm, st, s) : launch_lu<cf>(d, n, maxm, st, s);
}

}  // namespace h2k
