// Partial LU of the leading m x m block of a near-field diagonal block with
// row pivoting (Step 3, eqs. 9-11 and Algorithm 4; pivot = largest |z| in
// the column, ties to the lowest row), followed by the explicit L^{-1} P and
// U^{-1} that the panels, the Schur updates' operands and the solve apply.
//
// One CTA per task, blocked:
//   * panels of nb columns are factorized in shared memory (pivot search by
//     warp shuffles, one row swap, scaling, rank-1 update per column);
//   * the row swaps are then applied to the other columns, U12 = L11^{-1} A12
//     with the inverse of the 32 x 32 diagonal block (formed in shared
//     memory), and the trailing block is updated by a CTA-wide tiled GEMM
//     (64 x 64 output tiles, 32-deep K slices staged in shared memory, 4 x 4
//     complex micro-tiles);
//   * in a second launch (two CTAs per task, concurrently) L^{-1} and U^{-1}
//     are formed block row by block row with the same GEMM
//     (X[I, :I] = -L[I,I]^{-1} L[I, :I] X[:I, :I]); L^{-1} P is L^{-1} with
//     its columns permuted.
// A zero pivot sets status bit 1 and the CTA returns.
#include <algorithm>

#include "h2_kernels.h"

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

template <class E>
__global__ void __launch_bounds__(NT) k_lu_blk(const LuTask* __restrict__ tasks, int nb, int maxm, int* status) {
  using R = typename RealOf<E>::T;
  extern __shared__ __align__(16) unsigned char smraw[];
  GemmSmem<R>& gs = *reinterpret_cast<GemmSmem<R>*>(smraw);
  E* Ls = reinterpret_cast<E*>(smraw + sizeof(GemmSmem<R>));  // NBMAX x NBMAX, ld NBMAX
  E* Ds = Ls + NBMAX * NBMAX;                                  // NBMAX x NBMAX, ld NBMAX
  E* Pn = Ds + NBMAX * NBMAX;                                  // panel, (m - j0) x nb
  int* perm = reinterpret_cast<int*>(Pn + (size_t)maxm * nb);  // m
  const LuTask t = tasks[blockIdx.x];
  const int m = t.m, ld = t.lda;
  __shared__ R wv[NT / 32];
  __shared__ int wi[NT / 32];
  __shared__ int spiv[NBMAX];
  const int tid = threadIdx.x;
  E* A = (E*)t.A;
  for (int i = tid; i < m; i += NT) perm[i] = i;
  __syncthreads();

  // ------------------------------------------------------------ LU ------
  for (int j0 = 0; j0 < m; j0 += nb) {
    const int jb = min(nb, m - j0), pl = m - j0;
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
        if (tid == 0 && status) atomicMax(status, 1);
        return;
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
    for (int idx = tid; idx < pl * jb; idx += NT) {
      const int r = idx % pl, c = idx / pl;
      A[(size_t)(j0 + r) + (size_t)(j0 + c) * ld] = Pn[idx];
    }
    // the panel's row swaps on every other column
    for (int c = tid; c < m; c += NT) {
      if (c >= j0 && c < j0 + jb) continue;
      for (int q = 0; q < jb; ++q) {
        const int pr = spiv[q];
        if (pr == q) continue;
        E* x = A + (size_t)c * ld;
        const E a = x[j0 + q];
        x[j0 + q] = x[j0 + pr];
        x[j0 + pr] = a;
      }
    }
    __syncthreads();
    const int rest = m - j0 - jb;
    if (rest > 0) {
      for (int idx = tid; idx < jb * jb; idx += NT) Ls[(idx % jb) + (idx / jb) * NBMAX] = Pn[(idx % jb) + (idx / jb) * pl];
      __syncthreads();
      // U12 = L11^{-1} A12 (unit lower L11), in place
      diag_inverse<E, R>(Ls, jb, Ds, false);
      __syncthreads();
      cta_gemm<E, R>(A + (size_t)j0 + (size_t)(j0 + jb) * ld, ld, Ds, NBMAX, A + (size_t)j0 + (size_t)(j0 + jb) * ld,
                     ld, jb, rest, jb, (R)1, true, gs);
      __syncthreads();
      cta_gemm<E, R>(A + (size_t)(j0 + jb) + (size_t)(j0 + jb) * ld, ld, A + (size_t)(j0 + jb) + (size_t)j0 * ld, ld,
                     A + (size_t)j0 + (size_t)(j0 + jb) * ld, ld, rest, rest, jb, (R)-1, false, gs);
      __syncthreads();
    }
  }
  for (int i = tid; i < m; i += NT) t.piv[i] = perm[i];
}

// L^{-1} P (even CTA of the task's pair) or U^{-1} (odd CTA) from the packed
// LU of k_lu_blk; both run at once.
template <class E>
__global__ void __launch_bounds__(NT) k_lu_inv(const LuTask* __restrict__ tasks) {
  using R = typename RealOf<E>::T;
  extern __shared__ __align__(16) unsigned char smraw[];
  GemmSmem<R>& gs = *reinterpret_cast<GemmSmem<R>*>(smraw);
  E* Ls = reinterpret_cast<E*>(smraw + sizeof(GemmSmem<R>));  // NBMAX x NBMAX, ld NBMAX
  E* Ds = Ls + NBMAX * NBMAX;                                  // NBMAX x NBMAX, ld NBMAX
  const LuTask t = tasks[blockIdx.x >> 1];
  const bool lower = (blockIdx.x & 1) == 0;
  const int m = t.m, ld = t.lda;
  const int tid = threadIdx.x;
  const E* A = (const E*)t.A;
  if (lower) {
    // ------------------------------------------------ L^{-1} (in scratch) --
    // X[I, 0:I0] = -L[I,I]^{-1} L[I, 0:I0] X[0:I0, 0:I0]; X[I, I] = L[I,I]^{-1}
    E* X = (E*)t.scratch;
    for (int I0 = 0; I0 < m; I0 += NBMAX) {
      const int ib = min(NBMAX, m - I0);
      if (I0 > 0) cta_gemm<E, R>(X + I0, m, A + I0, ld, X, m, ib, I0, I0, (R)-1, true, gs);
      for (int idx = tid; idx < ib * ib; idx += NT) {
        const int r = idx % ib, c = idx / ib;
        Ls[r + c * NBMAX] = A[(size_t)(I0 + r) + (size_t)(I0 + c) * ld];
      }
      __syncthreads();
      diag_inverse<E, R>(Ls, ib, Ds, false);
      __syncthreads();
      if (I0 > 0) cta_gemm<E, R>(X + I0, m, Ds, NBMAX, X + I0, m, ib, I0, ib, (R)1, true, gs);
      for (int idx = tid; idx < ib * (m - I0); idx += NT) {
        const int r = idx % ib, c = I0 + idx / ib;
        E v;
        if (c < I0 + ib) {
          v = Ds[r + (c - I0) * NBMAX];
        } else {
          v.re = 0;
          v.im = 0;
        }
        X[(size_t)(I0 + r) + (size_t)c * m] = v;
      }
      __syncthreads();
    }
    // L^{-1} P: column r of L^{-1} is column piv[r] of the result
    E* Lp = (E*)t.Linv;
    for (int idx = tid; idx < m * m; idx += NT) {
      const int i = idx % m, r = idx / m;
      Lp[(size_t)i + (size_t)t.piv[r] * m] = X[idx];
    }
    __syncthreads();
    return;
  }
  // ------------------------------------------------ U^{-1} (odd CTA) ------
  // Y[I, J0:m] = -U[I,I]^{-1} U[I, J0:m] Y[J0:m, J0:m]; Y[I, I] = U[I,I]^{-1}
  E* Y = (E*)t.Uinv;
  const int nblk = (m + NBMAX - 1) / NBMAX;
  for (int bI = nblk - 1; bI >= 0; --bI) {
    const int I0 = bI * NBMAX, ib = min(NBMAX, m - I0), J0 = I0 + ib;
    if (J0 < m)
      cta_gemm<E, R>(Y + (size_t)I0 + (size_t)J0 * m, m, A + (size_t)I0 + (size_t)J0 * ld, ld,
                     Y + (size_t)J0 + (size_t)J0 * m, m, ib, m - J0, m - J0, (R)-1, true, gs);
    for (int idx = tid; idx < ib * ib; idx += NT) {
      const int r = idx % ib, c = idx / ib;
      Ls[r + c * NBMAX] = A[(size_t)(I0 + r) + (size_t)(I0 + c) * ld];
    }
    __syncthreads();
    diag_inverse<E, R>(Ls, ib, Ds, true);
    __syncthreads();
    if (J0 < m)
      cta_gemm<E, R>(Y + (size_t)I0 + (size_t)J0 * m, m, Ds, NBMAX, Y + (size_t)I0 + (size_t)J0 * m, m, ib, m - J0,
                     ib, (R)1, true, gs);
    for (int idx = tid; idx < ib * J0; idx += NT) {
      const int r = idx % ib, c = idx / ib;
      E v;
      if (c >= I0) {
        v = Ds[r + (c - I0) * NBMAX];
      } else {
        v.re = 0;
        v.im = 0;
      }
      Y[(size_t)(I0 + r) + (size_t)c * m] = v;
    }
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
  return sizeof(GemmSmem<R>) + 2 * (size_t)NBMAX * NBMAX * sizeof(E) + 16;
}

template <class E>
cudaError_t launch_lu(const LuTask* d, int n, int maxm, int* st, cudaStream_t s) {
  // panel width: as wide as the shared-memory budget allows (at most 32)
  constexpr size_t kPanelBytes = 104 * 1024;
  int nb = (int)std::min<size_t>(NBMAX, kPanelBytes / ((size_t)std::max(maxm, 1) * sizeof(E)));
  if (nb < 1) return cudaErrorInvalidValue;
  const size_t sm = lu_smem<E>(maxm, nb);
  if (sm > 227 * 1024) return cudaErrorInvalidValue;
  cudaFuncSetAttribute(k_lu_blk<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_lu_blk<E><<<n, NT, sm, s>>>(d, nb, maxm, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smi = lu_inv_smem<E>();
  cudaFuncSetAttribute(k_lu_inv<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smi);
  k_lu_inv<E><<<2 * n, NT, smi, s>>>(d);
  return cudaGetLastError();
}

}  // namespace

cudaError_t lu_blocked(const LuTask* d, int n, int maxm, int prec, int* st, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (maxm > 4096) return cudaErrorInvalidValue;
  return prec == P64 ? launch_lu<cd>(d, n, maxm, st, s) : launch_lu<cf>(d, n, maxm, st, s);
}

}  // namespace h2k
