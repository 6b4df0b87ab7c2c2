// In-place application of a small square matrix to a block panel.
//
//  left : X[lo:p, cols] <- op(A)[lo:p, 0:p] * X[0:p, cols]    (column tiles)
//  right: X[rows, lo:p] <- X[rows, 0:p] * op(A)[0:p, lo:p]    (row tiles)
//
// A CTA first copies its whole input strip of X (p x tw or th x p) into
// shared memory, so writing the result back over X is safe.  These kernels
// carry Step 2 (Q~^H Z, Z conj(Q~), eq. 5), the partial-LU panels
// (L^{-1} P Z_i'c and Z_ci' U^{-1}, Algorithm 4) and the per-cluster steps of
// the forward / backward substitution (Algorithms 5, 6).
#include "h2_kernels.h"

namespace h2k {
namespace {

constexpr int NT = 256;
constexpr int RPT = 4;  // outputs per thread along the long dimension

template <class E> struct RealOf;
template <> struct RealOf<cd> { using T = double; };
template <> struct RealOf<cf> { using T = float; };

template <class E, class R>
__device__ __forceinline__ void op_elem(const E* A, int lda, int op, int r, int c, R& re, R& im) {
  const E v = (op == OP_N || op == OP_C) ? A[(size_t)r + (size_t)c * lda] : A[(size_t)c + (size_t)r * lda];
  re = (R)v.re;
  im = (op == OP_C || op == OP_H) ? -(R)v.im : (R)v.im;
}

template <class E>
__global__ void __launch_bounds__(NT) k_apply_left(const ApplyTask* __restrict__ tasks,
                                                  const ApplyTile* __restrict__ tiles, int tw) {
  using R = typename RealOf<E>::T;
  extern __shared__ unsigned char smem_raw[];
  E* Xs = reinterpret_cast<E*>(smem_raw);  // p x tw, column c at Xs[k*tw + c]
  const ApplyTile tl = tiles[blockIdx.x];
  const ApplyTask tk = tasks[tl.task];
  const int p = tk.p, c0 = tl.t0;
  const int wc = min(tw, tk.w - c0);
  E* X = (E*)tk.X;
  const E* A = (const E*)tk.A;
  for (int idx = threadIdx.x; idx < p * tw; idx += NT) {
    const int c = idx / p, k = idx % p;
    E v;
    if (c < wc) v = X[(size_t)k + (size_t)(c0 + c) * tk.ldx];
    else { v.re = 0; v.im = 0; }
    Xs[k * tw + c] = v;
  }
  __syncthreads();
  const int c = threadIdx.x % tw;
  const int rg = threadIdx.x / tw, ng = NT / tw;
  for (int rb = tk.lo + rg; rb < p; rb += ng * RPT) {
    R accr[RPT], acci[RPT];
#pragma unroll
    for (int j = 0; j < RPT; ++j) accr[j] = acci[j] = 0;
    for (int k = 0; k < p; ++k) {
      const E xv = Xs[k * tw + c];
      const R xr = (R)xv.re, xi = (R)xv.im;
#pragma unroll
      for (int j = 0; j < RPT; ++j) {
        const int r = rb + j * ng;
        if (r < p) {
          R ar, ai;
          op_elem<E, R>(A, tk.lda, tk.opA, r, k, ar, ai);
          accr[j] = fma(ar, xr, fma(-ai, xi, accr[j]));
          acci[j] = fma(ar, xi, fma(ai, xr, acci[j]));
        }
      }
    }
    if (c < wc) {
#pragma unroll
      for (int j = 0; j < RPT; ++j) {
        const int r = rb + j * ng;
        if (r < p) {
          E v;
          v.re = accr[j];
          v.im = acci[j];
          X[(size_t)r + (size_t)(c0 + c) * tk.ldx] = v;
        }
      }
    }
  }
}

template <class E>
__global__ void __launch_bounds__(NT) k_apply_right(const ApplyTask* __restrict__ tasks,
                                                   const ApplyTile* __restrict__ tiles, int th) {
  using R = typename RealOf<E>::T;
  extern __shared__ unsigned char smem_raw[];
  E* Xs = reinterpret_cast<E*>(smem_raw);  // th x p, row r at Xs[r*(p) + k]
  const ApplyTile tl = tiles[blockIdx.x];
  const ApplyTask tk = tasks[tl.task];
  const int p = tk.p, r0 = tl.t0;
  const int hr = min(th, tk.w - r0);
  E* X = (E*)tk.X;
  const E* A = (const E*)tk.A;
  for (int idx = threadIdx.x; idx < p * th; idx += NT) {
    const int r = idx % th, k = idx / th;
    E v;
    if (r < hr) v = X[(size_t)(r0 + r) + (size_t)k * tk.ldx];
    else { v.re = 0; v.im = 0; }
    Xs[r * p + k] = v;
  }
  __syncthreads();
  const int r = threadIdx.x % th;
  const int cg = threadIdx.x / th, ng = NT / th;
  for (int cb = tk.lo + cg; cb < p; cb += ng * RPT) {
    R accr[RPT], acci[RPT];
#pragma unroll
    for (int j = 0; j < RPT; ++j) accr[j] = acci[j] = 0;
    for (int k = 0; k < p; ++k) {
      const E xv = Xs[r * p + k];
      const R xr = (R)xv.re, xi = (R)xv.im;
#pragma unroll
      for (int j = 0; j < RPT; ++j) {
        const int c = cb + j * ng;
        if (c < p) {
          R ar, ai;
          op_elem<E, R>(A, tk.lda, tk.opA, k, c, ar, ai);
          accr[j] = fma(xr, ar, fma(-xi, ai, accr[j]));
          acci[j] = fma(xr, ai, fma(xi, ar, acci[j]));
        }
      }
    }
    if (r < hr) {
#pragma unroll
      for (int j = 0; j < RPT; ++j) {
        const int c = cb + j * ng;
        if (c < p) {
          E v;
          v.re = accr[j];
          v.im = acci[j];
          X[(size_t)(r0 + r) + (size_t)c * tk.ldx] = v;
        }
      }
    }
  }
}

constexpr size_t kSmemBudget = 200 * 1024;

}  // namespace

int apply_tile_width(int prec, int maxp) {
  const size_t es = prec == P64 ? sizeof(cd) : sizeof(cf);
  int tw = 16;
  while (tw > 1 && (size_t)tw * maxp * es > kSmemBudget) tw >>= 1;
  return tw;
}

template <class E>
static cudaError_t launch_apply(bool left, const ApplyTask* t, const ApplyTile* tl, int n, int maxp, int tw,
                                cudaStream_t s) {
  const size_t sm = (size_t)tw * maxp * sizeof(E);
  if (sm > 227 * 1024) return cudaErrorInvalidValue;
  if (left) {
    cudaFuncSetAttribute(k_apply_left<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_apply_left<E><<<n, NT, sm, s>>>(t, tl, tw);
  } else {
    cudaFuncSetAttribute(k_apply_right<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_apply_right<E><<<n, NT, sm, s>>>(t, tl, tw);
  }
  return cudaGetLastError();
}

cudaError_t apply_left(const ApplyTask* t, const ApplyTile* tl, int n, int prec, int maxp, int tw, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  return prec == P64 ? launch_apply<cd>(true, t, tl, n, maxp, tw, s) : launch_apply<cf>(true, t, tl, n, maxp, tw, s);
}

cudaError_t apply_right(const ApplyTask* t, const ApplyTile* tl, int n, int prec, int maxp, int th, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  return prec == P64 ? launch_apply<cd>(false, t, tl, n, maxp, th, s) : launch_apply<cf>(false, t, tl, n, maxp, th, s);
}

}  // namespace h2k
