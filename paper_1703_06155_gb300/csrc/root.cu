// Rank selection of Step 0 and the panel kernels of the blocked LU of the
// final block (Algorithm 1, last line).
#include "h2_kernels.h"

namespace h2k {
namespace {

constexpr int NT = 256;
constexpr size_t kPanelSmem = 200 * 1024;  // largest panel copied to shared memory

template <class E> struct RealOf;
template <> struct RealOf<cd> { using T = double; };
template <> struct RealOf<cf> { using T = float; };

// Keep lambda_j > eps^2 nu^2 with nu^2 = snorm2 + trace(M): snorm2 is the sum
// of ||S||_F^2 over the admissible blocks of the cluster's row and column,
// trace(M) the squared Frobenius norm of its fill-ins (eqs. 17 / 26).
__global__ void __launch_bounds__(NT) k_select(const SelTask* __restrict__ tasks) {
  __shared__ int cnt[NT];
  const SelTask t = tasks[blockIdx.x];
  const double thr = t.eps2 * (t.snorm2 + *t.trM);
  int c = 0;
  for (int j = threadIdx.x; j < t.p; j += NT) c += t.lam[j] > thr;
  cnt[threadIdx.x] = c;
  __syncthreads();
  for (int s = NT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) cnt[threadIdx.x] += cnt[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *t.out = cnt[0];
}

// largest |z|^2 of the CTA, ties to the lowest row; result to every thread
template <class R>
__device__ void panel_argmax(R& v, int& i, R* wv, int* wi) {
  for (int o = 16; o > 0; o >>= 1) {
    const R ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
  }
  if ((threadIdx.x & 31) == 0) { wv[threadIdx.x >> 5] = v; wi[threadIdx.x >> 5] = i; }
  __syncthreads();
  v = wv[0];
  i = wi[0];
  for (int w = 1; w < NT / 32; ++w)
    if (wv[w] > v || (wv[w] == v && wi[w] < i)) { v = wv[w]; i = wi[w]; }
  __syncthreads();
}

// One tall panel (nrows x kb) per CTA: pivot search, row swap, scaling and
// rank-1 update column by column, then the inverses of its unit lower and
// upper kb x kb triangles.  The panel is copied to shared memory when the
// launch provides room for it (dynamic shared memory >= nrows x kb entries),
// else it is worked on in place.
template <class E>
__global__ void __launch_bounds__(NT) k_lu_panel(const PanelTask* __restrict__ tasks, int* status, int in_smem) {
  using R = typename RealOf<E>::T;
  __shared__ R wv[NT / 32];
  __shared__ int wi[NT / 32];
  extern __shared__ __align__(16) unsigned char psm[];
  const PanelTask t = tasks[blockIdx.x];
  E* G = (E*)t.A + (size_t)t.row0 + (size_t)t.col0 * t.lda;
  const int kb = t.kb, nr = t.nrows;
  E* P = in_smem ? reinterpret_cast<E*>(psm) : G;
  const int ldp = in_smem ? nr : t.lda;
  if (in_smem) {
    for (int idx = threadIdx.x; idx < nr * kb; idx += NT) {
      const int r = idx % nr, c = idx / nr;
      P[idx] = G[(size_t)r + (size_t)c * t.lda];
    }
    __syncthreads();
  }
  auto at = [&](int r, int c) -> E& { return P[(size_t)r + (size_t)c * ldp]; };
  for (int j = 0; j < kb; ++j) {
    R best = -1;
    int bi = nr;
    for (int i = j + threadIdx.x; i < nr; i += NT) {
      const E v = at(i, j);
      const R a = (R)v.re * (R)v.re + (R)v.im * (R)v.im;
      if (a > best || (a == best && i < bi)) { best = a; bi = i; }
    }
    panel_argmax<R>(best, bi, wv, wi);
    const int pr = bi;
    const R pv = best;
    if (!(pv > (R)0)) {
      if (threadIdx.x == 0 && status) atomicMax(status, 1);
      return;
    }
    if (threadIdx.x == 0) t.ipiv[j] = t.row0 + pr;
    if (pr != j)
      for (int c = threadIdx.x; c < kb; c += NT) {
        const E a = at(j, c);
        at(j, c) = at(pr, c);
        at(pr, c) = a;
      }
    __syncthreads();
    const E d = at(j, j);
    const R dd = (R)d.re * (R)d.re + (R)d.im * (R)d.im;
    const R ir = (R)d.re / dd, ii = -(R)d.im / dd;
    for (int i = j + 1 + threadIdx.x; i < nr; i += NT) {
      E v = at(i, j);
      const R vr = (R)v.re * ir - (R)v.im * ii, vi = (R)v.re * ii + (R)v.im * ir;
      v.re = vr;
      v.im = vi;
      at(i, j) = v;
    }
    __syncthreads();
    const int rem_r = nr - j - 1, rem_c = kb - j - 1;
    for (int idx = threadIdx.x; idx < rem_r * rem_c; idx += NT) {
      const int i = j + 1 + idx % rem_r, c = j + 1 + idx / rem_r;
      const E l = at(i, j), u = at(j, c);
      E v = at(i, c);
      v.re = (R)v.re - ((R)l.re * (R)u.re - (R)l.im * (R)u.im);
      v.im = (R)v.im - ((R)l.re * (R)u.im + (R)l.im * (R)u.re);
      at(i, c) = v;
    }
    __syncthreads();
  }
  if (in_smem)
    for (int idx = threadIdx.x; idx < nr * kb; idx += NT) {
      const int r = idx % nr, c = idx / nr;
      G[(size_t)r + (size_t)c * t.lda] = P[idx];
    }
  // (unit lower L11)^{-1}
  E* X = (E*)t.Linv;
  for (int idx = threadIdx.x; idx < kb * kb; idx += NT) {
    E v;
    v.re = (idx % kb == idx / kb) ? 1 : 0;
    v.im = 0;
    X[idx] = v;
  }
  __syncthreads();
  for (int tt = 0; tt < kb - 1; ++tt) {
    const int rem = kb - tt - 1;
    for (int idx = threadIdx.x; idx < rem * kb; idx += NT) {
      const int i = tt + 1 + idx % rem, c = idx / rem;
      const E l = at(i, tt), x = X[tt + (size_t)c * kb];
      E v = X[i + (size_t)c * kb];
      v.re = (R)v.re - ((R)l.re * (R)x.re - (R)l.im * (R)x.im);
      v.im = (R)v.im - ((R)l.re * (R)x.im + (R)l.im * (R)x.re);
      X[i + (size_t)c * kb] = v;
    }
    __syncthreads();
  }
  // U11^{-1}
  E* Y = (E*)t.Uinv;
  for (int idx = threadIdx.x; idx < kb * kb; idx += NT) {
    E v;
    v.re = (idx % kb == idx / kb) ? 1 : 0;
    v.im = 0;
    Y[idx] = v;
  }
  __syncthreads();
  for (int tt = kb - 1; tt >= 0; --tt) {
    const E d = at(tt, tt);
    const R dd = (R)d.re * (R)d.re + (R)d.im * (R)d.im;
    const R ir = (R)d.re / dd, ii = -(R)d.im / dd;
    for (int c = threadIdx.x; c < kb; c += NT) {
      E v = Y[tt + (size_t)c * kb];
      const R vr = (R)v.re * ir - (R)v.im * ii, vi = (R)v.re * ii + (R)v.im * ir;
      v.re = vr;
      v.im = vi;
      Y[tt + (size_t)c * kb] = v;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < tt * kb; idx += NT) {
      const int i = idx % tt, c = idx / tt;
      const E u = at(i, tt), y = Y[tt + (size_t)c * kb];
      E v = Y[i + (size_t)c * kb];
      v.re = (R)v.re - ((R)u.re * (R)y.re - (R)u.im * (R)y.im);
      v.im = (R)v.im - ((R)u.re * (R)y.im + (R)u.im * (R)y.re);
      Y[i + (size_t)c * kb] = v;
    }
    __syncthreads();
  }
}

template <class E>
__global__ void k_swap_rows(E* A, int lda, const int* ipiv, int row0, int kb, int c0, int c1, int reverse) {
  for (int c = c0 + blockIdx.x * blockDim.x + threadIdx.x; c < c1; c += gridDim.x * blockDim.x) {
    for (int q = 0; q < kb; ++q) {
      const int j = reverse ? kb - 1 - q : q;
      const int r1 = row0 + j, r2 = ipiv[j];
      if (r1 != r2) {
        const E a = A[(size_t)r1 + (size_t)c * lda];
        A[(size_t)r1 + (size_t)c * lda] = A[(size_t)r2 + (size_t)c * lda];
        A[(size_t)r2 + (size_t)c * lda] = a;
      }
    }
  }
}

template <class E>
__global__ void k_swap_rows_batch(const SwapTask* __restrict__ tasks) {
  const SwapTask t = tasks[blockIdx.y];
  E* A = (E*)t.A;
  for (int c = t.c0 + blockIdx.x * blockDim.x + threadIdx.x; c < t.c1; c += gridDim.x * blockDim.x) {
    for (int q = 0; q < t.kb; ++q) {
      const int j = t.reverse ? t.kb - 1 - q : q;
      const int r1 = t.row0 + j, r2 = t.ipiv[j];
      if (r1 != r2) {
        const E a = A[(size_t)r1 + (size_t)c * t.lda];
        A[(size_t)r1 + (size_t)c * t.lda] = A[(size_t)r2 + (size_t)c * t.lda];
        A[(size_t)r2 + (size_t)c * t.lda] = a;
      }
    }
  }
}

}  // namespace

cudaError_t swap_rows_batch(const SwapTask* d, int n, int prec, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const dim3 g(8, n);
  if (prec == P64) k_swap_rows_batch<cd><<<g, 128, 0, s>>>(d);
  else k_swap_rows_batch<cf><<<g, 128, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t select_rank(const SelTask* d, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_select<<<n, NT, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t lu_panel(const PanelTask* d, int n, int prec, int maxrows, int maxkb, int* st, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const size_t es = prec == P64 ? sizeof(cd) : sizeof(cf);
  const size_t need = (size_t)maxrows * maxkb * es;
  const int in_smem = need <= kPanelSmem ? 1 : 0;
  const size_t dyn = in_smem ? need : 0;
  cudaError_t e = cudaSuccess;
  if (prec == P64) {
    if (dyn) e = cudaFuncSetAttribute(k_lu_panel<cd>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    k_lu_panel<cd><<<n, NT, dyn, s>>>(d, st, in_smem);
  } else {
    if (dyn) e = cudaFuncSetAttribute(k_lu_panel<cf>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    k_lu_panel<cf><<<n, NT, dyn, s>>>(d, st, in_smem);
  }
  return cudaGetLastError();
}

cudaError_t swap_rows(void* A, int lda, const int* ipiv, int row0, int kb, int c0, int c1, int prec, int reverse,
                      cudaStream_t s) {
  if (c1 <= c0) return cudaSuccess;
  const int n = c1 - c0;
  const int g = (n + 127) / 128;
  if (prec == P64) k_swap_rows<cd><<<g, 128, 0, s>>>((cd*)A, lda, ipiv, row0, kb, c0, c1, reverse);
  else k_swap_rows<cf><<<g, 128, 0, s>>>((cf*)A, lda, ipiv, row0, kb, c0, c1, reverse);
  return cudaGetLastError();
}

}  // namespace h2k
