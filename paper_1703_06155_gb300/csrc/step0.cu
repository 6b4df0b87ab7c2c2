// Step 0 (eqs. 16-17 / 25-26) in FP64: the dominant subspace of the fill-in
// Gram G' (p x p, Hermitian positive semidefinite, in complement coordinates).
//
// The truncation keeps the eigenpairs of G' above thr = eps^2 nu^2.  Instead of
// a full p x p eigen-decomposition this kernel
//   1. runs a pivoted Cholesky of G' until the trace of the remaining Schur
//      complement E = G' - L L^H is <= thr / 10; since E is positive
//      semidefinite, ||E|| <= trace(E), so the Ritz values of G' on span(L)
//      are within thr / 10 of its eigenvalues;
//   2. Householder-QR-factorizes L (p x r') and returns the compact WY form
//      Q = I - Y T Y^H of the reflectors and Qx = Q(:, 0:r'), an orthonormal
//      basis of span(L).
// The caller then forms the Ritz matrix Qx^H G' Qx (r' x r'), diagonalizes it
// (Jacobi), keeps the Ritz pairs above thr, and applies Q to the complement
// basis with GEMMs.  Reductions use warp shuffles; one CTA per cluster.
#include "h2_kernels.h"

namespace h2k {
namespace {

constexpr int NT = 256;

__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double bsum(double v, double* red) {
  v = wsum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0;
  if (threadIdx.x < 32) {
    t = (l < NT / 32) ? red[l] : 0.0;
    t = wsum(t);
    if (l == 0) red[0] = t;
  }
  __syncthreads();
  t = red[0];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(NT) k_pchol_wy(const PcholTask* __restrict__ tasks) {
  __shared__ double red[32];
  __shared__ double bv[NT];
  __shared__ int bi[NT];
  __shared__ double tau_r[1024], tau_i[1024], tmp_r[1024], tmp_i[1024];
  extern __shared__ unsigned char sm_raw[];
  double* d = reinterpret_cast<double*>(sm_raw);  // p diagonal residuals
  int* piv = reinterpret_cast<int*>(d + tasks[blockIdx.x].p + 1);
  const PcholTask t = tasks[blockIdx.x];
  const int p = t.p;
  cd* G = t.G;
  cd* L = t.L;  // p x p scratch (ld p); becomes Y
  // nu^2 = snorm2 + trace(M)
  double tr = 0;
  if (t.M)
    for (int i = threadIdx.x; i < t.n; i += NT) tr += t.M[i + (size_t)i * t.n].re;
  tr = bsum(tr, red);
  const double thr = t.eps2 * (t.snorm2 + tr);
  const double tau = thr / 10.0;  // bound on the trace of the remainder
  for (int i = threadIdx.x; i < p; i += NT) {
    d[i] = G[i + (size_t)i * p].re;
    piv[i] = i;
  }
  for (int idx = threadIdx.x; idx < p * p; idx += NT) {
    cd z;
    z.re = 0;
    z.im = 0;
    L[idx] = z;
  }
  __syncthreads();
  int r = 0;
  const int rmax = p < 1024 ? p : 1024;
  for (int j = 0; j < rmax; ++j) {
    // pivot: largest remaining diagonal (ties -> lowest position)
    double best = -1;
    int bq = p;
    double trs = 0;
    for (int q = j + threadIdx.x; q < p; q += NT) {
      const double v = d[piv[q]];
      trs += v > 0 ? v : 0;
      if (v > best || (v == best && q < bq)) { best = v; bq = q; }
    }
    trs = bsum(trs, red);
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = bq;
    __syncthreads();
    for (int s = NT / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        const double o = bv[threadIdx.x + s];
        const int oi = bi[threadIdx.x + s];
        if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
          bv[threadIdx.x] = o;
          bi[threadIdx.x] = oi;
        }
      }
      __syncthreads();
    }
    const double dv = bv[0];
    const int qb = bi[0];
    __syncthreads();
    if (!(trs > tau) || !(dv > 0.0)) break;
    if (threadIdx.x == 0) {
      const int x = piv[j];
      piv[j] = piv[qb];
      piv[qb] = x;
    }
    __syncthreads();
    const int pc = piv[j];
    const double sd = sqrt(dv);
    // column j of L for the rows not yet pivoted (original row indexing)
    for (int q = j + threadIdx.x; q < p; q += NT) {
      const int i = piv[q];
      double vr = G[i + (size_t)pc * p].re, vi = G[i + (size_t)pc * p].im;
      for (int k = 0; k < j; ++k) {
        const cd a = L[i + (size_t)k * p], b = L[pc + (size_t)k * p];  // a * conj(b)
        vr -= a.re * b.re + a.im * b.im;
        vi -= a.im * b.re - a.re * b.im;
      }
      cd z;
      z.re = vr / sd;
      z.im = vi / sd;
      L[i + (size_t)j * p] = z;
    }
    __syncthreads();
    for (int q = j + 1 + threadIdx.x; q < p; q += NT) {
      const int i = piv[q];
      const cd z = L[i + (size_t)j * p];
      d[i] -= z.re * z.re + z.im * z.im;
    }
    __syncthreads();
    r = j + 1;
  }
  // Householder QR of L(:, 0:r) in place (zlarfg convention, v_0 = 1)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = NT / 32;
  for (int j = 0; j < r; ++j) {
    double s = 0;
    for (int i = j + 1 + threadIdx.x; i < p; i += NT) {
      const cd v = L[i + (size_t)j * p];
      s += v.re * v.re + v.im * v.im;
    }
    s = bsum(s, red);
    const cd al = L[j + (size_t)j * p];
    double tr_ = 0, ti_ = 0;
    if (!(s == 0.0 && al.im == 0.0)) {
      const double nrm = sqrt(al.re * al.re + al.im * al.im + s);
      const double beta = al.re >= 0 ? -nrm : nrm;
      tr_ = (beta - al.re) / beta;
      ti_ = -al.im / beta;
      const double dr = al.re - beta, di = al.im, dd = dr * dr + di * di;
      const double scr = dr / dd, sci = -di / dd;
      for (int i = j + 1 + threadIdx.x; i < p; i += NT) {
        cd v = L[i + (size_t)j * p];
        const double vr = v.re * scr - v.im * sci, vi = v.re * sci + v.im * scr;
        v.re = vr;
        v.im = vi;
        L[i + (size_t)j * p] = v;
      }
    }
    if (threadIdx.x == 0) { tau_r[j] = tr_; tau_i[j] = ti_; }
    __syncthreads();
    if (!(tr_ == 0.0 && ti_ == 0.0))
      for (int c = j + 1 + warp; c < r; c += nw) {
        double dr = 0, di = 0;
        for (int i = j + lane; i < p; i += 32) {
          const cd w = L[i + (size_t)c * p];
          cd v;
          if (i == j) { v.re = 1; v.im = 0; } else v = L[i + (size_t)j * p];
          dr += v.re * w.re + v.im * w.im;
          di += v.re * w.im - v.im * w.re;
        }
        dr = wsum(dr);
        di = wsum(di);
        const double fr = tr_ * dr + ti_ * di, fi = tr_ * di - ti_ * dr;  // conj(tau) d
        for (int i = j + lane; i < p; i += 32) {
          cd v;
          if (i == j) { v.re = 1; v.im = 0; } else v = L[i + (size_t)j * p];
          cd w = L[i + (size_t)c * p];
          w.re -= v.re * fr - v.im * fi;
          w.im -= v.re * fi + v.im * fr;
          L[i + (size_t)c * p] = w;
        }
      }
    __syncthreads();
  }
  // Y: unit lower trapezoidal reflectors (upper part zeroed, v_0 = 1)
  for (int idx = threadIdx.x; idx < p * r; idx += NT) {
    const int i = idx % p, j = idx / p;
    if (i < j) { L[idx].re = 0; L[idx].im = 0; }
    else if (i == j) { L[idx].re = 1; L[idx].im = 0; }
  }
  __syncthreads();
  // compact WY: T upper triangular, T_jj = tau_j,
  // T(0:j, j) = -tau_j T(0:j, 0:j) (Y(:, 0:j)^H Y(:, j))
  cd* T = t.T;  // r x r (ld r)
  for (int idx = threadIdx.x; idx < r * r; idx += NT) {
    cd z;
    z.re = 0;
    z.im = 0;
    T[idx] = z;
  }
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    // w = Y(:, 0:j)^H Y(:, j)   (stored temporarily in T(0:j, j))
    for (int k = warp; k < j; k += nw) {
      double sr = 0, si = 0;
      for (int i = lane; i < p; i += 32) {
        const cd a = L[i + (size_t)k * p], b = L[i + (size_t)j * p];
        sr += a.re * b.re + a.im * b.im;
        si += a.re * b.im - a.im * b.re;
      }
      sr = wsum(sr);
      si = wsum(si);
      if (lane == 0) { T[k + (size_t)j * r].re = sr; T[k + (size_t)j * r].im = si; }
    }
    __syncthreads();
    // T(0:j, j) = -tau_j T(0:j,0:j) w   (upper triangular matvec)
    for (int i = threadIdx.x; i < j; i += NT) {
      double sr = 0, si = 0;
      for (int k = i; k < j; ++k) {
        const cd a = T[i + (size_t)k * r], w = T[k + (size_t)j * r];
        sr += a.re * w.re - a.im * w.im;
        si += a.re * w.im + a.im * w.re;
      }
      tmp_r[i] = sr;
      tmp_i[i] = si;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < j; i += NT) {
      const double sr = tmp_r[i], si = tmp_i[i];
      const double tr2 = tau_r[j], ti2 = tau_i[j];
      T[i + (size_t)j * r].re = -(tr2 * sr - ti2 * si);
      T[i + (size_t)j * r].im = -(tr2 * si + ti2 * sr);
    }
    if (threadIdx.x == 0) { T[j + (size_t)j * r].re = tau_r[j]; T[j + (size_t)j * r].im = tau_i[j]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) *t.rout = r;
}

}  // namespace

cudaError_t pchol_wy(const PcholTask* d, int n, int maxp, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const size_t sm = (size_t)(maxp + 2) * sizeof(double) + (size_t)(maxp + 2) * sizeof(int);
  k_pchol_wy<<<n, NT, sm, s>>>(d);
  return cudaGetLastError();
}

}  // namespace h2k
