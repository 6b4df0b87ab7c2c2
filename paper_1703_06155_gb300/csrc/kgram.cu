// Far-field sample Gram of the H^2 construction (h2_build):
//   G_t = Z(rows_t, F*(t)) Z(rows_t, F*(t))^H
// with the kernel entries Z(p, q) = s sqrt(chi_p chi_q) k^2 h^3 e^{-jkr}/(4 pi r)
// evaluated on the fly while the Gram is accumulated, so the (rows x far)
// sample is never stored.  One CTA computes one 64 x 64 tile of the upper
// triangle of one G_t; the far field of a cluster is a list of contiguous
// tree-order ranges (its admissible partners and those of its ancestors).
#include "h2_kernels.h"

namespace h2k {
namespace {

constexpr int BM = 64, BK = 16, NT = 256;

__device__ __forceinline__ void zval(const double* __restrict__ pts, const double* __restrict__ sq, int64_t p,
                                     int64_t q, double k, double w, double& re, double& im) {
  const double dx = pts[3 * p] - pts[3 * q], dy = pts[3 * p + 1] - pts[3 * q + 1], dz = pts[3 * p + 2] - pts[3 * q + 2];
  const double r = sqrt(dx * dx + dy * dy + dz * dz);
  double s, c;
  sincos(k * r, &s, &c);
  const double a = w * sq[p] * sq[q] / r;
  re = a * c;
  im = -a * s;
}

__global__ void __launch_bounds__(NT) k_kgram(const KGramTask* __restrict__ tasks, const KGramTile* __restrict__ tiles,
                                             const double* __restrict__ pts, const double* __restrict__ sq, double k,
                                             double w) {
  __shared__ double Ar[BK][BM], Ai[BK][BM], Br[BK][BM], Bi[BK][BM];
  const KGramTile tl = tiles[blockIdx.x];
  const KGramTask t = tasks[tl.task];
  const int m0 = tl.tm * BM, n0 = tl.tn * BM;
  const bool diag = tl.tm == tl.tn;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double cr[4][4], ci[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) cr[i][j] = ci[i][j] = 0;
  for (int g = 0; g < t.nranges; ++g) {
    const int64_t c0 = t.ranges[2 * g], cn = t.ranges[2 * g + 1];
    for (int64_t k0 = 0; k0 < cn; k0 += BK) {
#pragma unroll
      for (int r = 0; r < (BM * BK) / NT; ++r) {
        const int l = tid + r * NT;
        const int i = l % BM, kk = l / BM;
        double re = 0, im = 0;
        if (m0 + i < t.nr && k0 + kk < cn) zval(pts, sq, t.rows[m0 + i], c0 + k0 + kk, k, w, re, im);
        Ar[kk][i] = re;
        Ai[kk][i] = im;
        if (!diag) {
          double re2 = 0, im2 = 0;
          if (n0 + i < t.nr && k0 + kk < cn) zval(pts, sq, t.rows[n0 + i], c0 + k0 + kk, k, w, re2, im2);
          Br[kk][i] = re2;
          Bi[kk][i] = im2;
        }
      }
      __syncthreads();
      double (*Xr)[BM] = diag ? Ar : Br;
      double (*Xi)[BM] = diag ? Ai : Bi;
#pragma unroll 4
      for (int kk = 0; kk < BK; ++kk) {
        double ar[4], ai[4], br[4], bi[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) { ar[i] = Ar[kk][ty + 16 * i]; ai[i] = Ai[kk][ty + 16 * i]; }
#pragma unroll
        for (int j = 0; j < 4; ++j) { br[j] = Xr[kk][tx + 16 * j]; bi[j] = Xi[kk][tx + 16 * j]; }
        // a * conj(b)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            cr[i][j] = fma(ar[i], br[j], fma(ai[i], bi[j], cr[i][j]));
            ci[i][j] = fma(ai[i], br[j], fma(-ar[i], bi[j], ci[i][j]));
          }
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= t.nr) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= t.nr) continue;
      cd v;
      v.re = cr[i][j];
      v.im = ci[i][j];
      t.G[(size_t)m + (size_t)n * t.nr] = v;
    }
  }
}

}  // namespace

cudaError_t kernel_gram(const KGramTask* d_tasks, const KGramTile* d_tiles, int ntiles, const double* d_pts,
                        const double* d_sq, double k, double w, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  k_kgram<<<ntiles, NT, 0, s>>>(d_tasks, d_tiles, d_pts, d_sq, k, w);
  return cudaGetLastError();
}

}  // namespace h2k
