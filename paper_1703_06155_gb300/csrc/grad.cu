// Per-cell derivative of a real objective through the solution map
// x = A(chi)^{-1} b, A = I + s K D_chi.
//
// With g the objective's gradient with respect to x (conjugate-Wirtinger
// convention: dL = Re sum conj(g) dx) and mu = A^{-H} g the adjoint solution,
// dA / dchi_i = s K e_i e_i^T gives
//   dL / dchi_i = -Re( conj((s K^H mu)_i) x_i ),
// and A^H mu = g turns (s K^H mu)_i into (g_i - mu_i) / chi_i, so that
//   dL / dchi_i = Re( x_i conj(mu_i - g_i) ) / chi_i
// summed over the right-hand sides.  One pass over x, mu, g: HBM-bound.
#include <algorithm>

#include "h2_kernels.h"

namespace h2k {
namespace {

constexpr int NT = 256;

__global__ void __launch_bounds__(NT) k_grad_chi(const cd* __restrict__ x, const cd* __restrict__ mu,
                                                const cd* __restrict__ g, const double* __restrict__ sqchi,
                                                int64_t N, int nrhs, double alpha, double* __restrict__ grad,
                                                int accumulate) {
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < N; i += (int64_t)gridDim.x * NT) {
    double acc = 0;
    for (int c = 0; c < nrhs; ++c) {
      const int64_t o = i + (int64_t)c * N;
      const cd xv = x[o], mv = mu[o];
      double dr = mv.re, di = mv.im;
      if (g) {
        const cd gv = g[o];
        dr -= gv.re;
        di -= gv.im;
      }
      // Re(x conj(d)) = x.re d.re + x.im d.im
      acc = fma(xv.re, dr, fma(xv.im, di, acc));
    }
    const double sq = sqchi[i];
    const double v = alpha * acc / (sq * sq);
    grad[i] = accumulate ? grad[i] + v : v;
  }
}

}  // namespace

cudaError_t grad_chi(const cd* x, const cd* mu, const cd* g, const double* sqchi, int64_t N, int nrhs, double alpha,
                     double* grad, int accumulate, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  const int64_t want = (N + NT - 1) / NT;
  const int blocks = (int)std::min<int64_t>(want, 152 * 16);
  k_grad_chi<<<blocks, NT, 0, s>>>(x, mu, g, sqchi, N, nrhs, alpha, grad, accumulate);
  return cudaGetLastError();
}

}  // namespace h2k
