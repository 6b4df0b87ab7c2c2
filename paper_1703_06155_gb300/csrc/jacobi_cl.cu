// Hermitian Jacobi eigen-decomposition spread over a thread-block cluster.
//
// Same method as the one-CTA kernel (cyclic Jacobi, parallel round-robin
// ordering; a 2 x 2 block [[a, g e^{i phi}], [g e^{-i phi}, d]] is rotated by
// G = diag(1, e^{-i phi}) J with J the real Jacobi rotation of [[a, g],[g, d]]),
// but each eigenproblem runs on one cluster of CTAs so that its FP64 work is
// spread over several SMs.  Per round:
//   1. each CTA computes the rotations of the pairs it owns (pair i is owned by
//      CTA i mod C), publishes them in global scratch and rotates the columns
//      of A and U of those pairs (no other CTA touches them in this phase);
//   2. each CTA applies all row rotations to the columns it owns (col mod C).
// Phases are separated by cluster barriers with release / acquire semantics
// (hardware barrier.cluster; no software spin), which order the global-memory
// traffic of the cluster's threads.  A matrix whose sweeps do not converge
// within kMaxSweeps sets status bit 2 and returns its current state.
#include <cooperative_groups.h>

#include "h2_kernels.h"

namespace cg = cooperative_groups;

namespace h2k {
namespace {

constexpr int NT = 512;
constexpr int kMaxSweeps = 60;

// cluster-wide barrier: arrive with release, wait with acquire (cluster scope)
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(NT) k_jacobi_cl(const EigTask* __restrict__ tasks, double* __restrict__ scratch,
                                                 int64_t scratch_per_task, int* status) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int ti = blockIdx.x / C;
  const EigTask t = tasks[ti];
  const int p = t.p;
  if (p <= 1) {
    if (rank == 0) {
      for (int idx = threadIdx.x; idx < p * p; idx += NT) {
        t.U[idx].re = 1;
        t.U[idx].im = 0;
      }
      if (threadIdx.x == 0 && p == 1) t.lam[0] = t.A[0].re;
      if (threadIdx.x == 0 && t.sweeps) *t.sweeps = 0;
    }
    return;
  }
  const int pe = p + (p & 1);
  const int np = pe / 2;
  double* base = scratch + ti * scratch_per_task;
  double* rc = base;
  double* rs = rc + np;
  double* rer = rs + np;
  double* rei = rer + np;
  int* pa = (int*)(rei + np);
  int* pb = pa + np;
  int* flags = pb + np;           // per sweep: a rotation happened (zeroed by the host)
  int* open = flags + kMaxSweeps;  // per sweep: an entry above its threshold at the start
  cd* A = t.A;
  cd* U = t.U;
  __shared__ double red[32];
  // U = I (columns owned by this CTA)
  for (int idx = threadIdx.x; idx < p * p; idx += NT) {
    const int col = idx / p;
    if (col % C != rank) continue;
    U[idx].re = (idx % p == col) ? 1.0 : 0.0;
    U[idx].im = 0;
  }
  // ||A||_F^2 (every CTA computes it redundantly)
  double fro = 0;
  for (int idx = threadIdx.x; idx < p * p; idx += NT) fro += A[idx].re * A[idx].re + A[idx].im * A[idx].im;
  for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = fro;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  fro = red[0];
  // off-diagonal entries at the rounding level of the matrix are not rotated
  const double gmin = fmax(1e-300, 4e-16 * sqrt(fro));
  cluster_barrier();
  int sweep = 0;
  for (; sweep < kMaxSweeps; ++sweep) {
    if (fro == 0.0) break;
    // converged when no off-diagonal entry is above its rotation threshold:
    // such a sweep would rotate nothing, so one pass over the owned columns
    // replaces it
    {
      int any = 0;
      const int ncol = (p - rank + C - 1) / C;
      for (int idx = threadIdx.x; idx < ncol * p && !any; idx += NT) {
        const int col = rank + (idx / p) * C, row = idx % p;
        if (row >= col) continue;
        const cd v = A[row + (size_t)col * p];
        const double g = sqrt(v.re * v.re + v.im * v.im);
        if (g > gmin && g > 1e-17 * sqrt(fabs(A[row + (size_t)row * p].re * A[col + (size_t)col * p].re))) any = 1;
      }
      if (__syncthreads_or(any) && threadIdx.x == 0) open[sweep] = 1;
      cluster_barrier();
      if (!open[sweep]) break;
    }
    for (int r = 0; r < pe - 1; ++r) {
      // 1a. rotations of own pairs (pair i is owned by CTA i mod C)
      for (int i = rank + threadIdx.x * C; i < np; i += NT * C) {
        int a, b;
        if (i == 0) { a = pe - 1; b = r; } else { a = (r + i) % (pe - 1); b = (r - i + pe - 1) % (pe - 1); }
        if (a > b) { const int x = a; a = b; b = x; }
        double c = 1, s = 0, er = 1, ei = 0;
        if (b < p) {
          const double app = A[a + (size_t)a * p].re, aqq = A[b + (size_t)b * p].re;
          const cd apq = A[a + (size_t)b * p];
          const double g = sqrt(apq.re * apq.re + apq.im * apq.im);
          if (g > gmin && g > 1e-17 * sqrt(fabs(app * aqq))) {
            er = apq.re / g;
            ei = apq.im / g;
            const double zeta = (aqq - app) / (2.0 * g);
            const double tt = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            c = 1.0 / sqrt(1.0 + tt * tt);
            s = tt * c;
            flags[sweep] = 1;
          }
        }
        pa[i] = a;
        pb[i] = b;
        rc[i] = c;
        rs[i] = s;
        rer[i] = er;
        rei[i] = ei;
      }
      __syncthreads();
      // 1b. columns of A and U of own pairs (pair ii is owned by CTA ii mod C)
      for (int ii = rank; ii < np; ii += C) {
        const double s = rs[ii];
        if (s == 0.0) continue;
        const int a = pa[ii], b = pb[ii];
        const double c = rc[ii], er = rer[ii], ei = -rei[ii];
        for (int idx = threadIdx.x; idx < 2 * p; idx += NT) {
          cd* M = idx < p ? A : U;
          const int row = idx < p ? idx : idx - p;
          const cd xa = M[row + (size_t)a * p], xb = M[row + (size_t)b * p];
          const double ebr = er * xb.re - ei * xb.im, ebi = er * xb.im + ei * xb.re;
          cd na, nb;
          na.re = c * xa.re - s * ebr;
          na.im = c * xa.im - s * ebi;
          nb.re = s * xa.re + c * ebr;
          nb.im = s * xa.im + c * ebi;
          M[row + (size_t)a * p] = na;
          M[row + (size_t)b * p] = nb;
        }
      }
      cluster_barrier();
      // 2. rows of A, columns owned by this CTA, all pairs
      const int ncol = (p - rank + C - 1) / C;
      for (int idx = threadIdx.x; idx < np * ncol; idx += NT) {
        const int i = idx / ncol, col = rank + (idx % ncol) * C;
        const double s = rs[i];
        if (s == 0.0) continue;
        const int a = pa[i], b = pb[i];
        const double c = rc[i], er = rer[i], ei = rei[i];
        const cd ya = A[a + (size_t)col * p], yb = A[b + (size_t)col * p];
        const double ebr = er * yb.re - ei * yb.im, ebi = er * yb.im + ei * yb.re;
        cd na, nb;
        na.re = c * ya.re - s * ebr;
        na.im = c * ya.im - s * ebi;
        nb.re = s * ya.re + c * ebr;
        nb.im = s * ya.im + c * ebi;
        // the rotated pair's off-diagonal entries are zero by construction
        if (col == b) { na.re = 0; na.im = 0; nb.im = 0; }
        if (col == a) { nb.re = 0; nb.im = 0; na.im = 0; }
        A[a + (size_t)col * p] = na;
        A[b + (size_t)col * p] = nb;
      }
      cluster_barrier();
    }
    if (!flags[sweep]) break;
  }
  if (rank != 0) return;
  if (sweep == kMaxSweeps && threadIdx.x == 0 && status) atomicMax(status, 2);
  if (threadIdx.x == 0 && t.sweeps) *t.sweeps = sweep;
  // decreasing order of the eigenvalues (ties: lower index first)
  int* rks = pa;  // np >= p / 2 ... reuse pa and pb (2 np >= p ints)
  for (int i = threadIdx.x; i < p; i += NT) {
    const double li = A[i + (size_t)i * p].re;
    int rk = 0;
    for (int j = 0; j < p; ++j) {
      const double lj = A[j + (size_t)j * p].re;
      rk += (lj > li) || (lj == li && j < i);
    }
    rks[i] = rk;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < p; i += NT) t.lam[rks[i]] = A[i + (size_t)i * p].re;
  __syncthreads();
  for (int idx = threadIdx.x; idx < p * p; idx += NT) A[idx] = U[idx];
  __syncthreads();
  for (int idx = threadIdx.x; idx < p * p; idx += NT) {
    const int row = idx % p, col = idx / p;
    U[row + (size_t)rks[col] * p] = A[idx];
  }
}

}  // namespace

int64_t jacobi_cluster_scratch(int maxp) {
  const int np = (maxp + 1) / 2 + 1;
  return (int64_t)np * 4 + (np * 2 + 2 * kMaxSweeps + 8) / 2 + 8;  // doubles
}

cudaError_t jacobi_eig_cluster(const EigTask* d_tasks, int ntasks, int maxp, int csize, double* d_scratch,
                               int* d_status, cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  const int64_t per = jacobi_cluster_scratch(maxp);
  cudaError_t e = cudaMemsetAsync(d_scratch, 0, (size_t)per * ntasks * sizeof(double), s);
  if (e != cudaSuccess) return e;
  if (csize > 8) {
    cudaFuncSetAttribute(k_jacobi_cl, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    // fall back to the portable size if the device cannot co-schedule csize CTAs
    cudaLaunchConfig_t q = {};
    q.gridDim = dim3(csize, 1, 1);
    q.blockDim = dim3(NT, 1, 1);
    cudaLaunchAttribute qa[1];
    qa[0].id = cudaLaunchAttributeClusterDimension;
    qa[0].val.clusterDim.x = csize;
    qa[0].val.clusterDim.y = 1;
    qa[0].val.clusterDim.z = 1;
    q.attrs = qa;
    q.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_jacobi_cl, &q) != cudaSuccess || nclusters < 1) {
      cudaGetLastError();
      csize = 8;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ntasks * csize, 1, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, k_jacobi_cl, d_tasks, d_scratch, per, d_status);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace h2k
