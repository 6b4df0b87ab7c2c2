// Hermitian Jacobi eigen-decomposition spread over a thread-block cluster.
//
// Same method as the one-CTA kernel (cyclic Jacobi, parallel round-robin
// ordering; a 2 x 2 block [[a, g e^{i phi}], [g e^{-i phi}, d]] is rotated by
// G = diag(1, e^{-i phi}) J with J the real Jacobi rotation of [[a, g],[g, d]]),
// but each eigenproblem runs on one cluster of CTAs so that its FP64 work is
// spread over several SMs.  Per round:
//   1. every CTA computes all rotations of the round into its shared memory;
//   2. the rotations form one block-diagonal unitary G, so each 2 x 2 block
//      of G^H A G is G_P^H A[P, Q] G_Q: each CTA updates the two columns of
//      the pairs Q it owns (pair q is owned by CTA q mod C), rows and columns
//      rotated at once, and the same columns of U.
// Rounds are separated by one cluster barrier with release / acquire
// semantics (hardware barrier.cluster; no software spin), which orders the
// global-memory traffic of the cluster's threads.  A matrix whose sweeps do
// not converge within kMaxSweeps sets status bit 2 and returns its current
// state.
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
  // entries that the next round's rotations read, double-buffered by round
  // parity: Dd[k] = A(k, k), Do[b] = A(a, b) of the pair (a < b); written by
  // the owner of column k / b after its updates, read by every CTA after the
  // cluster barrier (so no CTA reads A while another one writes it)
  double* Dd = base;                    // 2 x pe
  cd* Do = (cd*)(base + 2 * (size_t)pe);  // 2 x pe
  int* pa = (int*)(base + 6 * (size_t)pe);
  int* pb = pa + np;
  int* flags = pb + np;           // per sweep: a rotation happened (zeroed by the host)
  int* open = flags + kMaxSweeps;  // per sweep: an entry above its threshold at the start
  cd* A = t.A;
  cd* U = t.U;
  __shared__ double red[32];
  // rotation parameters of the current round (all pairs), dynamic shared memory
  extern __shared__ double jsh[];
  double* jc = jsh;
  double* js = jc + np;
  double* jer = js + np;
  double* jei = jer + np;
  int* ja = (int*)(jei + np);
  int* jb = ja + np;
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
  // entries at the rounding level of the matrix are not rotated, nor entries
  // far below the truncation threshold of the rank decision (eq. 17), whose
  // rotation would move the eigenvalues by less than that floor
  const double gmin = fmax(fmax(1e-300, 4e-16 * sqrt(fro)), t.trM ? t.tol_rel * t.eps2 * (t.snorm2 + *t.trM) : 0.0);
  const int m = pe - 1;  // round-robin modulus
  // partner of index k in round r (pair 0 = (pe - 1, r), pair i = (r + i, r - i) mod m)
  auto partner = [&](int k, int r) { return k == pe - 1 ? r : k == r ? pe - 1 : ((2 * r - k) % m + m) % m; };
  if (rank == 0)
    for (int k = threadIdx.x; k < p; k += NT) {
      Dd[k] = A[k + (size_t)k * p].re;
      const int j = partner(k, 0);
      if (j < k) Do[k] = A[j + (size_t)k * p];
    }
  cluster_barrier();
  int sweep = 0, tr = 0;  // tr: rounds so far (buffer parity)
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
      // 1. every CTA computes all rotations of the round (pair i = (a, b))
      //    from the entries published for it, into shared memory
      for (int i = threadIdx.x; i < np; i += NT) {
        int a, b;
        if (i == 0) { a = pe - 1; b = r; } else { a = (r + i) % (pe - 1); b = (r - i + pe - 1) % (pe - 1); }
        if (a > b) { const int x = a; a = b; b = x; }
        double c = 1, s = 0, er = 1, ei = 0;
        if (b < p) {
          const int bi = tr & 1;
          const double app = Dd[bi * pe + a], aqq = Dd[bi * pe + b];
          const cd apq = Do[bi * pe + b];
          const double g2 = apq.re * apq.re + apq.im * apq.im;
          const double g = sqrt(g2);  // the threshold test of the convergence check
          // one reciprocal square root (issued beside the test) gives 1/g for
          // e^{i phi} and zeta; the dependent chain is rsqrt -> sqrt -> divide -> rsqrt
          const double rg = g2 > 0.0 ? rsqrt(g2) : 0.0;
          if (g > gmin && g > 1e-17 * sqrt(fabs(app * aqq))) {
            er = apq.re * rg;
            ei = apq.im * rg;
            const double zeta = (aqq - app) * 0.5 * rg;
            const double tt = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            c = rsqrt(1.0 + tt * tt);
            s = tt * c;
            flags[sweep] = 1;
          }
        }
        ja[i] = a;
        jb[i] = b;
        jc[i] = c;
        js[i] = s;
        jer[i] = er;
        jei[i] = ei;
      }
      __syncthreads();
      // 2. the pair rotations form one block-diagonal unitary G, so every 2 x 2
      //    block of G^H A G is G_P^H A[P, Q] G_Q.  This CTA updates the two
      //    columns of its own pairs Q (pair q is owned by CTA q mod C) for all
      //    row pairs P, and the same columns of U (U G_Q); no other CTA
      //    touches them in this round.
      // Entries that the next round's rotations read (A(k, k) and A(j, k) of
      // its pairs j < k) are published by the thread that owns them here, from
      // unrotated blocks too, into the other parity's buffer.
      const int rn = (r + 1) % m, nbuf = (tr + 1) & 1;
      auto publish = [&](int row, int col, const cd& v) {
        if (row == col) Dd[nbuf * pe + col] = v.re;
        else if (row < col && partner(col, rn) == row) Do[nbuf * pe + col] = v;
      };
      auto needed = [&](int row, int col) { return row == col || (row < col && partner(col, rn) == row); };
      {
        const int nown = rank < np ? (np - rank + C - 1) / C : 0;
        const int totA = nown * np, tot = totA + nown * p;
        for (int idx = threadIdx.x; idx < tot; idx += NT) {
          if (idx < totA) {
            const int q = rank + (idx / np) * C, P = idx % np;
            const double sq = js[q], sp = js[P];
            const int aq = ja[q], bq = jb[q], ap = ja[P], bp = jb[P];
            const bool hq = bq < p, hp = bp < p;  // the padding index of an odd order has no row / column
            if (sq == 0.0 && sp == 0.0) {
              if (needed(ap, aq)) publish(ap, aq, A[ap + (size_t)aq * p]);
              if (hp && needed(bp, aq)) publish(bp, aq, A[bp + (size_t)aq * p]);
              if (hq && needed(ap, bq)) publish(ap, bq, A[ap + (size_t)bq * p]);
              if (hp && hq && needed(bp, bq)) publish(bp, bq, A[bp + (size_t)bq * p]);
              continue;
            }
            cd x11 = A[ap + (size_t)aq * p], x21, x12, x22;
            x21.re = x21.im = x12.re = x12.im = x22.re = x22.im = 0;
            if (hp) x21 = A[bp + (size_t)aq * p];
            if (hq) x12 = A[ap + (size_t)bq * p];
            if (hp && hq) x22 = A[bp + (size_t)bq * p];
            // columns: new a = c x_a - s conj(e) x_b ; new b = s x_a + c conj(e) x_b
            if (sq != 0.0) {
              const double c = jc[q], er = jer[q], ei = -jei[q];
              const double e1r = er * x12.re - ei * x12.im, e1i = er * x12.im + ei * x12.re;
              const double e2r = er * x22.re - ei * x22.im, e2i = er * x22.im + ei * x22.re;
              cd n11, n12, n21, n22;
              n11.re = c * x11.re - sq * e1r;
              n11.im = c * x11.im - sq * e1i;
              n12.re = sq * x11.re + c * e1r;
              n12.im = sq * x11.im + c * e1i;
              n21.re = c * x21.re - sq * e2r;
              n21.im = c * x21.im - sq * e2i;
              n22.re = sq * x21.re + c * e2r;
              n22.im = sq * x21.im + c * e2i;
              x11 = n11;
              x12 = n12;
              x21 = n21;
              x22 = n22;
            }
            // rows: new a = c y_a - s e y_b ; new b = s y_a + c e y_b
            if (sp != 0.0) {
              const double c = jc[P], er = jer[P], ei = jei[P];
              const double e1r = er * x21.re - ei * x21.im, e1i = er * x21.im + ei * x21.re;
              const double e2r = er * x22.re - ei * x22.im, e2i = er * x22.im + ei * x22.re;
              cd n11, n12, n21, n22;
              n11.re = c * x11.re - sp * e1r;
              n11.im = c * x11.im - sp * e1i;
              n21.re = sp * x11.re + c * e1r;
              n21.im = sp * x11.im + c * e1i;
              n12.re = c * x12.re - sp * e2r;
              n12.im = c * x12.im - sp * e2i;
              n22.re = sp * x12.re + c * e2r;
              n22.im = sp * x12.im + c * e2i;
              x11 = n11;
              x12 = n12;
              x21 = n21;
              x22 = n22;
            }
            // the rotated pair's off-diagonal entries are zero by construction
            if (P == q) {
              x12.re = x12.im = 0;
              x21.re = x21.im = 0;
              x11.im = 0;
              x22.im = 0;
            }
            A[ap + (size_t)aq * p] = x11;
            if (hp) A[bp + (size_t)aq * p] = x21;
            if (hq) A[ap + (size_t)bq * p] = x12;
            if (hp && hq) A[bp + (size_t)bq * p] = x22;
            publish(ap, aq, x11);
            if (hp) publish(bp, aq, x21);
            if (hq) publish(ap, bq, x12);
            if (hp && hq) publish(bp, bq, x22);
          } else {
            const int e = idx - totA;
            const int q = rank + (e / p) * C, row = e % p;
            const double sq = js[q];
            if (sq == 0.0) continue;
            const int aq = ja[q], bq = jb[q];
            const double c = jc[q], er = jer[q], ei = -jei[q];
            const cd xa = U[row + (size_t)aq * p], xb = U[row + (size_t)bq * p];
            const double ebr = er * xb.re - ei * xb.im, ebi = er * xb.im + ei * xb.re;
            cd na, nb;
            na.re = c * xa.re - sq * ebr;
            na.im = c * xa.im - sq * ebi;
            nb.re = sq * xa.re + c * ebr;
            nb.im = sq * xa.im + c * ebi;
            U[row + (size_t)aq * p] = na;
            U[row + (size_t)bq * p] = nb;
          }
        }
      }
      ++tr;
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
  // doubles; even, so that every task's block (which holds complex128
  // entries) starts on a 16-byte boundary
  const int64_t n = (int64_t)np * 12 + (np * 2 + 2 * kMaxSweeps + 8) / 2 + 8;
  return (n + 1) & ~(int64_t)1;
}

cudaError_t jacobi_eig_cluster(const EigTask* d_tasks, int ntasks, int maxp, int csize, double* d_scratch,
                               int* d_status, cudaStream_t s, int* csize_used) {
  if (ntasks <= 0) return cudaSuccess;
  const int64_t per = jacobi_cluster_scratch(maxp);
  cudaError_t e = cudaMemsetAsync(d_scratch, 0, (size_t)per * ntasks * sizeof(double), s);
  if (e != cudaSuccess) return e;
  const size_t smem = (size_t)((maxp + 1) / 2 + 1) * (4 * sizeof(double) + 2 * sizeof(int));
  e = cudaFuncSetAttribute(k_jacobi_cl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (csize > 8) {
    cudaFuncSetAttribute(k_jacobi_cl, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    // fall back to the portable size if the device cannot co-schedule csize CTAs
    cudaLaunchConfig_t q = {};
    q.gridDim = dim3(csize, 1, 1);
    q.blockDim = dim3(NT, 1, 1);
    q.dynamicSmemBytes = smem;
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
  if (csize_used) *csize_used = csize;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ntasks * csize, 1, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
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
