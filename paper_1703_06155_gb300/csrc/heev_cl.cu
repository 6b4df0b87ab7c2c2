// Hermitian eigen-decomposition of the Step-0 Ritz matrices (eq. 17: the
// eigenpairs of the fill-in Gram above eps^2 nu^2) by Householder reduction
// to real tridiagonal form, implicit QL iteration with accumulated rotations,
// and back-transformation; one thread-block cluster of C CTAs (1 .. 16) per
// matrix.
//
// GB300's FP64 pipe (2 FMA per clock per SM) makes flops the cost: cyclic
// Jacobi needs about 24 n^3 real flops per sweep and 5-7 sweeps here, this
// path about 18 n^3 in all:
//   1. tridiagonalization A = Q T Q^H, Q = H_0 ... H_{n-2}, H_j = I - tau_j
//      v_j v_j^H with a real subdiagonal (LAPACK's lower-Hermitian
//      convention).  Column c of the trailing matrix lives in the shared
//      memory of CTA c mod C.  Per step j: every CTA forms x_c = tau (A v)_c
//      for its own columns from the column itself ((A v)_c = sum_i
//      conj(A_ic) v_i, A Hermitian) and its part of x^H v; one cluster
//      barrier; every CTA then applies the rank-2 update A -= v w^H + w v^H,
//      w = x - tau (x^H v) v / 2, to its own columns, and the owner of column
//      j+1 forms reflector j+1; a second cluster barrier.  The reflectors go
//      to the input array (its column j, rows j+1 ..), the other CTAs read
//      them from there.
//   2. T = Z diag(lambda) Z^T by the implicit QL method with Wilkinson
//      shifts: one thread (CTA 0, warp 0) runs the scalar recurrence and
//      emits one bulge-chasing sweep of plane rotations per phase into a
//      double buffer in global memory; in the same phase the other warps of
//      every CTA apply the previous sweep to their block of rows of Z (kept
//      in shared memory); one cluster barrier per phase.
//   3. eigenvalues sorted in decreasing order (ties: lower index first);
//      U(:, rank(k)) = Q Z(:, k), one warp per column, the reflectors read
//      from global memory, no barrier between them.
// Every loop is bounded; an eigenvalue that needs more than kMaxIt QL steps
// sets status bit 2 and is taken as it stands.
#include <cooperative_groups.h>

#include <algorithm>

#include "h2_kernels.h"

namespace cg = cooperative_groups;

namespace h2k {
namespace {

constexpr int NT = 512;
constexpr int NW = NT / 32;
constexpr int kMaxIt = 60;       // QL steps per eigenvalue
constexpr int HEEV_SMEM = 227 * 1024 - 1024;  // dynamic shared memory (static use < 1 KB)

__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// CTA-wide sum, result to every thread
__device__ double bsum(double v, double* red) {
  v = wsum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0;
  if (threadIdx.x < 32) {
    t = (l < NW) ? red[l] : 0.0;
    t = wsum(t);
    if (l == 0) red[0] = t;
  }
  __syncthreads();
  t = red[0];
  __syncthreads();
  return t;
}

__device__ __forceinline__ cd cmul(cd a, cd b) {
  cd r;
  r.re = a.re * b.re - a.im * b.im;
  r.im = a.re * b.im + a.im * b.re;
  return r;
}
__device__ __forceinline__ cd cmulc(cd a, cd b) {  // conj(a) * b
  cd r;
  r.re = a.re * b.re + a.im * b.im;
  r.im = a.re * b.im - a.im * b.re;
  return r;
}

// scratch of one task, in doubles (offsets of the parts)
struct Lay {
  int64_t tau, d, e, x, part, ring, z, total;
};
__host__ __device__ inline Lay heev_layout(int n) {
  Lay L;
  int64_t o = 0;
  L.tau = o;  o += 2 * (int64_t)n;          // tau_j (complex)
  L.d = o;    o += n;                        // diagonal of T
  L.e = o;    o += n;                        // subdiagonal of T
  L.x = o;    o += 2 * (int64_t)n;          // x = tau A v (complex)
  L.part = o; o += 2 * 2 * 16;               // per-CTA parts of x^H v, by parity (complex)
  L.ring = o; o += 2 * (4 + 2 * (int64_t)n); // two QL sweeps: header (count, lo, hi, done) + c[], s[]
  L.z = o;    o += (int64_t)n * n;           // Z (n x n, column-major)
  L.total = (o + 1) & ~(int64_t)1;
  return L;
}

__global__ void __launch_bounds__(NT) k_heev_cl(const EigTask* __restrict__ tasks, double* __restrict__ scratch,
                                               int64_t per_task, int* status) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int ti = blockIdx.x / C;
  const EigTask t = tasks[ti];
  const int n = t.p;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __shared__ double red[32];
  __shared__ cd sh_alpha;
  cd* A = t.A;  // n x n in global memory; becomes the reflector store
  cd* U = t.U;
  if (n <= 1) {
    if (rank == 0 && tid == 0) {
      if (n == 1) {
        U[0].re = 1;
        U[0].im = 0;
        t.lam[0] = A[0].re;
      }
      if (t.sweeps) *t.sweeps = 0;
    }
    return;
  }
  double* base = scratch + ti * per_task;
  const Lay LY = heev_layout(n);
  cd* tau = (cd*)(base + LY.tau);
  double* dg = base + LY.d;
  double* eg = base + LY.e;
  cd* X = (cd*)(base + LY.x);
  cd* part = (cd*)(base + LY.part);
  double* ring = base + LY.ring;
  double* Zg = base + LY.z;
  extern __shared__ __align__(16) unsigned char hsm[];
  // own columns c = rank + C q (q = 0 .. ncol-1), full length n, ld n
  const int ncol = rank < n ? (n - rank + C - 1) / C : 0;
  cd* Ac = reinterpret_cast<cd*>(hsm);
  cd* vs = Ac + (size_t)ncol * n;  // current reflector (length n, rows j+1 ..)
  cd* ws = vs + n;                 // current w
  for (int idx = tid; idx < ncol * n; idx += NT) {
    const int q = idx / n, i = idx % n;
    Ac[idx] = A[i + (size_t)(rank + q * C) * n];
  }
  __syncthreads();

  // reflector of column j (owned here, local index qj): annihilates rows
  // j+2 .. n-1, makes row j+1 real; writes v (v_{j+1} = 1) to A(:, j), tau,
  // d_j and e_j; all threads of the owner CTA call it
  auto reflector = [&](int j, int qj) {
    cd* col = Ac + (size_t)qj * n;
    double s = 0;
    for (int i = j + 2 + tid; i < n; i += NT) s += col[i].re * col[i].re + col[i].im * col[i].im;
    s = bsum(s, red);
    const cd al = col[j + 1];
    cd tj;
    tj.re = 0;
    tj.im = 0;
    double beta = al.re;
    cd sc;
    sc.re = 0;
    sc.im = 0;
    if (!(s == 0.0 && al.im == 0.0)) {
      const double nrm = sqrt(al.re * al.re + al.im * al.im + s);
      beta = al.re >= 0 ? -nrm : nrm;
      tj.re = (beta - al.re) / beta;
      tj.im = -al.im / beta;
      const double dr = al.re - beta, di = al.im, dd = dr * dr + di * di;
      sc.re = dr / dd;  // 1 / (alpha - beta)
      sc.im = -di / dd;
    }
    for (int i = j + 1 + tid; i < n; i += NT) {
      cd v;
      if (i == j + 1) {
        v.re = 1;
        v.im = 0;
      } else if (tj.re == 0.0 && tj.im == 0.0) {
        v.re = 0;
        v.im = 0;
      } else {
        v = cmul(col[i], sc);
      }
      A[i + (size_t)j * n] = v;
    }
    if (tid == 0) {
      tau[j] = tj;
      dg[j] = col[j].re;
      eg[j] = beta;
    }
  };

  // -------------------------------------------------- 1. tridiagonalization
  if (rank == 0) reflector(0, 0);
  cluster_barrier();
  for (int j = 0; j < n - 1; ++j) {
    const cd tj = tau[j];
    const int len = n - j - 1;  // trailing rows / columns j+1 .. n-1
    for (int i = tid; i < len; i += NT) vs[j + 1 + i] = A[j + 1 + i + (size_t)j * n];
    __syncthreads();
    // own columns of the trailing block: c = rank + C q >= j + 1
    const int q0 = (j + 1 - rank + C - 1) / C > 0 ? (j + 1 - rank + C - 1) / C : 0;
    const bool active = !(tj.re == 0.0 && tj.im == 0.0);
    cd pacc;
    pacc.re = 0;
    pacc.im = 0;
    if (active) {
      // x_c = tau * sum_i conj(A_ic) v_i, one warp per own column
      for (int q = q0 + warp; q < ncol; q += NW) {
        const int c = rank + q * C;
        const cd* col = Ac + (size_t)q * n;
        double yr = 0, yi = 0;
        for (int i = j + 1 + lane; i < n; i += 32) {
          const cd a = col[i], v = vs[i];
          yr += a.re * v.re + a.im * v.im;  // conj(a) v
          yi += a.re * v.im - a.im * v.re;
        }
        yr = wsum(yr);
        yi = wsum(yi);
        if (lane == 0) {
          cd y;
          y.re = yr;
          y.im = yi;
          const cd x = cmul(tj, y);
          X[c] = x;
          const cd xv = cmulc(x, vs[c]);  // conj(x_c) v_c
          pacc.re += xv.re;
          pacc.im += xv.im;
        }
      }
    }
    // this CTA's part of x^H v (lane 0 of each warp holds its columns' sum)
    pacc.re = bsum(lane == 0 ? pacc.re : 0.0, red);
    pacc.im = bsum(lane == 0 ? pacc.im : 0.0, red);
    if (tid == 0) part[(j & 1) * 16 + rank] = pacc;
    cluster_barrier();
    if (active) {
      if (tid == 0) {
        cd s;
        s.re = 0;
        s.im = 0;
        for (int r = 0; r < C; ++r) {
          s.re += part[(j & 1) * 16 + r].re;
          s.im += part[(j & 1) * 16 + r].im;
        }
        // alpha = -tau (x^H v) / 2
        const cd a = cmul(tj, s);
        sh_alpha.re = -0.5 * a.re;
        sh_alpha.im = -0.5 * a.im;
      }
      __syncthreads();
      const cd al = sh_alpha;
      for (int i = tid; i < len; i += NT) {
        const cd x = X[j + 1 + i], v = vs[j + 1 + i];
        cd w = cmul(al, v);
        w.re += x.re;
        w.im += x.im;
        ws[j + 1 + i] = w;
      }
      __syncthreads();
      // A_ic -= v_i conj(w_c) + w_i conj(v_c), own columns c >= j + 1
      const int nq = ncol - q0;
      for (int idx = tid; idx < nq * len; idx += NT) {
        const int q = q0 + idx / len, i = j + 1 + idx % len;
        const int c = rank + q * C;
        const cd vi = vs[i], wi = ws[i], vc = vs[c], wc = ws[c];
        cd& a = Ac[(size_t)q * n + i];
        a.re -= vi.re * wc.re + vi.im * wc.im + wi.re * vc.re + wi.im * vc.im;
        a.im -= vi.im * wc.re - vi.re * wc.im + wi.im * vc.re - wi.re * vc.im;
      }
      __syncthreads();
    }
    // next reflector by the owner of column j + 1 (the last column only
    // gives its diagonal entry)
    if ((j + 1) % C == rank) {
      const int q = (j + 1) / C;
      if (j + 1 < n - 1) reflector(j + 1, q);
      else if (tid == 0) dg[n - 1] = Ac[(size_t)q * n + n - 1].re;
    }
    cluster_barrier();
  }

  // -------------------------------------------------- 2. implicit QL on T
  // rows [r0, r1) of Z in shared memory (ld rb), reusing the column store
  const int rb = (n + C - 1) / C;
  const int r0 = min(n, rank * rb), r1 = min(n, r0 + rb), nr = r1 - r0;
  double* Zs = reinterpret_cast<double*>(hsm);
  for (int idx = tid; idx < nr * n; idx += NT) {
    const int k = idx % nr, i = idx / nr;
    Zs[k + (size_t)i * rb] = (r0 + k == i) ? 1.0 : 0.0;
  }
  // the producer thread keeps T (scaled to max |entry| = 1) in shared memory
  double* Td = reinterpret_cast<double*>(ws + n);  // after the column store's w
  double* Te = Td + n;
  __shared__ double tscale;
  __shared__ int qsweeps;
  const bool producer = rank == 0 && tid == 0;
  if (rank == 0) {
    if (tid == 0) {
      double mx = 0;
      for (int i = 0; i < n; ++i) mx = fmax(mx, fabs(dg[i]));
      for (int i = 0; i < n - 1; ++i) mx = fmax(mx, fabs(eg[i]));
      tscale = mx > 0 ? mx : 1.0;
      qsweeps = 0;
    }
    __syncthreads();
    for (int i = tid; i < n; i += NT) {
      Td[i] = dg[i] / tscale;
      Te[i] = i < n - 1 ? eg[i] / tscale : 0.0;
    }
    __syncthreads();
  }
  // producer state: current eigenvalue index and its iteration count
  int l = 0, it = 0;
  // one QL sweep into ring slot b: header (count, lo, hi, done), then c, s
  auto produce = [&](int b) {
    double* hd = ring + (int64_t)b * (4 + 2 * (int64_t)n);
    double* cs = hd + 4;
    double* sn = cs + n;
    const double epsm = 2.220446049250313e-16;
    while (l < n) {
      int m = l;
      for (; m < n - 1; ++m) {
        // negligible: relative to the neighbouring diagonal, or below the
        // rounding level of T itself (|T| = 1 here), which is already the
        // accuracy of the Householder reduction; the absolute floor lets
        // exactly or nearly degenerate pairs of tiny eigenvalues deflate
        const double dd = fabs(Td[m]) + fabs(Td[m + 1]);
        if (fabs(Te[m]) <= epsm * dd + 0.25 * epsm) break;
      }
      if (m == l) {
        ++l;
        it = 0;
        continue;
      }
      if (it++ >= kMaxIt) {
        if (status) atomicOr(status, 2);
        Te[l] = 0.0;
        continue;
      }
      // Wilkinson-type shift from the leading 2 x 2 of the block [l, m]
      double g = (Td[l + 1] - Td[l]) / (2.0 * Te[l]);
      double r = sqrt(g * g + 1.0);
      g = Td[m] - Td[l] + Te[l] / (g + (g >= 0 ? r : -r));
      double s = 1.0, c = 1.0, p = 0.0;
      int i = m - 1;
      int cnt = 0;
      bool split = false;
      for (; i >= l; --i) {
        const double f = s * Te[i], bq = c * Te[i];
        const double rr = f * f + g * g;
        if (rr == 0.0) {  // the block splits: no rotation here
          Td[i + 1] -= p;
          Te[m] = 0.0;
          split = true;
          break;
        }
        const double ir = rsqrt(rr);
        r = rr * ir;
        Te[i + 1] = r;
        s = f * ir;
        c = g * ir;
        g = Td[i + 1] - p;
        r = (Td[i] - g) * s + 2.0 * c * bq;
        p = s * r;
        Td[i + 1] = g + p;
        g = c * r - bq;
        cs[cnt] = c;
        sn[cnt] = s;
        ++cnt;
      }
      if (!split) {
        Td[l] -= p;
        Te[l] = g;
        Te[m] = 0.0;
      }
      // rotations hi = m - 1 down to lo = hi - cnt + 1
      hd[0] = cnt;
      hd[1] = m - cnt;
      hd[2] = m - 1;
      hd[3] = 0;
      ++qsweeps;
      return;
    }
    hd[0] = 0;
    hd[3] = 1;  // done
  };
  // apply the sweep in slot b to the own rows (warps 1 .. NW-1 of every CTA)
  auto apply = [&](int b) {
    const double* hd = ring + (int64_t)b * (4 + 2 * (int64_t)n);
    const int cnt = (int)hd[0], hi = (int)hd[2];
    if (cnt <= 0) return;
    const double* cs = hd + 4;
    const double* sn = cs + n;
    for (int k = tid - 32; k < nr; k += NT - 32) {
      double carry = Zs[k + (size_t)(hi + 1) * rb];
      for (int u = 0; u < cnt; ++u) {
        const int i = hi - u;
        const double c = cs[u], s = sn[u];
        const double zi = Zs[k + (size_t)i * rb];
        Zs[k + (size_t)(i + 1) * rb] = s * zi + c * carry;
        carry = c * zi - s * carry;
      }
      Zs[k + (size_t)(hi - cnt + 1) * rb] = carry;
    }
  };
  if (producer) produce(0);
  cluster_barrier();
  for (int ph = 0;; ++ph) {
    const double* hd = ring + (int64_t)(ph & 1) * (4 + 2 * (int64_t)n);
    if (hd[3] != 0.0) break;
    if (producer) produce((ph + 1) & 1);
    else if (tid >= 32) apply(ph & 1);
    cluster_barrier();
  }
  // eigenvalues back to the matrix scale, Z to global memory
  if (producer) {
    for (int i = 0; i < n; ++i) dg[i] = Td[i] * tscale;
    if (t.sweeps) *t.sweeps = qsweeps;
  }
  for (int idx = tid; idx < nr * n; idx += NT) {
    const int k = idx % nr, i = idx / nr;
    Zg[(r0 + k) + (size_t)i * n] = Zs[k + (size_t)i * rb];
  }
  cluster_barrier();

  // -------------------------------------------------- 3. sort, U = Q Z
  // rank of eigenvalue k in decreasing order (ties: lower index first)
  int* rk = reinterpret_cast<int*>(hsm);
  for (int k = tid; k < n; k += NT) {
    const double lk = dg[k];
    int r = 0;
    for (int j = 0; j < n; ++j) {
      const double lj = dg[j];
      r += (lj > lk) || (lj == lk && j < k);
    }
    rk[k] = r;
    if (rank == 0) t.lam[r] = lk;
  }
  __syncthreads();
  // eigenvector k = rank + C u: one warp per vector, u = Z(:, k) in shared memory
  cd* ub = reinterpret_cast<cd*>(hsm + ((n * sizeof(int) + 15) / 16) * 16) + (size_t)warp * n;
  for (int k = rank + warp * C; k < n; k += NW * C) {
    for (int i = lane; i < n; i += 32) {
      ub[i].re = Zg[i + (size_t)k * n];
      ub[i].im = 0;
    }
    __syncwarp();
    for (int j = n - 2; j >= 0; --j) {
      const cd tj = tau[j];
      if (tj.re == 0.0 && tj.im == 0.0) continue;
      double dr = 0, di = 0;
      for (int i = j + 1 + lane; i < n; i += 32) {
        const cd v = A[i + (size_t)j * n], u = ub[i];
        dr += v.re * u.re + v.im * u.im;  // conj(v) u
        di += v.re * u.im - v.im * u.re;
      }
      dr = wsum(dr);
      di = wsum(di);
      cd dd;
      dd.re = dr;
      dd.im = di;
      const cd f = cmul(tj, dd);  // u -= tau v (v^H u)
      for (int i = j + 1 + lane; i < n; i += 32) {
        const cd v = A[i + (size_t)j * n];
        ub[i].re -= v.re * f.re - v.im * f.im;
        ub[i].im -= v.re * f.im + v.im * f.re;
      }
      __syncwarp();
    }
    const int col = rk[k];
    for (int i = lane; i < n; i += 32) U[i + (size_t)col * n] = ub[i];
    __syncwarp();
  }
}

size_t heev_smem_bytes(int n, int C) {
  const int ncol = (n + C - 1) / C;
  const size_t cols = (size_t)ncol * n * sizeof(cd) + 2 * (size_t)n * sizeof(cd) + 2 * (size_t)n * sizeof(double);
  const size_t sortb = ((n * sizeof(int) + 15) / 16) * 16 + (size_t)NW * n * sizeof(cd);
  return cols > sortb ? cols : sortb;
}

}  // namespace

int heev_max_order() { return 452; }

int64_t heev_cluster_scratch(int maxp) { return heev_layout(maxp).total; }

// CTAs per problem: the own columns of every CTA must fit in shared memory;
// few problems get more CTAs (the SMs are idle otherwise)
int heev_cluster_size(int ntasks, int maxp, int cmax) {
  int C = 1;
  while (C < 16 && heev_smem_bytes(maxp, C) > (size_t)HEEV_SMEM) C *= 2;
  int want = ntasks * 16 <= 2 * 152 ? 16 : ntasks * 8 <= 2 * 152 ? 8 : 4;
  want = std::min(want, std::max(1, (maxp + 15) / 16));
  C = std::max(C, want);
  C = std::min(C, std::max(1, cmax));
  while (C < 16 && heev_smem_bytes(maxp, C) > (size_t)HEEV_SMEM) C *= 2;
  return C;
}

cudaError_t heev_cluster(const EigTask* d_tasks, int ntasks, int maxp, int csize, double* d_scratch, int* d_status,
                         cudaStream_t s, int* csize_used) {
  if (ntasks <= 0) return cudaSuccess;
  if (maxp > heev_max_order() || csize < 1 || csize > 16) return cudaErrorInvalidValue;
  const size_t smem = heev_smem_bytes(maxp, csize);
  if (smem > (size_t)HEEV_SMEM) return cudaErrorInvalidValue;
  const int64_t per = heev_cluster_scratch(maxp);
  cudaError_t e = cudaFuncSetAttribute(k_heev_cl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (csize > 8) {
    cudaFuncSetAttribute(k_heev_cl, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
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
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_heev_cl, &q) != cudaSuccess || nclusters < 1) {
      cudaGetLastError();
      csize = 8;
      if (heev_smem_bytes(maxp, csize) > (size_t)HEEV_SMEM) return cudaErrorInvalidValue;
      e = cudaFuncSetAttribute(k_heev_cl, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)heev_smem_bytes(maxp, csize));
      if (e != cudaSuccess) return e;
    }
  }
  if (csize_used) *csize_used = csize;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ntasks * csize, 1, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = heev_smem_bytes(maxp, csize);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, k_heev_cl, d_tasks, d_scratch, per, d_status);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace h2k
