// Step-0 eigen-decomposition (eq. 17) by a one-sided Jacobi SVD of the
// Cholesky factor, in double-float arithmetic on the FP32 pipe.
//
// The pivoted Cholesky of the fill-in Gram gives G' = L L^H + E with E
// positive semidefinite and trace(E) <= thr / 10, and its Householder QR gives
// L = Q [R; 0].  The eigenvalues of L L^H are the squared singular values of
// the r' x r' factor R, and by Weyl's inequality they lie within
// ||E|| <= trace(E) <= thr / 10 of the eigenvalues of G' (the same margin as
// the Ritz values on span(L)), so the truncation can be decided on R.  This
// kernel computes R R^H = U diag(lam) U^H without forming R R^H:
//   W = R^H; for column pairs (x, y) of W: with alpha = |w_x|^2,
//   beta = |w_y|^2 and gamma = w_x^H w_y = g e^{i phi}, the unitary
//   V = [[c, s], [-s e^{-i phi}, c e^{-i phi}]] (t = tan of the real Jacobi
//   angle of [[alpha, g], [g, beta]], c = 1 / sqrt(1 + t^2), s = c t) makes
//   the two columns of W V orthogonal; V is applied to W and accumulated into
//   J (J = I at the start).  At convergence W^H W = J^H (R R^H) J is
//   diagonal: lam_j = |w_j|^2 and U = J.
// Working on the square root halves the exponent range the arithmetic has to
// resolve: an eigenvalue at the threshold, thr ~ eps^2 ||G'||, is a singular
// value at eps ||R||, which double-float (about 48 significant bits) resolves
// to ~1e-9 relative at eps = 1e-6.  J is a product of exactly normalized
// rotations (c^2 + s^2 = 1 and |e^{i phi}| = 1 to double-float accuracy), so
// it stays unitary to ~1e-13 whatever the singular values.
//
// Parallel order: the r' columns are split into 2C blocks of b columns.  Each
// sweep is a round-robin tournament of the blocks (2C - 1 super-rounds, block
// 2C - 1 fixed); in a super-round each CTA of the cluster takes one block pair,
// stages its 2b columns of W and J in shared memory and rotates all b^2
// cross pairs (b rounds of b disjoint pairs); the first super-round of a sweep
// also rotates the pairs inside the two blocks (a round robin over the 2b
// columns).  Every column pair is rotated once per sweep.  A team of warps
// takes one pair of a round.  Super-rounds are separated by one cluster
// barrier (release / acquire), after the CTAs have written their columns
// back.  Pairs whose |gamma| is below 1e-7 sqrt(alpha beta) or below tol_rel
// of the truncation threshold are not rotated; a sweep that rotates nothing
// ends the iteration.  A problem that has not converged after kMaxSweeps
// sweeps sets status bit 2 and returns its state.
#include <cooperative_groups.h>

#include "dfloat.cuh"
#include "h2_kernels.h"

namespace cg = cooperative_groups;

namespace h2k {
namespace {

using namespace dfl;

constexpr int NT = 512;
constexpr int NW = NT / 32;
constexpr int kMaxSweeps = 40;
constexpr int kMaxB = 16;  // columns per block
#ifndef OSJ_TDIV
#define OSJ_TDIV 128  // column entries per warp of a pair's team, at least
#endif
constexpr size_t kSmemMax = 225 * 1024;

__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// [x', y'] = [x, y] V with V = [[c, s], [-sg, kp]], sg = s conj(e), kp = c conj(e)
__device__ __forceinline__ void rotate(float4& xv, float4& yv, df c, df s, df sgr, df sgi, df kpr, df kpi) {
  const df xr = re_of(xv), xi = im_of(xv), yr = re_of(yv), yi = im_of(yv);
  // x' = c x - sg y
  df nxr = dmul(c, xr), nxi = dmul(c, xi);
  nxr = dfma(dneg(sgr), yr, nxr);
  nxr = dfma(sgi, yi, nxr);
  nxi = dfma(dneg(sgr), yi, nxi);
  nxi = dfma(dneg(sgi), yr, nxi);
  // y' = s x + kp y
  df nyr = dmul(s, xr), nyi = dmul(s, xi);
  nyr = dfma(kpr, yr, nyr);
  nyr = dfma(dneg(kpi), yi, nyr);
  nyi = dfma(kpr, yi, nyi);
  nyi = dfma(kpi, yr, nyi);
  xv = pack(nxr, nxi);
  yv = pack(nyr, nyi);
}

__global__ void __launch_bounds__(NT, 1) k_osj_cl(const EigTask* __restrict__ tasks, unsigned char* __restrict__ scratch,
                                                 int64_t per_task, int* status) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int ti = blockIdx.x / C;
  const EigTask t = tasks[ti];
  const int r = t.p;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const cd* R = t.A;  // r x r upper triangular (ld r)
  if (r <= 1) {
    if (rank == 0 && tid == 0) {
      if (r == 1) {
        t.U[0].re = 1;
        t.U[0].im = 0;
        t.lam[0] = R[0].re * R[0].re + R[0].im * R[0].im;
      }
      if (t.sweeps) *t.sweeps = 0;
    }
    return;
  }
  unsigned char* base = scratch + (size_t)ti * per_task;
  float4* Wg = reinterpret_cast<float4*>(base);
  float4* Jg = Wg + (size_t)r * r;
  double* lamd = reinterpret_cast<double*>(Jg + (size_t)r * r);
  int* flags = reinterpret_cast<int*>(lamd + r);  // per sweep: a rotation happened (zeroed by the host)
  const int nblk = 2 * C;
  const int b = (r + nblk - 1) / nblk;
  if (b > kMaxB) {  // the launcher sizes clusters so that this never happens
    if (rank == 0 && tid == 0 && status) atomicMax(status, 2);
    return;
  }
  extern __shared__ float4 osm[];
  float4* Ws = osm;                  // 2b columns of W (ld r)
  float4* Js = osm + (size_t)2 * b * r;  // the same columns of J
  __shared__ df s_nrm[2 * kMaxB];    // |w|^2 of the staged columns
  __shared__ float4 s_part[NW];      // per-warp partial gamma
  __shared__ double s_red[NW];

  // power-of-two scaling: max |R| in [0.5, 1) keeps every product inside the
  // single-precision exponent range
  double mx = 0;
  for (int idx = tid; idx < r * r; idx += NT) {
    const int i = idx % r, j = idx / r;
    if (i <= j) mx = fmax(mx, fmax(fabs(R[idx].re), fabs(R[idx].im)));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) s_red[warp] = mx;
  __syncthreads();
  mx = 0;
  for (int w = 0; w < NW; ++w) mx = fmax(mx, s_red[w]);
  int ex = 0;
  if (mx > 0) frexp(mx, &ex);
  // rotation floor in the scaled units (squared quantities scale by 2^-2ex)
  const double floor_lam = t.trM ? t.tol_rel * t.eps2 * (t.snorm2 + *t.trM) : 0.0;
  const float gmin = (float)fmin(ldexp(floor_lam, -2 * ex), 1e30);
  // relative floor: an unrotated pair with |gamma| <= 1e-7 sqrt(alpha beta)
  // moves an eigenvalue by at most 1e-7 of itself (both columns near the
  // threshold) or by 1e-14 of the smaller one (a large and a small column),
  // and tilts a kept direction into a dropped one by at most that much
  const float tol = 1e-7f;

  // W = R^H (scaled), J = I; columns j = rank (mod C)
  for (int j = rank; j < r; j += C)
    for (int i = tid; i < r; i += NT) {
      float4 w = make_float4(0, 0, 0, 0);
      if (i >= j) {
        const cd v = R[j + (size_t)i * r];
        w = pack(dsplit(ldexp(v.re, -ex)), dsplit(-ldexp(v.im, -ex)));
      }
      Wg[i + (size_t)j * r] = w;
      Jg[i + (size_t)j * r] = make_float4(i == j ? 1.0f : 0.0f, 0, 0, 0);
    }
  cluster_barrier();

  // warps per team (one team per pair of a round): one warp unless the
  // columns are long enough to give every lane of a larger team >= 4 entries
  // (each warp of a team repeats the pair's reductions and parameters)
  const int T = max(1, min(NW / b, r / OSJ_TDIV));
  const int team = warp / T, wt = warp % T;
  int sweep = 0;
  bool done = false;
  for (; sweep < kMaxSweeps && !done; ++sweep) {
    int rot = 0;
    for (int s = 0; s < nblk - 1; ++s) {
      int A, B;
      if (rank == 0) {
        A = nblk - 1;
        B = s;
      } else {
        const int m = nblk - 1;
        A = (s + rank) % m;
        B = (s - rank + m) % m;
      }
      const int a0 = A * b, b0 = B * b;
      const int na = max(0, min(b, r - a0)), nb = max(0, min(b, r - b0));
      auto col_of = [&](int k) { return k < b ? (k < na ? a0 + k : -1) : (k - b < nb ? b0 + k - b : -1); };
      for (int idx = tid; idx < 2 * b * r; idx += NT) {
        const int k = idx / r, i = idx - k * r;
        const int col = col_of(k);
        if (col >= 0) {
          Ws[idx] = Wg[i + (size_t)col * r];
          Js[idx] = Jg[i + (size_t)col * r];
        }
      }
      __syncthreads();
      for (int k = warp; k < 2 * b; k += NW) {
        df a = {0.0f, 0.0f};
        if (col_of(k) >= 0)
          for (int i = lane; i < r; i += 32) {
            const float4 v = Ws[(size_t)k * r + i];
            a = dfma(re_of(v), re_of(v), a);
            a = dfma(im_of(v), im_of(v), a);
          }
        a = wsum(a);
        if (lane == 0) s_nrm[k] = a;
      }
      __syncthreads();
      const int nrounds = s == 0 ? 2 * b - 1 : b;
      for (int k = 0; k < nrounds; ++k) {
        int x = -1, y = -1;
        if (team < b) {
          if (s == 0) {
            const int q = 2 * b - 1;
            if (team == 0) {
              x = q;
              y = k;
            } else {
              x = (k + team) % q;
              y = (k - team + q) % q;
            }
          } else {
            x = team;
            y = b + (team + k) % b;
          }
          if (col_of(x) < 0 || col_of(y) < 0) x = y = -1;
        }
        const bool act = x >= 0;
        df al = {0.0f, 0.0f}, be = {0.0f, 0.0f};
        df gr = {0.0f, 0.0f}, gi = {0.0f, 0.0f};
        if (act) {
          al = s_nrm[x];
          be = s_nrm[y];
          const float4* xs = Ws + (size_t)x * r;
          const float4* ys = Ws + (size_t)y * r;
          for (int i = wt * 32 + lane; i < r; i += T * 32) {
            const float4 xv = xs[i], yv = ys[i];
            // gamma += conj(x) y
            gr = dfma(re_of(xv), re_of(yv), gr);
            gr = dfma(im_of(xv), im_of(yv), gr);
            gi = dfma(re_of(xv), im_of(yv), gi);
            gi = dfma(dneg(im_of(xv)), re_of(yv), gi);
          }
          gr = wsum(gr);
          gi = wsum(gi);
          if (T > 1 && lane == 0) s_part[warp] = pack(gr, gi);
        }
        if (T > 1) {
          // the team's warps combine their partial sums
          __syncthreads();
          if (act) {
            gr = {0.0f, 0.0f};
            gi = {0.0f, 0.0f};
            for (int w = 0; w < T; ++w) {
              const float4 v = s_part[team * T + w];
              gr = dadd(gr, re_of(v));
              gi = dadd(gi, im_of(v));
            }
          }
        }
        if (act) {
          const float gf = hypotf(gr.h, gi.h);
          // entries below 1e-30 of the scaled matrix (max |R| ~ 1) are never
          // rotated: far below any truncation threshold, and keeps the
          // parameters below inside the single-precision exponent range
          if (gf > gmin && gf > 1e-30f && gf > tol * sqrtf(al.h) * sqrtf(be.h)) {
            // gamma scaled by a power of two to unit order for the square roots
            int e2 = 0;
            frexpf(fmaxf(fabsf(gr.h), fabsf(gi.h)), &e2);
            const float f = ldexpf(1.0f, -e2);
            const df grs = dscale(gr, f), gis = dscale(gi, f);
            const df g2s = dfma(grs, grs, dmul(gis, gis));
            const df igs = drsqrt(g2s);
            const df gs = dmul(g2s, igs);                // |gamma| f
            const df g = dscale(gs, ldexpf(1.0f, e2));  // |gamma|
            const df er = dmul(grs, igs), ei = dmul(gis, igs);  // e^{i phi}
            const float zeta = __fdividef(__fmul_rn(dsub(be, al).h, f), 2.0f * gs.h);
            const float az = fabsf(zeta);
            float tt = az > 1e15f ? 0.5f / az : 1.0f / (az + sqrtf(fmaf(az, az, 1.0f)));
            if (zeta < 0) tt = -tt;
            const float p = __fmul_rn(tt, tt);
            const df n1 = quick_two_sum(1.0f, p);
            const df n1e = dadd(n1, df{__fmaf_rn(tt, tt, -p), 0.0f});
            const df c = drsqrt(n1e);
            const df sn = dmul(c, df{tt, 0.0f});
            const df sgr = dmul(sn, er), sgi = dneg(dmul(sn, ei));  // s conj(e)
            const df kpr = dmul(c, er), kpi = dneg(dmul(c, ei));    // c conj(e)
            float4* xs = Ws + (size_t)x * r;
            float4* ys = Ws + (size_t)y * r;
            float4* xj = Js + (size_t)x * r;
            float4* yj = Js + (size_t)y * r;
            for (int i = wt * 32 + lane; i < r; i += T * 32) {
              float4 xv = xs[i], yv = ys[i];
              rotate(xv, yv, c, sn, sgr, sgi, kpr, kpi);
              xs[i] = xv;
              ys[i] = yv;
              float4 xu = xj[i], yu = yj[i];
              rotate(xu, yu, c, sn, sgr, sgi, kpr, kpi);
              xj[i] = xu;
              yj[i] = yu;
            }
            if (wt == 0 && lane == 0) {
              // |w_x'|^2 = c^2 alpha + s^2 beta - 2 c s g, |w_y'|^2 = s^2 alpha + c^2 beta + 2 c s g
              const df cc = dmul(c, c), ss = dmul(sn, sn), csg = dscale(dmul(dmul(c, sn), g), 2.0f);
              s_nrm[x] = dsub(dfma(cc, al, dmul(ss, be)), csg);
              s_nrm[y] = dadd(dfma(ss, al, dmul(cc, be)), csg);
            }
            rot = 1;
          }
        }
        __syncthreads();
      }
      for (int idx = tid; idx < 2 * b * r; idx += NT) {
        const int k = idx / r, i = idx - k * r;
        const int col = col_of(k);
        if (col >= 0) {
          Wg[i + (size_t)col * r] = Ws[idx];
          Jg[i + (size_t)col * r] = Js[idx];
        }
      }
      if (s == nblk - 2 && __syncthreads_or(rot) && tid == 0) flags[sweep] = 1;
      cluster_barrier();
    }
    done = *(volatile int*)&flags[sweep] == 0;
  }
  if (!done && rank == 0 && tid == 0 && status) atomicMax(status, 2);
  if (rank == 0 && tid == 0 && t.sweeps) *t.sweeps = sweep;

  // eigenvalues lam_j = |w_j|^2 (unscaled), own columns j = rank (mod C)
  for (int j = rank + warp * C; j < r; j += NW * C) {
    df a = {0.0f, 0.0f};
    for (int i = lane; i < r; i += 32) {
      const float4 v = Wg[i + (size_t)j * r];
      a = dfma(re_of(v), re_of(v), a);
      a = dfma(im_of(v), im_of(v), a);
    }
    a = wsum(a);
    if (lane == 0) lamd[j] = ldexp(djoin(a), 2 * ex);
  }
  cluster_barrier();
  // decreasing order (ties: lower index first); U(:, rank_j) = J(:, j)
  for (int j = rank + warp * C; j < r; j += NW * C) {
    const double lj = lamd[j];
    int rk = 0;
    for (int i = lane; i < r; i += 32) {
      const double li = lamd[i];
      rk += (li > lj) || (li == lj && i < j);
    }
    for (int o = 16; o > 0; o >>= 1) rk += __shfl_xor_sync(0xffffffffu, rk, o);
    if (lane == 0) t.lam[rk] = lj;
    for (int i = lane; i < r; i += 32) {
      const float4 v = Jg[i + (size_t)j * r];
      cd u;
      u.re = djoin(re_of(v));
      u.im = djoin(im_of(v));
      t.U[i + (size_t)rk * r] = u;
    }
  }
}

size_t smem_bytes(int r, int C) {
  const int b = (r + 2 * C - 1) / (2 * C);
  return (size_t)4 * b * r * sizeof(float4);
}

// smallest cluster whose blocks hold at most kMaxB columns and whose staged
// columns fit in shared memory (orders <= osj_max_order() fit with 16)
int min_cluster(int r) {
  int c = 1;
  while (c < 16 && ((r + 2 * c - 1) / (2 * c) > kMaxB || smem_bytes(r, c) > kSmemMax)) ++c;
  return c;
}

}  // namespace

int osj_max_order() {
  int r = 1;
  while (smem_bytes(r + 1, 16) <= kSmemMax && (r + 1 + 31) / 32 <= kMaxB) ++r;
  return r;
}

int64_t osj_cluster_scratch(int maxp) {
  const int64_t n = (int64_t)2 * maxp * maxp * sizeof(float4) + (int64_t)maxp * sizeof(double) + kMaxSweeps * 4;
  return (n + 255) & ~(int64_t)255;
}

int osj_cluster_size(int ntasks, int maxp, int cmax) {
  // blocks of about 8 columns (8 pairs per round, two warps per SM
  // sub-partition), at most 16 CTAs, and the launch's clusters within the 152
  // SMs when the problems are many
  int c = std::min(std::min(16, std::max(cmax, 1)), std::max(1, (maxp + 15) / 16));
  if (ntasks > 0) c = std::min(c, std::max(1, 152 / ntasks));
  return std::max(c, min_cluster(maxp));
}

cudaError_t osj_eig_cluster(const EigTask* d_tasks, int ntasks, int maxp, int csize, void* d_scratch, int* d_status,
                            cudaStream_t s, int* csize_used) {
  if (ntasks <= 0) return cudaSuccess;
  if (maxp > osj_max_order()) return cudaErrorInvalidValue;
  const int64_t per = osj_cluster_scratch(maxp);
  cudaError_t e = cudaMemsetAsync(d_scratch, 0, (size_t)per * ntasks, s);
  if (e != cudaSuccess) return e;
  csize = std::max(min_cluster(maxp), std::min(16, csize));
  const size_t smem = smem_bytes(maxp, csize);
  e = cudaFuncSetAttribute(k_osj_cl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (csize > 8) {
    cudaFuncSetAttribute(k_osj_cl, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
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
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_osj_cl, &q) != cudaSuccess || nclusters < 1) {
      cudaGetLastError();
      return cudaErrorInvalidConfiguration;
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
  e = cudaLaunchKernelEx(&cfg, k_osj_cl, d_tasks, (unsigned char*)d_scratch, per, d_status);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace h2k
