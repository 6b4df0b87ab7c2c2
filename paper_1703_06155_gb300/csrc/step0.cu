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
// basis with GEMMs.
//
// FP64 runs at 2 FMA per clock per SM on this GPU, so one problem is spread
// over a thread-block cluster of C CTAs (C = 1 .. 16, chosen per launch):
//   * pivoted Cholesky: rows are split in contiguous blocks over the CTAs;
//     per pivot step each CTA forms its rows of the new column (left-looking,
//     the k-sum split over several threads per row), updates its diagonal
//     residuals and publishes its local pivot candidate and remaining trace;
//     after one cluster barrier every CTA reduces the candidates read through
//     distributed shared memory, so all take the same decisions;
//   * Householder QR: columns are dealt round-robin; per column one cluster
//     barrier (the owner of column j+1 applies reflector j to it first, then
//     forms reflector j+1 before the barrier);
//   * compact WY: W = Y^H Y by column owners, then the rows of T
//     (T(i,j) = -tau_j sum_k T(i,k) W(k,j)) are independent and split over
//     the CTAs.
// Barriers are hardware cluster barriers with release / acquire semantics;
// every loop is bounded by p.
#include <cooperative_groups.h>

#include <algorithm>

#include "dfloat.cuh"
#include "h2_kernels.h"

namespace cg = cooperative_groups;
namespace D = h2k::dfl;

namespace h2k {
namespace {

constexpr int NT = 256;
constexpr int PMAX = 1024;

// cluster-wide barrier: arrive with release, wait with acquire (cluster scope;
// orders the global and distributed-shared-memory traffic of the cluster)
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// CTA-wide sum (all threads call; result to all)
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

// better candidate: larger value, ties -> lower row
__device__ __forceinline__ bool better(double v, int i, double bv, int bi) { return v > bv || (v == bv && i < bi); }

__global__ void __launch_bounds__(NT) k_pchol_wy_cl(const PcholTask* __restrict__ tasks, int lrow_smem) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const PcholTask t = tasks[blockIdx.x / C];
  const int p = t.p;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = NT / 32;
  __shared__ double red[32];
  __shared__ double dl[PMAX];            // diagonal residuals of the own rows
  __shared__ unsigned char used[PMAX];   // own rows already pivoted
  __shared__ __align__(16) cd prow[PMAX];  // pivot row L[pc, 0:j]
  __shared__ double cand_v[2], cand_t[2];
  __shared__ int cand_i[2];
  __shared__ double wv[NT / 32];
  __shared__ int wi[NT / 32];
  cd* G = t.G;
  cd* L = t.L;  // p x p (ld p); becomes Y
  // the own rows of L during the pivoted Cholesky: row-major in shared memory
  // (ld = rmax) when they fit (lrow_smem), else in place in L
  extern __shared__ __align__(16) unsigned char lsm[];
  cd* Ls = reinterpret_cast<cd*>(lsm);
  // own rows: a contiguous block
  const int rb = (p + C - 1) / C;
  const int r0 = min(p, rank * rb), r1 = min(p, r0 + rb), nr = r1 - r0;
  // nu^2 = snorm2 + trace(M)
  const double thr = t.eps2 * (t.snorm2 + *t.trM);
  const double tau = thr / 10.0;  // bound on the trace of the remainder
  const int rmax = p < PMAX ? p : PMAX;
  for (int i = tid; i < nr; i += NT) {
    dl[i] = G[(r0 + i) + (size_t)(r0 + i) * p].re;
    used[i] = 0;
  }
  // element (li, k) of the own rows
  const size_t ls_r = lrow_smem ? (size_t)rmax : 1, ls_k = lrow_smem ? 1 : (size_t)p;
  cd* Lo = lrow_smem ? Ls : L + r0;
  for (int idx = tid; idx < nr * rmax; idx += NT) {
    const int li = idx % nr, k = idx / nr;
    Lo[li * ls_r + k * ls_k].re = 0;
    Lo[li * ls_r + k * ls_k].im = 0;
  }
  __syncthreads();
  // threads per row for the left-looking k-sums
  int tpr = 1;
  while (tpr < 32 && tpr * 2 * max(nr, 1) <= NT) tpr *= 2;

  // local candidate + remaining trace -> slot s
  auto publish = [&](int s) {
    double bv = -1, ts = 0;
    int bi = 0x7fffffff;
    for (int i = tid; i < nr; i += NT) {
      if (used[i]) continue;
      const double v = dl[i];
      ts += v > 0 ? v : 0;
      if (better(v, r0 + i, bv, bi)) { bv = v; bi = r0 + i; }
    }
    // block argmax (warp shuffles, then warp 0)
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, bv, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (better(ov, oi, bv, bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { wv[warp] = bv; wi[warp] = bi; }
    ts = bsum(ts, red);  // contains __syncthreads
    if (tid < 32) {
      bv = lane < nw ? wv[lane] : -1.0;
      bi = lane < nw ? wi[lane] : 0x7fffffff;
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, bv, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (better(ov, oi, bv, bi)) { bv = ov; bi = oi; }
      }
      if (tid == 0) { cand_v[s] = bv; cand_i[s] = bi; cand_t[s] = ts; }
    }
  };
  // reduce the C published candidates of slot s (all CTAs get the same):
  // lane q of warp 0 reads candidate q through distributed shared memory
  // (one remote read per candidate and CTA), a warp reduction (the argmax
  // rule is order-free: larger value, ties -> lower row; the trace sum runs
  // in a fixed tree order), then the result to the CTA through shared memory
  __shared__ double g_dv, g_trs;
  __shared__ int g_pc;
  auto gather = [&](int s, double& dv, int& pc, double& trs) {
    if (warp == 0) {
      dv = -1;
      pc = 0x7fffffff;
      trs = 0;
      if (lane < C) {
        dv = *cl.map_shared_rank(&cand_v[s], lane);
        pc = *cl.map_shared_rank(&cand_i[s], lane);
        trs = *cl.map_shared_rank(&cand_t[s], lane);
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, dv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, pc, o);
        trs += __shfl_xor_sync(0xffffffffu, trs, o);
        if (better(ov, oi, dv, pc)) { dv = ov; pc = oi; }
      }
      if (lane == 0) {
        g_dv = dv;
        g_pc = pc;
        g_trs = trs;
      }
    }
    __syncthreads();
    dv = g_dv;
    pc = g_pc;
    trs = g_trs;
  };

  // ---------------------------------------------------- pivoted Cholesky
  publish(0);
  cluster_barrier();
  int r = 0;
  for (int j = 0; j < rmax; ++j) {
    double dv, trs;
    int pc;
    gather(j & 1, dv, pc, trs);
    if (!(trs > tau) || !(dv > 0.0)) break;
    const double sd = sqrt(dv);
    // pivot row entries L[pc, 0:j] (written by its owner in earlier steps;
    // read from the owner's shared memory when the rows live there)
    if (lrow_smem) {
      const int owner = pc / rb, lpc = pc - owner * rb;
      const cd* src = cl.map_shared_rank(Ls, owner) + (size_t)lpc * rmax;
      for (int k = tid; k < j; k += NT) prow[k] = src[k];
    } else {
      for (int k = tid; k < j; k += NT) prow[k] = L[pc + (size_t)k * p];
    }
    __syncthreads();
    // column j for the own rows not yet pivoted (the pivot row gives sd)
    const int rows_per_pass = NT / tpr;
    for (int base = 0; base < nr; base += rows_per_pass) {
      const int li = base + tid / tpr, sub = tid % tpr;
      const bool act = li < nr && !used[li];
      const int i = r0 + li;
      double vr = 0, vi = 0;
      if (act)
        for (int k = sub; k < j; k += tpr) {
          const cd a = Lo[li * ls_r + k * ls_k], b = prow[k];  // a * conj(b)
          vr += a.re * b.re + a.im * b.im;
          vi += a.im * b.re - a.re * b.im;
        }
      for (int o = tpr / 2; o > 0; o >>= 1) {
        vr += __shfl_xor_sync(0xffffffffu, vr, o);
        vi += __shfl_xor_sync(0xffffffffu, vi, o);
      }
      if (act && sub == 0) {
        cd z;
        z.re = (G[i + (size_t)pc * p].re - vr) / sd;
        z.im = (G[i + (size_t)pc * p].im - vi) / sd;
        Lo[li * ls_r + j * ls_k] = z;
        if (i == pc) {
          used[li] = 1;
        } else {
          dl[li] -= z.re * z.re + z.im * z.im;
        }
      }
    }
    __syncthreads();
    publish((j + 1) & 1);
    cluster_barrier();
    r = j + 1;
  }

  if (lrow_smem) {
    // own rows to the column-major L for the QR (columns 0:r)
    for (int idx = tid; idx < nr * r; idx += NT) {
      const int li = idx % nr, k = idx / nr;
      L[(r0 + li) + (size_t)k * p] = Ls[li * (size_t)rmax + k];
    }
    cluster_barrier();
  }
  // ---------------------------------------- Householder QR of L(:, 0:r)
  cd* T = t.T;  // r x r (ld r): tau_j on the diagonal while the QR runs
  cd* W = t.W;
  if (t.dfqr) {
    // The QR in double-float on the FP32 pipe.  L's entries are of the order
    // of the square roots of G's: the directions at the truncation threshold
    // have singular values near eps ||L||, which double-float's ~48 bits
    // carry to ~1e-9 relative at eps = 1e-6, while Q stays unitary to ~1e-13.
    // The columns are held as {re.h, re.l, im.h, im.l} in L's own storage.
    float4* Lf = reinterpret_cast<float4*>(L);
    float4* vsf = reinterpret_cast<float4*>(prow);  // reflector j (pivot-row buffer, free now)
    __shared__ float2 redf[NT / 32];
    auto bsum_df = [&](D::df v) {
      v = D::wsum(v);
      __syncthreads();
      if (lane == 0) redf[warp] = make_float2(v.h, v.l);
      __syncthreads();
      D::df s = {0.0f, 0.0f};
      for (int w = 0; w < nw; ++w) s = D::dadd(s, D::df{redf[w].x, redf[w].y});
      __syncthreads();
      return s;
    };
    // power-of-two scaling to max |L| in [0.5, 1) (Q, Y and T do not change;
    // R is scaled back): with diagonal pivoting |L(i, j)| <= L(p_0, 0), the
    // largest entry of column 0, which every CTA reads
    double mx = 0;
    if (r > 0)
      for (int i = tid; i < p; i += NT) {
        const cd v = L[i];
        mx = fmax(mx, fmax(fabs(v.re), fabs(v.im)));
      }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    mx = 0;
    for (int w = 0; w < nw; ++w) mx = fmax(mx, red[w]);
    int ex = 0;
    if (mx > 0) frexp(mx, &ex);
    cluster_barrier();  // column 0 read by all before its owner converts it
    for (int c = rank; c < r; c += C)
      for (int i = tid; i < p; i += NT) {
        const cd v = L[i + (size_t)c * p];
        Lf[i + (size_t)c * p] = D::pack(D::dsplit(ldexp(v.re, -ex)), D::dsplit(ldexp(v.im, -ex)));
      }
    __syncthreads();
    auto reflector_df = [&](int j) {
      D::df s = {0.0f, 0.0f};
      for (int i = j + 1 + tid; i < p; i += NT) {
        const float4 v = Lf[i + (size_t)j * p];
        s = D::dfma(D::re_of(v), D::re_of(v), s);
        s = D::dfma(D::im_of(v), D::im_of(v), s);
      }
      s = bsum_df(s);
      const float4 alv = Lf[j + (size_t)j * p];
      const D::df ar = D::re_of(alv), ai = D::im_of(alv);
      D::df tr = {0.0f, 0.0f}, ti = {0.0f, 0.0f};
      // R(j, j) (unscaled): beta of the reflection, or the entry itself when none is needed
      double rjj = ldexp(D::djoin(ar), ex);
      if (!(s.h == 0.0f && ai.h == 0.0f)) {
        const D::df nrm = D::dsqrt(D::dfma(ar, ar, D::dfma(ai, ai, s)));
        const D::df beta = ar.h >= 0.0f ? D::dneg(nrm) : nrm;
        rjj = ldexp(D::djoin(beta), ex);
        const D::df ib = D::drcp(beta);
        tr = D::dmul(D::dsub(beta, ar), ib);  // tau = (beta - alpha) / beta
        ti = D::dneg(D::dmul(ai, ib));
        // v = x / (alpha - beta) = x conj(d) / |d|^2, d = alpha - beta
        const D::df dr = D::dsub(ar, beta), di = ai;
        const D::df idd = D::drcp(D::dfma(dr, dr, D::dmul(di, di)));
        const D::df scr = D::dmul(dr, idd), sci = D::dneg(D::dmul(di, idd));
        for (int i = j + 1 + tid; i < p; i += NT) {
          const float4 v = Lf[i + (size_t)j * p];
          const D::df vr = D::re_of(v), vi = D::im_of(v);
          Lf[i + (size_t)j * p] =
              D::pack(D::dfma(vr, scr, D::dneg(D::dmul(vi, sci))), D::dfma(vr, sci, D::dmul(vi, scr)));
        }
      }
      if (tid == 0) {
        T[j + (size_t)j * r].re = D::djoin(tr);
        T[j + (size_t)j * r].im = D::djoin(ti);
        if (t.R) {
          t.R[j + (size_t)j * r].re = rjj;
          t.R[j + (size_t)j * r].im = 0;
        }
      }
    };
    // apply H_j^H to column c (one warp): w -= v conj(tau) (v^H w); up to 32 WRD
    // entries of the column stay in registers between the two passes
    constexpr int WRD = 12;
    auto apply_col_df = [&](int j, int c, D::df tr, D::df ti) {
      D::df dr = {0.0f, 0.0f}, di = {0.0f, 0.0f};
      float4* col = Lf + (size_t)c * p;
      if (p - j <= 32 * WRD) {
        float4 w[WRD];
#pragma unroll
        for (int u = 0; u < WRD; ++u) {
          const int i = j + lane + 32 * u;
          if (i < p) w[u] = col[i];
        }
#pragma unroll
        for (int u = 0; u < WRD; ++u) {
          const int i = j + lane + 32 * u;
          if (i < p) {
            const float4 v = vsf[i];
            dr = D::dfma(D::re_of(v), D::re_of(w[u]), dr);
            dr = D::dfma(D::im_of(v), D::im_of(w[u]), dr);
            di = D::dfma(D::re_of(v), D::im_of(w[u]), di);
            di = D::dfma(D::dneg(D::im_of(v)), D::re_of(w[u]), di);
          }
        }
        dr = D::wsum(dr);
        di = D::wsum(di);
        const D::df fr = D::dfma(tr, dr, D::dmul(ti, di)), fi = D::dfma(tr, di, D::dneg(D::dmul(ti, dr)));
#pragma unroll
        for (int u = 0; u < WRD; ++u) {
          const int i = j + lane + 32 * u;
          if (i < p) {
            const float4 v = vsf[i];
            const D::df vr = D::re_of(v), vi = D::im_of(v);
            const D::df nr = D::dsub(D::re_of(w[u]), D::dfma(vr, fr, D::dneg(D::dmul(vi, fi))));
            const D::df ni = D::dsub(D::im_of(w[u]), D::dfma(vr, fi, D::dmul(vi, fr)));
            col[i] = D::pack(nr, ni);
          }
        }
        return;
      }
      for (int i = j + lane; i < p; i += 32) {
        const float4 v = vsf[i], x = col[i];
        dr = D::dfma(D::re_of(v), D::re_of(x), dr);
        dr = D::dfma(D::im_of(v), D::im_of(x), dr);
        di = D::dfma(D::re_of(v), D::im_of(x), di);
        di = D::dfma(D::dneg(D::im_of(v)), D::re_of(x), di);
      }
      dr = D::wsum(dr);
      di = D::wsum(di);
      const D::df fr = D::dfma(tr, dr, D::dmul(ti, di)), fi = D::dfma(tr, di, D::dneg(D::dmul(ti, dr)));
      for (int i = j + lane; i < p; i += 32) {
        const float4 v = vsf[i], x = col[i];
        const D::df vr = D::re_of(v), vi = D::im_of(v);
        const D::df nr = D::dsub(D::re_of(x), D::dfma(vr, fr, D::dneg(D::dmul(vi, fi))));
        const D::df ni = D::dsub(D::im_of(x), D::dfma(vr, fi, D::dmul(vi, fr)));
        col[i] = D::pack(nr, ni);
      }
    };
    if (r > 0) {
      if (rank == 0) reflector_df(0);
      cluster_barrier();
    }
    for (int j = 0; j < r; ++j) {
      const D::df tr = D::dsplit(T[j + (size_t)j * r].re), ti = D::dsplit(T[j + (size_t)j * r].im);
      for (int i = j + tid; i < p; i += NT) vsf[i] = (i == j) ? make_float4(1.0f, 0.0f, 0.0f, 0.0f) : Lf[i + (size_t)j * p];
      __syncthreads();
      if (!(tr.h == 0.0f && ti.h == 0.0f)) {
        int first = j + 1 + ((rank - (j + 1)) % C + C) % C;
        for (int c = first + warp * C; c < r; c += nw * C) apply_col_df(j, c, tr, ti);
      }
      __syncthreads();
      if (j + 1 < r && (j + 1) % C == rank) reflector_df(j + 1);
      cluster_barrier();
    }
    // strict upper triangle of R, and W(k, c) = Y(:, k)^H Y(:, c) for k < c
    // (Y unit lower trapezoidal: Y(c, c) = 1, Y(i, c) = 0 for i < c), by
    // column owners, summed in double-float
    for (int c = rank; c < r; c += C) {
      if (t.R)
        for (int i = tid; i < c; i += NT) {
          const float4 v = Lf[i + (size_t)c * p];
          t.R[i + (size_t)c * r].re = ldexp(D::djoin(D::re_of(v)), ex);
          t.R[i + (size_t)c * r].im = ldexp(D::djoin(D::im_of(v)), ex);
        }
      for (int k = warp; k < c; k += nw) {
        D::df sr = {0.0f, 0.0f}, si = {0.0f, 0.0f};
        for (int i = c + lane; i < p; i += 32) {
          const float4 a = Lf[i + (size_t)k * p];
          if (i == c) {
            sr = D::dadd(sr, D::re_of(a));
            si = D::dsub(si, D::im_of(a));
          } else {
            const float4 bv = Lf[i + (size_t)c * p];
            sr = D::dfma(D::re_of(a), D::re_of(bv), sr);
            sr = D::dfma(D::im_of(a), D::im_of(bv), sr);
            si = D::dfma(D::re_of(a), D::im_of(bv), si);
            si = D::dfma(D::dneg(D::im_of(a)), D::re_of(bv), si);
          }
        }
        sr = D::wsum(sr);
        si = D::wsum(si);
        if (lane == 0) {
          W[k + (size_t)c * r].re = D::djoin(sr);
          W[k + (size_t)c * r].im = D::djoin(si);
        }
      }
    }
    cluster_barrier();
    // own columns back to complex128: Y
    for (int c = rank; c < r; c += C)
      for (int i = tid; i < p; i += NT) {
        cd y;
        if (i < c) {
          y.re = 0;
          y.im = 0;
        } else if (i == c) {
          y.re = 1;
          y.im = 0;
        } else {
          const float4 v = Lf[i + (size_t)c * p];
          y.re = D::djoin(D::re_of(v));
          y.im = D::djoin(D::im_of(v));
        }
        L[i + (size_t)c * p] = y;
      }
  } else {
    auto reflector = [&](int j) {
      double s = 0;
      for (int i = j + 1 + tid; i < p; i += NT) {
        const cd v = L[i + (size_t)j * p];
        s += v.re * v.re + v.im * v.im;
      }
      s = bsum(s, red);
      const cd al = L[j + (size_t)j * p];
      double tr_ = 0, ti_ = 0;
      double rjj = al.re;  // R(j, j): beta of the reflection, or the entry itself when none is needed
      if (!(s == 0.0 && al.im == 0.0)) {
        const double nrm = sqrt(al.re * al.re + al.im * al.im + s);
        const double beta = al.re >= 0 ? -nrm : nrm;
        rjj = beta;
        tr_ = (beta - al.re) / beta;
        ti_ = -al.im / beta;
        const double dr = al.re - beta, di = al.im, dd = dr * dr + di * di;
        const double scr = dr / dd, sci = -di / dd;
        for (int i = j + 1 + tid; i < p; i += NT) {
          cd v = L[i + (size_t)j * p];
          const double vr = v.re * scr - v.im * sci, vi = v.re * sci + v.im * scr;
          v.re = vr;
          v.im = vi;
          L[i + (size_t)j * p] = v;
        }
      }
      if (tid == 0) {
        T[j + (size_t)j * r].re = tr_;
        T[j + (size_t)j * r].im = ti_;
        if (t.R) {
          t.R[j + (size_t)j * r].re = rjj;
          t.R[j + (size_t)j * r].im = 0;
        }
      }
    };
    // apply H_j^H to column c (one warp); vs = reflector j in shared memory
    // (vs[j] = 1).  A column of up to 32 WR entries stays in registers between
    // the dot product and the update, its loads all in flight together.
    constexpr int WR = 12;
    cd* vs = prow;  // the pivot-row buffer is free after the Cholesky
    auto apply_col = [&](int j, int c, double tr_, double ti_) {
      double dr = 0, di = 0;
      if (p - j <= 32 * WR) {
        cd w[WR];
  #pragma unroll
        for (int u = 0; u < WR; ++u) {
          const int i = j + lane + 32 * u;
          if (i < p) w[u] = L[i + (size_t)c * p];
        }
  #pragma unroll
        for (int u = 0; u < WR; ++u) {
          const int i = j + lane + 32 * u;
          if (i < p) {
            const cd v = vs[i];
            dr += v.re * w[u].re + v.im * w[u].im;
            di += v.re * w[u].im - v.im * w[u].re;
          }
        }
        dr = wsum(dr);
        di = wsum(di);
        const double fr = tr_ * dr + ti_ * di, fi = tr_ * di - ti_ * dr;  // conj(tau) d
  #pragma unroll
        for (int u = 0; u < WR; ++u) {
          const int i = j + lane + 32 * u;
          if (i < p) {
            const cd v = vs[i];
            w[u].re -= v.re * fr - v.im * fi;
            w[u].im -= v.re * fi + v.im * fr;
            L[i + (size_t)c * p] = w[u];
          }
        }
        return;
      }
      for (int i = j + lane; i < p; i += 32) {
        const cd w = L[i + (size_t)c * p];
        const cd v = vs[i];
        dr += v.re * w.re + v.im * w.im;
        di += v.re * w.im - v.im * w.re;
      }
      dr = wsum(dr);
      di = wsum(di);
      const double fr = tr_ * dr + ti_ * di, fi = tr_ * di - ti_ * dr;  // conj(tau) d
      for (int i = j + lane; i < p; i += 32) {
        const cd v = vs[i];
        cd w = L[i + (size_t)c * p];
        w.re -= v.re * fr - v.im * fi;
        w.im -= v.re * fi + v.im * fr;
        L[i + (size_t)c * p] = w;
      }
    };
    if (r > 0) {
      if (rank == 0) reflector(0);
      cluster_barrier();
    }
    for (int j = 0; j < r; ++j) {
      const double tr_ = T[j + (size_t)j * r].re, ti_ = T[j + (size_t)j * r].im;
      // reflector j (written by its owner before the last cluster barrier) to shared memory
      for (int i = j + tid; i < p; i += NT) {
        if (i == j) {
          vs[i].re = 1;
          vs[i].im = 0;
        } else {
          vs[i] = L[i + (size_t)j * p];
        }
      }
      __syncthreads();
      if (!(tr_ == 0.0 && ti_ == 0.0)) {
        // own columns c > j, c = rank (mod C)
        int first = j + 1 + ((rank - (j + 1)) % C + C) % C;
        for (int c = first + warp * C; c < r; c += nw * C) apply_col(j, c, tr_, ti_);
      }
      __syncthreads();
      if (j + 1 < r && (j + 1) % C == rank) reflector(j + 1);
      cluster_barrier();
    }
    // Y: unit lower trapezoidal reflectors (upper part zeroed, v_0 = 1), own
    // columns; the strict upper triangle of R is saved first when asked for
    for (int c = rank; c < r; c += C)
      for (int i = tid; i <= c && i < p; i += NT) {
        if (t.R && i < c) t.R[i + (size_t)c * r] = L[i + (size_t)c * p];
        L[i + (size_t)c * p].re = (i == c) ? 1 : 0;
        L[i + (size_t)c * p].im = 0;
      }
    cluster_barrier();

    // ------------------------------------------------------- compact WY T
    // W(k, j) = Y(:, k)^H Y(:, j), k < j, into the scratch (ld r), by column owners
    for (int c = rank; c < r; c += C)
      for (int k = warp; k < c; k += nw) {
        double sr = 0, si = 0;
        for (int i = c + lane; i < p; i += 32) {  // Y(i, c) = 0 for i < c
          const cd a = L[i + (size_t)k * p], b = L[i + (size_t)c * p];
          sr += a.re * b.re + a.im * b.im;
          si += a.re * b.im - a.im * b.re;
        }
        sr = wsum(sr);
        si = wsum(si);
        if (lane == 0) { W[k + (size_t)c * r].re = sr; W[k + (size_t)c * r].im = si; }
      }
    cluster_barrier();
  }
  // rows of T: T(i, i) = tau_i, T(i, j) = -tau_j sum_{k=i}^{j-1} T(i, k) W(k, j);
  // one warp per own row (rows i = rank mod C), strictly lower part zeroed
  for (int i = rank + warp * C; i < r; i += nw * C) {
    for (int k = lane; k < i; k += 32) {
      T[i + (size_t)k * r].re = 0;
      T[i + (size_t)k * r].im = 0;
    }
    for (int j = i + 1; j < r; ++j) {
      double sr = 0, si = 0;
      for (int k = i + lane; k < j; k += 32) {
        const cd a = T[i + (size_t)k * r], w = W[k + (size_t)j * r];
        sr += a.re * w.re - a.im * w.im;
        si += a.re * w.im + a.im * w.re;
      }
      sr = wsum(sr);
      si = wsum(si);
      const double tr2 = T[j + (size_t)j * r].re, ti2 = T[j + (size_t)j * r].im;
      if (lane == 0) {
        T[i + (size_t)j * r].re = -(tr2 * sr - ti2 * si);
        T[i + (size_t)j * r].im = -(tr2 * si + ti2 * sr);
      }
      __syncwarp();
    }
  }
  if (rank == 0 && tid == 0) *t.rout = r;
}

}  // namespace

cudaError_t pchol_wy(const PcholTask* d, int n, int maxp, int cmax, cudaStream_t s, int* csize_used) {
  if (n <= 0) return cudaSuccess;
  if (maxp > PMAX) return cudaErrorInvalidValue;
  // CTAs per problem: spread few problems over the SMs, keep >= 16 rows each
  int csize = std::max(1, std::min(std::min(16, cmax), std::min(152 / n, maxp / 16)));
  if (csize > 8) {
    cudaFuncSetAttribute(k_pchol_wy_cl, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
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
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_pchol_wy_cl, &q) != cudaSuccess || nclusters < 1) {
      cudaGetLastError();
      csize = 8;
    }
  }
  // own rows of L in shared memory when they fit
  const int rb = (maxp + csize - 1) / csize, rmax = maxp < PMAX ? maxp : PMAX;
  const size_t lbytes = (size_t)rb * rmax * sizeof(cd);
  const int lrow_smem = lbytes <= 180 * 1024 ? 1 : 0;
  const size_t dyn = lrow_smem ? lbytes : 0;
  if (dyn > 0) cudaFuncSetAttribute(k_pchol_wy_cl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n * csize, 1, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (csize_used) *csize_used = csize;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_pchol_wy_cl, d, lrow_smem);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace h2k
