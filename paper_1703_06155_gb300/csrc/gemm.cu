// Batched variable-size complex sum-GEMM:  C = alpha * sum_p op(A_p) op(B_p) + beta * C
//
// One CTA computes one BM x BN tile of one task.  The host lists the tiles,
// so a single launch covers every product of a colour class (Schur updates
// grouped by target block, Step-0 Grams, H^2 matvec stages ...).  Operands
// are staged through shared memory as split real / imaginary planes; each
// thread owns a 4 x 4 complex micro-tile (rows ty + 16 i, columns tx + 16 j),
// which keeps the shared-memory reads conflict-free.
#include "h2_kernels.h"

namespace h2k {
namespace {

template <class E> struct RealOf;
template <> struct RealOf<cd> { using T = double; };
template <> struct RealOf<cf> { using T = float; };

template <class E, class R>
__device__ __forceinline__ void load_op(const E* base, int ld, int op, int r, int c, R& re, R& im) {
  // element (r, c) of op(X)
  const E v = (op == OP_N || op == OP_C) ? base[(size_t)r + (size_t)c * ld] : base[(size_t)c + (size_t)r * ld];
  re = (R)v.re;
  im = (op == OP_C || op == OP_H) ? -(R)v.im : (R)v.im;
}

template <class E, class R>
__device__ __forceinline__ void store_val(E* p, R re, R im) {
  E v;
  v.re = (decltype(v.re))re;
  v.im = (decltype(v.im))im;
  *p = v;
}

constexpr int BK = 8, NT = 256;

template <class R> struct CxOf;
template <> struct CxOf<double> { using T = cd; };
template <> struct CxOf<float> { using T = cf; };

// Tile BM x BN with BM in {16, 32, 64}, BN in {16, 32, 64}: each thread owns a
// (BM / 16) x (BN / 16) complex micro-tile.  Narrow tiles serve the
// right-hand-side products of the solve and the matvec and the small
// complement-side Grams of Step 0, where 64 x 64 tiles would mostly compute
// padding.
template <class EA, class EB, class R, class EO, int BM, int BN>
__global__ void __launch_bounds__(NT) k_gemm(const GemmTask* __restrict__ tasks,
                                            const GemmPair* __restrict__ pairs,
                                            const GemmTile* __restrict__ tiles,
                                            typename CxOf<R>::T* __restrict__ ws) {
  constexpr int TX = BN >= 16 ? 16 : BN, TY = NT / TX, TN = BN / TX, TMR = BM / TY;
  static_assert(BN % TX == 0 && BM % TY == 0, "tile shape");
  __shared__ R As_r[BK][BM], As_i[BK][BM];
  __shared__ R Bs_r[BK][BN], Bs_i[BK][BN];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmTask tk = tasks[tl.task];
  const int m0 = tl.tm * BM, n0 = tl.tn * BN;
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  R acc_r[TMR][TN], acc_i[TMR][TN];
#pragma unroll
  for (int i = 0; i < TMR; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc_r[i][j] = acc_i[i][j] = (R)0;

  // this tile's share of the concatenated K range of all pairs
  const int64_t klo = tk.nk > 1 ? (int64_t)tl.kc * tk.ksz : 0;
  const int64_t khi = tk.nk > 1 ? klo + tk.ksz : ((int64_t)1 << 62);
  int64_t koff = 0;
  for (int pi = tk.p0; pi < tk.p0 + tk.np; ++pi) {
    const GemmPair pr = pairs[pi];
    const int64_t kb = koff;
    koff += pr.K;
    if (koff <= klo || kb >= khi) continue;
    const int kbeg = (int)(klo > kb ? klo - kb : 0);
    const int kend = (int)(khi - kb < pr.K ? khi - kb : pr.K);
    const EA* A = (const EA*)pr.A;
    const EB* B = (const EB*)pr.B;
    const bool at = (pr.opA == OP_T || pr.opA == OP_H);
    const bool bt = (pr.opB == OP_T || pr.opB == OP_H);
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
      // A tile: BM x BK of op(A)
#pragma unroll
      for (int r = 0; r < (BM * BK + NT - 1) / NT; ++r) {
        const int l = tid + r * NT;
        if (l >= BM * BK) break;
        int i, k;
        if (!at) { i = l % BM; k = l / BM; } else { k = l % BK; i = l / BK; }
        R re = 0, im = 0;
        if (m0 + i < tk.M && k0 + k < kend) load_op<EA, R>(A, pr.lda, pr.opA, m0 + i, k0 + k, re, im);
        As_r[k][i] = re;
        As_i[k][i] = im;
      }
      // B tile: BK x BN of op(B)
#pragma unroll
      for (int r = 0; r < (BK * BN + NT - 1) / NT; ++r) {
        const int l = tid + r * NT;
        if (l >= BK * BN) break;
        int k, j;
        if (!bt) { k = l % BK; j = l / BK; } else { j = l % BN; k = l / BN; }
        R re = 0, im = 0;
        if (n0 + j < tk.N && k0 + k < kend) load_op<EB, R>(B, pr.ldb, pr.opB, k0 + k, n0 + j, re, im);
        Bs_r[k][j] = re;
        Bs_i[k][j] = im;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < BK; ++k) {
        R ar[TMR], ai[TMR], br[TN], bi[TN];
#pragma unroll
        for (int i = 0; i < TMR; ++i) { ar[i] = As_r[k][ty + TY * i]; ai[i] = As_i[k][ty + TY * i]; }
#pragma unroll
        for (int j = 0; j < TN; ++j) { br[j] = Bs_r[k][tx + TX * j]; bi[j] = Bs_i[k][tx + TX * j]; }
#pragma unroll
        for (int i = 0; i < TMR; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) {
            acc_r[i][j] = fma(ar[i], br[j], fma(-ai[i], bi[j], acc_r[i][j]));
            acc_i[i][j] = fma(ar[i], bi[j], fma(ai[i], br[j], acc_i[i][j]));
          }
      }
      __syncthreads();
    }
  }
  if (tk.nk > 1) {
    // partial sums of this chunk, unscaled
    typename CxOf<R>::T* W = ws + tk.ws_off + (int64_t)tl.kc * tk.M * tk.N;
#pragma unroll
    for (int i = 0; i < TMR; ++i) {
      const int m = m0 + ty + TY * i;
      if (m >= tk.M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int n = n0 + tx + TX * j;
        if (n >= tk.N) continue;
        typename CxOf<R>::T v;
        v.re = acc_r[i][j];
        v.im = acc_i[i][j];
        W[(int64_t)m + (int64_t)n * tk.M] = v;
      }
    }
    return;
  }
  EO* C = (EO*)tk.C;
  const R al = (R)tk.alpha, be = (R)tk.beta;
#pragma unroll
  for (int i = 0; i < TMR; ++i) {
    const int m = m0 + ty + TY * i;
    if (m >= tk.M) continue;
    // a row's C values in flight together, then the updates
    EO old[TN];
    if (tk.beta != 0.0) {
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int n = n0 + tx + TX * j;
        if (n < tk.N) old[j] = C[(size_t)m + (size_t)n * tk.ldc];
      }
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int n = n0 + tx + TX * j;
      if (n >= tk.N) continue;
      R re = al * acc_r[i][j], im = al * acc_i[i][j];
      if (tk.beta != 0.0) {
        re = fma(be, (R)old[j].re, re);
        im = fma(be, (R)old[j].im, im);
      }
      store_val<EO, R>(C + (size_t)m + (size_t)n * tk.ldc, re, im);
    }
  }
}

// ---- complex64 products accumulated to FP64 accuracy on the FP32 pipe ----
//
// For the Step-0 Grams of complex64 operands.  A product a b of two FP32
// numbers is exact as p + e with p = fl(a b) and e = fma(a, b, -p).  The
// products of one BK-long K slice are summed in double-float: hi takes p
// through an error-free TwoSum and lo collects the TwoSum errors and the e
// parts; the slice totals hi + lo (error <= ~4 BK 2^-48 of the slice's
// magnitude) are summed in a double-float chunk accumulator (TwoSum, as
// dd_acc below), which is added to an FP64 accumulator every kDfFlush
// slices (FP64 adds run at 1/64 of the FP32 rate here: one per slice would
// cost as much as the slice's products).  About ten FP32 operations replace
// one FP64 FMA, on a pipe that runs 64x the FP64 rate here.  The
// rounded operations are the _rn intrinsics, which the compiler never fuses
// into FMAs.  (Operands below ~1e-19 in magnitude would lose the exactness of
// their products to FP32 underflow; Gram operands are far above that.)
constexpr int kDfFlush = 8;

// (H, L) += (h, l) in double-float
__device__ __forceinline__ void dd_acc(float& H, float& L, float h, float l) {
  const float s = __fadd_rn(H, h);
  const float bb = __fsub_rn(s, H);
  const float t = __fadd_rn(__fsub_rn(H, __fsub_rn(s, bb)), __fsub_rn(h, bb));
  const float lo = __fadd_rn(__fadd_rn(L, l), t);
  H = __fadd_rn(s, lo);
  L = __fsub_rn(lo, __fsub_rn(H, s));
}

__device__ __forceinline__ void df_madd(float& h, float& l, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = fmaf(a, b, -p);
  const float s = __fadd_rn(h, p);
  const float bb = __fsub_rn(s, h);
  const float t = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  h = s;
  l = __fadd_rn(l, __fadd_rn(t, e));
}

template <int BM, int BN>
__global__ void __launch_bounds__(NT) k_gemm_df(const GemmTask* __restrict__ tasks,
                                               const GemmPair* __restrict__ pairs,
                                               const GemmTile* __restrict__ tiles, cd* __restrict__ ws) {
  constexpr int TX = BN >= 16 ? 16 : BN, TY = NT / TX, TN = BN / TX, TMR = BM / TY;
  static_assert(BN % TX == 0 && BM % TY == 0, "tile shape");
  __shared__ float As_r[BK][BM], As_i[BK][BM];
  __shared__ float Bs_r[BK][BN], Bs_i[BK][BN];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmTask tk = tasks[tl.task];
  const int m0 = tl.tm * BM, n0 = tl.tn * BN;
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  double acc_r[TMR][TN], acc_i[TMR][TN];
  float Hr[TMR][TN], Lr[TMR][TN], Hi[TMR][TN], Li[TMR][TN];  // chunk accumulators
#pragma unroll
  for (int i = 0; i < TMR; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      acc_r[i][j] = acc_i[i][j] = 0.0;
      Hr[i][j] = Lr[i][j] = Hi[i][j] = Li[i][j] = 0.f;
    }
  int nsl = 0;
  auto flush = [&]() {
#pragma unroll
    for (int i = 0; i < TMR; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        acc_r[i][j] += (double)Hr[i][j] + (double)Lr[i][j];
        acc_i[i][j] += (double)Hi[i][j] + (double)Li[i][j];
        Hr[i][j] = Lr[i][j] = Hi[i][j] = Li[i][j] = 0.f;
      }
    nsl = 0;
  };

  const int64_t klo = tk.nk > 1 ? (int64_t)tl.kc * tk.ksz : 0;
  const int64_t khi = tk.nk > 1 ? klo + tk.ksz : ((int64_t)1 << 62);
  int64_t koff = 0;
  for (int pi = tk.p0; pi < tk.p0 + tk.np; ++pi) {
    const GemmPair pr = pairs[pi];
    const int64_t kb = koff;
    koff += pr.K;
    if (koff <= klo || kb >= khi) continue;
    const int kbeg = (int)(klo > kb ? klo - kb : 0);
    const int kend = (int)(khi - kb < pr.K ? khi - kb : pr.K);
    const cf* A = (const cf*)pr.A;
    const cf* B = (const cf*)pr.B;
    const bool at = (pr.opA == OP_T || pr.opA == OP_H);
    const bool bt = (pr.opB == OP_T || pr.opB == OP_H);
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
      for (int r = 0; r < (BM * BK + NT - 1) / NT; ++r) {
        const int l = tid + r * NT;
        if (l >= BM * BK) break;
        int i, k;
        if (!at) { i = l % BM; k = l / BM; } else { k = l % BK; i = l / BK; }
        float re = 0, im = 0;
        if (m0 + i < tk.M && k0 + k < kend) load_op<cf, float>(A, pr.lda, pr.opA, m0 + i, k0 + k, re, im);
        As_r[k][i] = re;
        As_i[k][i] = im;
      }
#pragma unroll
      for (int r = 0; r < (BK * BN + NT - 1) / NT; ++r) {
        const int l = tid + r * NT;
        if (l >= BK * BN) break;
        int k, j;
        if (!bt) { k = l % BK; j = l / BK; } else { j = l % BN; k = l / BN; }
        float re = 0, im = 0;
        if (n0 + j < tk.N && k0 + k < kend) load_op<cf, float>(B, pr.ldb, pr.opB, k0 + k, n0 + j, re, im);
        Bs_r[k][j] = re;
        Bs_i[k][j] = im;
      }
      __syncthreads();
      float hr[TMR][TN], lr[TMR][TN], hi[TMR][TN], li[TMR][TN];
#pragma unroll
      for (int i = 0; i < TMR; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) hr[i][j] = lr[i][j] = hi[i][j] = li[i][j] = 0.f;
#pragma unroll
      for (int k = 0; k < BK; ++k) {
        float ar[TMR], ai[TMR], br[TN], bi[TN];
#pragma unroll
        for (int i = 0; i < TMR; ++i) { ar[i] = As_r[k][ty + TY * i]; ai[i] = As_i[k][ty + TY * i]; }
#pragma unroll
        for (int j = 0; j < TN; ++j) { br[j] = Bs_r[k][tx + TX * j]; bi[j] = Bs_i[k][tx + TX * j]; }
#pragma unroll
        for (int i = 0; i < TMR; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) {
            df_madd(hr[i][j], lr[i][j], ar[i], br[j]);
            df_madd(hr[i][j], lr[i][j], -ai[i], bi[j]);
            df_madd(hi[i][j], li[i][j], ar[i], bi[j]);
            df_madd(hi[i][j], li[i][j], ai[i], br[j]);
          }
      }
#pragma unroll
      for (int i = 0; i < TMR; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          dd_acc(Hr[i][j], Lr[i][j], hr[i][j], lr[i][j]);
          dd_acc(Hi[i][j], Li[i][j], hi[i][j], li[i][j]);
        }
      if (++nsl == kDfFlush) flush();
      __syncthreads();
    }
  }
  flush();
  if (tk.nk > 1) {
    cd* W = ws + tk.ws_off + (int64_t)tl.kc * tk.M * tk.N;
#pragma unroll
    for (int i = 0; i < TMR; ++i) {
      const int m = m0 + ty + TY * i;
      if (m >= tk.M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int n = n0 + tx + TX * j;
        if (n >= tk.N) continue;
        cd v;
        v.re = acc_r[i][j];
        v.im = acc_i[i][j];
        W[(int64_t)m + (int64_t)n * tk.M] = v;
      }
    }
    return;
  }
  cd* C = (cd*)tk.C;
#pragma unroll
  for (int i = 0; i < TMR; ++i) {
    const int m = m0 + ty + TY * i;
    if (m >= tk.M) continue;
    cd old[TN];
    if (tk.beta != 0.0) {
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int n = n0 + tx + TX * j;
        if (n < tk.N) old[j] = C[(size_t)m + (size_t)n * tk.ldc];
      }
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int n = n0 + tx + TX * j;
      if (n >= tk.N) continue;
      cd v;
      v.re = tk.alpha * acc_r[i][j];
      v.im = tk.alpha * acc_i[i][j];
      if (tk.beta != 0.0) {
        v.re = fma(tk.beta, old[j].re, v.re);
        v.im = fma(tk.beta, old[j].im, v.im);
      }
      C[(size_t)m + (size_t)n * tk.ldc] = v;
    }
  }
}

// ---- complex128 products in double-float on the FP32 pipe ---------------
//
// For the FP64 stages of the H^2 matvec that refinement residuals run
// through.  Each FP64 operand is split on load into hi = fl32(x) and
// lo = fl32(x - hi) (48 of its 53 bits); a product (ah + al)(bh + bl) is
// taken as the exact ah bh = p + e (e = fma(ah, bh, -p)) plus ah bl + al bh
// (al bl, 2^-48 of the product, is dropped); one BK-long K slice is summed in
// double-float as in k_gemm_df and the slice totals are added to a
// double-float accumulator (TwoSum), which becomes FP64 at the end.  About 12
// FP32 operations per real product: the relative error of an output is a few
// 2^-47 per term (~1e-13 of its magnitude for thousands of terms), against
// ~1e-16 with FP64 FMAs, at about a fifth of the FP64 pipe time.
__device__ __forceinline__ void dd_madd(float& h, float& l, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  const float s = __fadd_rn(h, p);
  const float bb = __fsub_rn(s, h);
  const float t = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  h = s;
  l = __fadd_rn(l, __fadd_rn(t, e));
}

__device__ __forceinline__ void dd_split(double x, float& h, float& l) {
  h = __double2float_rn(x);
  l = __double2float_rn(x - (double)h);
}

template <int BM, int BN>
__global__ void __launch_bounds__(NT) k_gemm_dd(const GemmTask* __restrict__ tasks,
                                               const GemmPair* __restrict__ pairs,
                                               const GemmTile* __restrict__ tiles, cd* __restrict__ ws) {
  constexpr int TX = BN >= 16 ? 16 : BN, TY = NT / TX, TN = BN / TX, TMR = BM / TY;
  static_assert(BN % TX == 0 && BM % TY == 0, "tile shape");
  __shared__ float As_rh[BK][BM], As_rl[BK][BM], As_ih[BK][BM], As_il[BK][BM];
  __shared__ float Bs_rh[BK][BN], Bs_rl[BK][BN], Bs_ih[BK][BN], Bs_il[BK][BN];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmTask tk = tasks[tl.task];
  const int m0 = tl.tm * BM, n0 = tl.tn * BN;
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  float Hr[TMR][TN], Lr[TMR][TN], Hi[TMR][TN], Li[TMR][TN];
#pragma unroll
  for (int i = 0; i < TMR; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) Hr[i][j] = Lr[i][j] = Hi[i][j] = Li[i][j] = 0.f;

  const int64_t klo = tk.nk > 1 ? (int64_t)tl.kc * tk.ksz : 0;
  const int64_t khi = tk.nk > 1 ? klo + tk.ksz : ((int64_t)1 << 62);
  int64_t koff = 0;
  for (int pi = tk.p0; pi < tk.p0 + tk.np; ++pi) {
    const GemmPair pr = pairs[pi];
    const int64_t kb = koff;
    koff += pr.K;
    if (koff <= klo || kb >= khi) continue;
    const int kbeg = (int)(klo > kb ? klo - kb : 0);
    const int kend = (int)(khi - kb < pr.K ? khi - kb : pr.K);
    const cd* A = (const cd*)pr.A;
    const cd* B = (const cd*)pr.B;
    const bool at = (pr.opA == OP_T || pr.opA == OP_H);
    const bool bt = (pr.opB == OP_T || pr.opB == OP_H);
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
      for (int r = 0; r < (BM * BK + NT - 1) / NT; ++r) {
        const int l = tid + r * NT;
        if (l >= BM * BK) break;
        int i, k;
        if (!at) { i = l % BM; k = l / BM; } else { k = l % BK; i = l / BK; }
        double re = 0, im = 0;
        if (m0 + i < tk.M && k0 + k < kend) load_op<cd, double>(A, pr.lda, pr.opA, m0 + i, k0 + k, re, im);
        dd_split(re, As_rh[k][i], As_rl[k][i]);
        dd_split(im, As_ih[k][i], As_il[k][i]);
      }
#pragma unroll
      for (int r = 0; r < (BK * BN + NT - 1) / NT; ++r) {
        const int l = tid + r * NT;
        if (l >= BK * BN) break;
        int k, j;
        if (!bt) { k = l % BK; j = l / BK; } else { j = l % BN; k = l / BN; }
        double re = 0, im = 0;
        if (n0 + j < tk.N && k0 + k < kend) load_op<cd, double>(B, pr.ldb, pr.opB, k0 + k, n0 + j, re, im);
        dd_split(re, Bs_rh[k][j], Bs_rl[k][j]);
        dd_split(im, Bs_ih[k][j], Bs_il[k][j]);
      }
      __syncthreads();
      float hr[TMR][TN], lr[TMR][TN], hi[TMR][TN], li[TMR][TN];
#pragma unroll
      for (int i = 0; i < TMR; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) hr[i][j] = lr[i][j] = hi[i][j] = li[i][j] = 0.f;
#pragma unroll
      for (int k = 0; k < BK; ++k) {
        float arh[TMR], arl[TMR], aih[TMR], ail[TMR], brh[TN], brl[TN], bih[TN], bil[TN];
#pragma unroll
        for (int i = 0; i < TMR; ++i) {
          arh[i] = As_rh[k][ty + TY * i];
          arl[i] = As_rl[k][ty + TY * i];
          aih[i] = As_ih[k][ty + TY * i];
          ail[i] = As_il[k][ty + TY * i];
        }
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          brh[j] = Bs_rh[k][tx + TX * j];
          brl[j] = Bs_rl[k][tx + TX * j];
          bih[j] = Bs_ih[k][tx + TX * j];
          bil[j] = Bs_il[k][tx + TX * j];
        }
#pragma unroll
        for (int i = 0; i < TMR; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) {
            dd_madd(hr[i][j], lr[i][j], arh[i], arl[i], brh[j], brl[j]);
            dd_madd(hr[i][j], lr[i][j], -aih[i], -ail[i], bih[j], bil[j]);
            dd_madd(hi[i][j], li[i][j], arh[i], arl[i], bih[j], bil[j]);
            dd_madd(hi[i][j], li[i][j], aih[i], ail[i], brh[j], brl[j]);
          }
      }
#pragma unroll
      for (int i = 0; i < TMR; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          dd_acc(Hr[i][j], Lr[i][j], hr[i][j], lr[i][j]);
          dd_acc(Hi[i][j], Li[i][j], hi[i][j], li[i][j]);
        }
      __syncthreads();
    }
  }
  if (tk.nk > 1) {
    cd* W = ws + tk.ws_off + (int64_t)tl.kc * tk.M * tk.N;
#pragma unroll
    for (int i = 0; i < TMR; ++i) {
      const int m = m0 + ty + TY * i;
      if (m >= tk.M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int n = n0 + tx + TX * j;
        if (n >= tk.N) continue;
        cd v;
        v.re = (double)Hr[i][j] + (double)Lr[i][j];
        v.im = (double)Hi[i][j] + (double)Li[i][j];
        W[(int64_t)m + (int64_t)n * tk.M] = v;
      }
    }
    return;
  }
  cd* C = (cd*)tk.C;
#pragma unroll
  for (int i = 0; i < TMR; ++i) {
    const int m = m0 + ty + TY * i;
    if (m >= tk.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int n = n0 + tx + TX * j;
      if (n >= tk.N) continue;
      cd v;
      v.re = tk.alpha * ((double)Hr[i][j] + (double)Lr[i][j]);
      v.im = tk.alpha * ((double)Hi[i][j] + (double)Li[i][j]);
      if (tk.beta != 0.0) {
        const cd old = C[(size_t)m + (size_t)n * tk.ldc];
        v.re = fma(tk.beta, old.re, v.re);
        v.im = fma(tk.beta, old.im, v.im);
      }
      C[(size_t)m + (size_t)n * tk.ldc] = v;
    }
  }
}

// ---- complex64 tiles on the tensor cores (3xTF32) ----------------------
//
// The same 64 x 64 tile / task / pair / split-K scheme as k_gemm, with the
// products on warp-level TF32 MMAs (m16n8k8, FP32 accumulation).  Each FP32
// operand x is split into x_hi = tf32(x) and x_lo = tf32(x - x_hi), and
// a b ~ a_lo b_hi + a_hi b_lo + a_hi b_hi (the a_lo b_lo term is below FP32
// rounding), so the result keeps FP32 accuracy.  Complex products:
// C_re += A_re B_re + (-A_im) B_im, C_im += A_re B_im + A_im B_re.
// 8 warps in a 2 x 4 grid, each owning a 32 x 16 sub-tile (2 x 2 MMA tiles).

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// c += a b with the three-term split (small terms first)
__device__ __forceinline__ void mma3(float* c, const uint32_t* ah, const uint32_t* al, const uint32_t* bh,
                                     const uint32_t* bl) {
  mma_tf32(c, al, bh);
  mma_tf32(c, ah, bl);
  mma_tf32(c, ah, bh);
}

__global__ void __launch_bounds__(NT) k_gemm_tc(const GemmTask* __restrict__ tasks,
                                               const GemmPair* __restrict__ pairs,
                                               const GemmTile* __restrict__ tiles, cf* __restrict__ ws) {
  constexpr int BM = 64, BN = 64, LA = BM + 8, LB = BN + 8;  // padded rows: conflict-free fragments
  __shared__ float As_r[BK][LA], As_i[BK][LA];
  __shared__ float Bs_r[BK][LB], Bs_i[BK][LB];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmTask tk = tasks[tl.task];
  const int m0 = tl.tm * BM, n0 = tl.tn * BN;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 2, wn = warp & 3, g = lane >> 2, q = lane & 3;
  float cr[2][2][4], ci[2][2][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int e = 0; e < 4; ++e) cr[a][b][e] = ci[a][b][e] = 0.f;

  const int64_t klo = tk.nk > 1 ? (int64_t)tl.kc * tk.ksz : 0;
  const int64_t khi = tk.nk > 1 ? klo + tk.ksz : ((int64_t)1 << 62);
  int64_t koff = 0;
  for (int pi = tk.p0; pi < tk.p0 + tk.np; ++pi) {
    const GemmPair pr = pairs[pi];
    const int64_t kb = koff;
    koff += pr.K;
    if (koff <= klo || kb >= khi) continue;
    const int kbeg = (int)(klo > kb ? klo - kb : 0);
    const int kend = (int)(khi - kb < pr.K ? khi - kb : pr.K);
    const cf* A = (const cf*)pr.A;
    const cf* B = (const cf*)pr.B;
    const bool at = (pr.opA == OP_T || pr.opA == OP_H);
    const bool bt = (pr.opB == OP_T || pr.opB == OP_H);
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
      for (int r = 0; r < (BM * BK) / NT; ++r) {
        const int l = tid + r * NT;
        int i, k;
        if (!at) { i = l % BM; k = l / BM; } else { k = l % BK; i = l / BK; }
        float re = 0, im = 0;
        if (m0 + i < tk.M && k0 + k < kend) load_op<cf, float>(A, pr.lda, pr.opA, m0 + i, k0 + k, re, im);
        As_r[k][i] = re;
        As_i[k][i] = im;
      }
#pragma unroll
      for (int r = 0; r < (BK * BN) / NT; ++r) {
        const int l = tid + r * NT;
        int k, j;
        if (!bt) { k = l % BK; j = l / BK; } else { j = l % BN; k = l / BN; }
        float re = 0, im = 0;
        if (n0 + j < tk.N && k0 + k < kend) load_op<cf, float>(B, pr.ldb, pr.opB, k0 + k, n0 + j, re, im);
        Bs_r[k][j] = re;
        Bs_i[k][j] = im;
      }
      __syncthreads();
      // B fragments (k x n = 8 x 8): b0 = B[q][g], b1 = B[q + 4][g]
      uint32_t brh[2][2], brl[2][2], bih[2][2], bil[2][2];
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int c = wn * 16 + nt * 8 + g;
        split_tf32(Bs_r[q][c], brh[nt][0], brl[nt][0]);
        split_tf32(Bs_r[q + 4][c], brh[nt][1], brl[nt][1]);
        split_tf32(Bs_i[q][c], bih[nt][0], bil[nt][0]);
        split_tf32(Bs_i[q + 4][c], bih[nt][1], bil[nt][1]);
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        // A fragments (m x k = 16 x 8): a0 = A[g][q], a1 = A[g + 8][q], a2 = A[g][q + 4], a3 = A[g + 8][q + 4]
        const int rw = wm * 32 + mt * 16 + g;
        uint32_t arh[4], arl[4], aih[4], ail[4], anh[4], anl[4];
        split_tf32(As_r[q][rw], arh[0], arl[0]);
        split_tf32(As_r[q][rw + 8], arh[1], arl[1]);
        split_tf32(As_r[q + 4][rw], arh[2], arl[2]);
        split_tf32(As_r[q + 4][rw + 8], arh[3], arl[3]);
        split_tf32(As_i[q][rw], aih[0], ail[0]);
        split_tf32(As_i[q][rw + 8], aih[1], ail[1]);
        split_tf32(As_i[q + 4][rw], aih[2], ail[2]);
        split_tf32(As_i[q + 4][rw + 8], aih[3], ail[3]);
#pragma unroll
        for (int e = 0; e < 4; ++e) {  // -A_im: flip the sign bits
          anh[e] = aih[e] ^ 0x80000000u;
          anl[e] = ail[e] ^ 0x80000000u;
        }
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          mma3(cr[mt][nt], arh, arl, brh[nt], brl[nt]);
          mma3(cr[mt][nt], anh, anl, bih[nt], bil[nt]);
          mma3(ci[mt][nt], arh, arl, bih[nt], bil[nt]);
          mma3(ci[mt][nt], aih, ail, brh[nt], brl[nt]);
        }
      }
      __syncthreads();
    }
  }
  // C fragment: c0 = (g, 2q), c1 = (g, 2q + 1), c2 = (g + 8, 2q), c3 = (g + 8, 2q + 1)
  const bool useold = tk.nk <= 1 && tk.beta != 0.0;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    cf old[2][4];  // this row block's C values in flight together
    if (useold) {
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int m = m0 + wm * 32 + mt * 16 + g + (e >> 1) * 8;
          const int n = n0 + wn * 16 + nt * 8 + 2 * q + (e & 1);
          if (m < tk.M && n < tk.N) old[nt][e] = ((const cf*)tk.C)[(size_t)m + (size_t)n * tk.ldc];
        }
    }
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int m = m0 + wm * 32 + mt * 16 + g + (e >> 1) * 8;
        const int n = n0 + wn * 16 + nt * 8 + 2 * q + (e & 1);
        if (m >= tk.M || n >= tk.N) continue;
        if (tk.nk > 1) {
          cf v;
          v.re = cr[mt][nt][e];
          v.im = ci[mt][nt][e];
          ws[tk.ws_off + (int64_t)tl.kc * tk.M * tk.N + (int64_t)m + (int64_t)n * tk.M] = v;
        } else {
          float re = (float)tk.alpha * cr[mt][nt][e], im = (float)tk.alpha * ci[mt][nt][e];
          if (useold) {
            re = fmaf((float)tk.beta, old[nt][e].re, re);
            im = fmaf((float)tk.beta, old[nt][e].im, im);
          }
          cf v;
          v.re = re;
          v.im = im;
          ((cf*)tk.C)[(size_t)m + (size_t)n * tk.ldc] = v;
        }
      }
  }
}

// ---- complex64 tiles on the 5th-generation tensor cores (tcgen05, 3xTF32) --
//
// The same 64 x 64 tile / task / pair / split-K scheme again, with the
// products issued asynchronously to the tensor cores and accumulated in tensor
// memory (TMEM).  The complex tile is one real 128 x 64 product
//   D = A' B'^T,  A' row m      = [Re A(m,k), -Im A(m,k)]_k
//                 A' row 64 + m = [Im A(m,k),  Re A(m,k)]_k
//                 B' row n      = [Re B(k,n),  Im B(k,n)]_k
// so that TMEM lanes 0..63 end up holding Re C and lanes 64..127 Im C.  Every
// operand is staged as hi = tf32(x) and lo = tf32(x - hi) planes and
// D += A'lo B'hi + A'hi B'lo + A'hi B'hi (the lo*lo term is below FP32
// rounding).  Shared-memory operands use the K-major, no-swizzle canonical
// layout: core matrices of 8 rows x 16 bytes, 8-row groups 128 B apart (SBO),
// K-adjacent core matrices LBO apart; LBO is padded by 16 B so that the
// 16-byte staging stores of a warp spread over all banks.
//
// All 256 threads stage one chunk of BKC complex K into one of S stages
// (global loads -> hi/lo split -> shared stores, the next chunk's loads issued
// before the barrier); thread 0 then issues the chunk's MMAs and commits them
// to the stage's mbarrier, which the stagers wait on before they refill it.
// Every wait is bounded: a wait that runs out marks the tile (NaN output) and
// counts in g_umma_timeouts, and the CTA still frees its TMEM.

__device__ unsigned int g_umma_timeouts = 0;

namespace umma {
__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// shared-memory matrix descriptor: start, LBO, SBO = 128 B, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t a, uint32_t lbo) {
  return (uint64_t)((a >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) | ((uint64_t)(128 >> 4) << 32) |
         (1ull << 46);
}
// instruction descriptor: kind::tf32, FP32 accumulator, A and B TF32 K-major, M = 128, N = BN
template <int BN>
constexpr uint32_t idesc() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

template <int BN>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc<BN>()), "r"(acc));
}
__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool try_wait(uint32_t bar, uint32_t parity) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"(bar), "r"(parity)
      : "memory");
  return r != 0;
}
// wait for the given phase of `bar`; gives up after ~2 s (or, unless
// draining, at once when another thread of the CTA already gave up) and
// reports it in *fail
__device__ __forceinline__ bool wait(uint32_t bar, uint32_t parity, volatile int* fail, bool drain = false) {
  const long long t0 = clock64();
  while (!try_wait(bar, parity)) {
    if (!drain && *fail) return false;
    if (clock64() - t0 > 4000000000ll) {
      *fail = 1;
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ float tf(float x) { return __uint_as_float(to_tf32(x)); }

template <int BKC, int S, int BN>
struct Cfg {
  static constexpr int KC = BKC / 2;  // 16-byte K groups (2 complex) per operand row
  static constexpr int LBO_A = 16 * 128 + 16, LBO_B = (BN / 8) * 128 + 16;
  static constexpr int PLANE_A = KC * LBO_A, PLANE_B = KC * LBO_B;
  static constexpr int STAGE = 2 * PLANE_A + 2 * PLANE_B;  // A hi, A lo, B hi, B lo
  static constexpr int DLD = BN + 1;                       // epilogue staging row stride (floats)
  static constexpr int BODY = S * STAGE > 128 * DLD * 4 ? S * STAGE : 128 * DLD * 4;
  static constexpr int SMEM = BODY + 1024;                 // + alignment slack
  static constexpr int NI = 64 * KC / NT;                  // A items per thread and chunk
  static constexpr int NIB = BN * KC / NT;                 // B items per thread and chunk
  static_assert(BKC % 4 == 0 && NI >= 1 && 64 * KC % NT == 0 && BN * KC % NT == 0, "chunk shape");
};

// position in the concatenated K range of a tile's pairs, with the current
// pair's operands (read once, when the cursor enters the pair)
struct Cursor {
  int pi, k0, kend;
  int64_t koff;
  const cf* A;
  const cf* B;
  int lda, ldb, opA, opB;
};
}  // namespace umma

template <int BKC, int S, int BN>
__global__ void __launch_bounds__(NT, BN == 64 ? 4 : 3) k_gemm_umma(const GemmTask* __restrict__ tasks,
                                                                const GemmPair* __restrict__ pairs,
                                                                const GemmTile* __restrict__ tiles,
                                                                cf* __restrict__ ws) {
  using C_ = umma::Cfg<BKC, S, BN>;
  constexpr int KC = C_::KC, NI = C_::NI, NIB = C_::NIB;
  extern __shared__ unsigned char smraw[];
  __shared__ uint64_t bars[S];
  __shared__ uint32_t tslot;
  __shared__ int fail;
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  const GemmTile tl = tiles[blockIdx.x];
  const GemmTask tk = tasks[tl.task];
  const int m0 = tl.tm * 64, n0 = tl.tn * BN;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t klo = tk.nk > 1 ? (int64_t)tl.kc * tk.ksz : 0;
  const int64_t khi = tk.nk > 1 ? klo + tk.ksz : ((int64_t)1 << 62);

  // next chunk of BKC complex K (within one pair); false at the end
  auto advance = [&](umma::Cursor& c) -> bool {
    c.k0 += BKC;
    while (c.k0 >= c.kend) {
      if (++c.pi >= tk.p0 + tk.np) return false;
      const GemmPair pr = pairs[c.pi];
      const int64_t kb = c.koff;
      c.koff += pr.K;
      if (c.koff <= klo || kb >= khi) {
        c.k0 = c.kend = 0;
        continue;
      }
      c.k0 = (int)(klo > kb ? klo - kb : 0);
      c.kend = (int)(khi - kb < pr.K ? khi - kb : pr.K);
      c.A = (const cf*)pr.A;
      c.B = (const cf*)pr.B;
      c.lda = pr.lda;
      c.ldb = pr.ldb;
      c.opA = pr.opA;
      c.opB = pr.opB;
    }
    return true;
  };
  // this thread's share of a chunk: NI A items and NI B items of 2 complex
  // each, as loaded (no operation on the values, so the loads stay in flight
  // until the chunk is staged); out-of-range elements are read from a clamped
  // in-range address and zeroed at staging (validity bits am / bm)
  float4 ra[NI], rb[NIB];
  unsigned am = 0, bm = 0;
  auto elem = [](const cf* X, int ld, bool tr, int r, int k) -> const cf& {
    return tr ? X[(size_t)k + (size_t)r * ld] : X[(size_t)r + (size_t)k * ld];
  };
  auto load = [&](const umma::Cursor& c) {
    const bool at = (c.opA == OP_T || c.opA == OP_H), bt = (c.opB == OP_T || c.opB == OP_H);
    am = bm = 0;
#pragma unroll
    for (int r = 0; r < NI; ++r) {
      const int it = tid + r * NT;
      const int m = at ? it / KC : (it & 63), kp = at ? it % KC : (it >> 6);
      const int k = c.k0 + 2 * kp;
      const bool vm = m0 + m < tk.M, v0 = vm && k < c.kend, v1 = vm && k + 1 < c.kend;
      am |= (v0 ? 1u : 0u) << (2 * r) | (v1 ? 1u : 0u) << (2 * r + 1);
      const int mm = vm ? m0 + m : 0;
      const cf x0 = elem(c.A, c.lda, at, mm, v0 ? k : c.k0), x1 = elem(c.A, c.lda, at, mm, v1 ? k + 1 : c.k0);
      ra[r] = make_float4(x0.re, x0.im, x1.re, x1.im);
    }
#pragma unroll
    for (int r = 0; r < NIB; ++r) {
      const int it = tid + r * NT;
      const int n = bt ? (it & (BN - 1)) : it / KC, kp = bt ? (it / BN) : it % KC;
      const int k = c.k0 + 2 * kp;
      const bool vn = n0 + n < tk.N, v0 = vn && k < c.kend, v1 = vn && k + 1 < c.kend;
      bm |= (v0 ? 1u : 0u) << (2 * r) | (v1 ? 1u : 0u) << (2 * r + 1);
      const int nn = vn ? n0 + n : 0;
      // op(B)(k, n): B(k, n) stored (ld = ldb) or B^T's (n, k) when transposed
      const cf x0 = elem(c.B, c.ldb, !bt, nn, v0 ? k : c.k0), x1 = elem(c.B, c.ldb, !bt, nn, v1 ? k + 1 : c.k0);
      rb[r] = make_float4(x0.re, x0.im, x1.re, x1.im);
    }
  };
  // mask, conjugate and split the staged registers into the hi / lo planes of stage st
  auto store = [&](unsigned char* st, const umma::Cursor& c) {
    const bool at = (c.opA == OP_T || c.opA == OP_H), bt = (c.opB == OP_T || c.opB == OP_H);
    const float sa = (c.opA == OP_C || c.opA == OP_H) ? -1.f : 1.f, sb = (c.opB == OP_C || c.opB == OP_H) ? -1.f : 1.f;
#pragma unroll
    for (int r = 0; r < NI; ++r) {
      const int it = tid + r * NT;
      const int m = at ? it / KC : (it & 63), kp = at ? it % KC : (it >> 6);
      const bool v0 = (am >> (2 * r)) & 1u, v1 = (am >> (2 * r + 1)) & 1u;
      const float4 v = make_float4(v0 ? ra[r].x : 0.f, v0 ? sa * ra[r].y : 0.f, v1 ? ra[r].z : 0.f,
                                   v1 ? sa * ra[r].w : 0.f);
      const float4 h = make_float4(umma::tf(v.x), umma::tf(v.y), umma::tf(v.z), umma::tf(v.w));
      const float4 l = make_float4(umma::tf(v.x - h.x), umma::tf(v.y - h.y), umma::tf(v.z - h.z), umma::tf(v.w - h.w));
      const int o0 = kp * C_::LBO_A + (m >> 3) * 128 + (m & 7) * 16;
      const int o1 = o0 + 8 * 128;  // row 64 + m
      *(float4*)(st + o0) = make_float4(h.x, -h.y, h.z, -h.w);
      *(float4*)(st + o1) = make_float4(h.y, h.x, h.w, h.z);
      *(float4*)(st + C_::PLANE_A + o0) = make_float4(l.x, -l.y, l.z, -l.w);
      *(float4*)(st + C_::PLANE_A + o1) = make_float4(l.y, l.x, l.w, l.z);
    }
#pragma unroll
    for (int r = 0; r < NIB; ++r) {
      const int it = tid + r * NT;
      const int n = bt ? (it & (BN - 1)) : it / KC, kp = bt ? (it / BN) : it % KC;
      const bool v0 = (bm >> (2 * r)) & 1u, v1 = (bm >> (2 * r + 1)) & 1u;
      const float4 v = make_float4(v0 ? rb[r].x : 0.f, v0 ? sb * rb[r].y : 0.f, v1 ? rb[r].z : 0.f,
                                   v1 ? sb * rb[r].w : 0.f);
      const float4 h = make_float4(umma::tf(v.x), umma::tf(v.y), umma::tf(v.z), umma::tf(v.w));
      const float4 l = make_float4(umma::tf(v.x - h.x), umma::tf(v.y - h.y), umma::tf(v.z - h.z), umma::tf(v.w - h.w));
      const int o = 2 * C_::PLANE_A + kp * C_::LBO_B + (n >> 3) * 128 + (n & 7) * 16;
      *(float4*)(st + o) = h;
      *(float4*)(st + C_::PLANE_B + o) = l;
    }
  };
  // store alpha * (re, im) (+ beta C) or the unscaled split-K partial
  auto emit = [&](int m, int n, float re, float im) {
    if (tk.nk > 1) {
      cf v;
      v.re = re;
      v.im = im;
      ws[tk.ws_off + (int64_t)tl.kc * tk.M * tk.N + (int64_t)m + (int64_t)n * tk.M] = v;
    } else {
      cf* p = (cf*)tk.C + (size_t)m + (size_t)n * tk.ldc;
      re *= (float)tk.alpha;
      im *= (float)tk.alpha;
      if (tk.beta != 0.0) {
        const cf cv = *p;
        re = fmaf((float)tk.beta, cv.re, re);
        im = fmaf((float)tk.beta, cv.im, im);
      }
      p->re = re;
      p->im = im;
    }
  };

  umma::Cursor cur{tk.p0 - 1, 0, 0, 0, nullptr, nullptr, 0, 0, 0, 0};
  if (!advance(cur)) {  // no K overlaps this tile: C = beta C (zero partial)
    for (int e = tid; e < 64 * BN; e += NT) {
      const int m = m0 + (e & 63), n = n0 + (e >> 6);
      if (m < tk.M && n < tk.N) emit(m, n, 0.f, 0.f);
    }
    return;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(umma::saddr(&tslot)),
                 "r"(BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < S; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(umma::saddr(&bars[s])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fail = 0;
  }
  load(cur);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tmem = tslot;
  const uint32_t sbase = umma::saddr(sm);

  int c = 0;
  for (;;) {
    const int s = c % S;
    if (c >= S) umma::wait(umma::saddr(&bars[s]), (uint32_t)((c / S - 1) & 1), &fail);
    store(sm + s * C_::STAGE, cur);
    const bool more = advance(cur);
    if (more) load(cur);  // next chunk's loads in flight across the barrier and the MMAs
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      umma::fence_after();
      const uint32_t a = sbase + s * C_::STAGE, bb = a + 2 * C_::PLANE_A;
#pragma unroll
      for (int ks = 0; ks < BKC / 4; ++ks) {
        const uint64_t ah = umma::sdesc(a + 2 * ks * C_::LBO_A, C_::LBO_A);
        const uint64_t al = umma::sdesc(a + C_::PLANE_A + 2 * ks * C_::LBO_A, C_::LBO_A);
        const uint64_t bh = umma::sdesc(bb + 2 * ks * C_::LBO_B, C_::LBO_B);
        const uint64_t bl = umma::sdesc(bb + C_::PLANE_B + 2 * ks * C_::LBO_B, C_::LBO_B);
        umma::mma<BN>(tmem, al, bh, (c > 0 || ks > 0) ? 1u : 0u);
        umma::mma<BN>(tmem, ah, bl, 1u);
        umma::mma<BN>(tmem, ah, bh, 1u);
      }
      umma::commit(umma::saddr(&bars[s]));
    }
    ++c;
    if (!more) break;
  }
  // drain: the last commit of every stage (the last of all covers every MMA
  // of the tile; waiting for each leaves no arrive in flight at exit)
  for (int s = 0; s < S && s < c; ++s) {
    const int ncommit = (c - 1 - s) / S + 1;
    umma::wait(umma::saddr(&bars[s]), (uint32_t)((ncommit - 1) & 1), &fail, true);
  }
  umma::fence_after();
  __syncthreads();
  // C values of the beta term: all loads in flight together (rather than one
  // load-store round trip per element), overlapping the TMEM read-out
  constexpr int EPT = 64 * BN / NT;
  const bool useold = tk.nk <= 1 && tk.beta != 0.0;
  cf cold[EPT];
  if (useold) {
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const int e = tid + i * NT, m = m0 + (e & 63), n = n0 + (e >> 6);
      if (m < tk.M && n < tk.N) cold[i] = ((const cf*)tk.C)[(size_t)m + (size_t)n * tk.ldc];
    }
  }
  const bool ok = fail == 0;
  float* Ds = (float*)sm;  // 128 x BN accumulator, row stride DLD
  if (ok) {
    // warp w reads TMEM lanes 32 (w mod 4) .. + 31 (its sub-partition's), columns
    // of half w / 4 of the tile
    const int row = 32 * (warp & 3) + lane, cb = (BN / 2) * (warp >> 2);
#pragma unroll
    for (int h = 0; h < BN / 16; ++h) {
      uint32_t v[8];
      const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(cb + 8 * h);
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                   : "r"(ta));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 8; ++j) Ds[row * C_::DLD + cb + 8 * h + j] = __uint_as_float(v[j]);
    }
  } else if (tid == 0) {
    atomicAdd(&g_umma_timeouts, 1u);
  }
  umma::fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
  const float nan = __int_as_float(0x7fc00000);
#pragma unroll
  for (int i = 0; i < EPT; ++i) {
    const int e = tid + i * NT, mi = e & 63, nj = e >> 6;
    const int m = m0 + mi, n = n0 + nj;
    if (m >= tk.M || n >= tk.N) continue;
    float re = ok ? Ds[mi * C_::DLD + nj] : nan, im = ok ? Ds[(64 + mi) * C_::DLD + nj] : nan;
    if (tk.nk > 1) {
      cf v;
      v.re = re;
      v.im = im;
      ws[tk.ws_off + (int64_t)tl.kc * tk.M * tk.N + (int64_t)m + (int64_t)n * tk.M] = v;
    } else {
      re *= (float)tk.alpha;
      im *= (float)tk.alpha;
      if (useold) {
        re = fmaf((float)tk.beta, cold[i].re, re);
        im = fmaf((float)tk.beta, cold[i].im, im);
      }
      cf v;
      v.re = re;
      v.im = im;
      ((cf*)tk.C)[(size_t)m + (size_t)n * tk.ldc] = v;
    }
  }
}

template <class R, class EO>
__global__ void k_gemm_reduce(const GemmTask* __restrict__ tasks, const typename CxOf<R>::T* __restrict__ ws) {
  const GemmTask tk = tasks[blockIdx.y];
  if (tk.nk <= 1) return;
  const int64_t mn = (int64_t)tk.M * tk.N;
  EO* C = (EO*)tk.C;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < mn; e += (int64_t)gridDim.x * blockDim.x) {
    R sr = 0, si = 0;
    for (int kc = 0; kc < tk.nk; ++kc) {
      const typename CxOf<R>::T v = ws[tk.ws_off + kc * mn + e];
      sr += v.re;
      si += v.im;
    }
    const int m = (int)(e % tk.M), n = (int)(e / tk.M);
    EO* p = C + (size_t)m + (size_t)n * tk.ldc;
    R re = (R)tk.alpha * sr, im = (R)tk.alpha * si;
    if (tk.beta != 0.0) {
      const EO c = *p;
      re = fma((R)tk.beta, (R)c.re, re);
      im = fma((R)tk.beta, (R)c.im, im);
    }
    store_val<EO, R>(p, re, im);
  }
}

template <class EO>
__global__ void k_gemm_mirror(const GemmTask* __restrict__ tasks, int bm) {
  const GemmTask tk = tasks[blockIdx.y];
  if (!tk.herm) return;
  const int64_t mn = (int64_t)tk.M * tk.N;
  EO* C = (EO*)tk.C;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < mn; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % tk.M), j = (int)(e / tk.M);
    if (i / bm > j / bm) {
      EO v = C[(size_t)j + (size_t)i * tk.ldc];
      v.im = -v.im;
      C[(size_t)i + (size_t)j * tk.ldc] = v;
    }
  }
}

}  // namespace

// tile shapes: 0 = 64 x 64, 1 = 64 x 16, 2 = 32 x 32, 3 = 32 x 16, 4 = 16 x 16
// shapes 0 64x64, 1 64x16, 2 32x32, 3 32x16, 4 16x16, 5 64x8, 6 64x4 (the
// narrow ones for products with a few right-hand sides; plain FP tiles only)
int gemm_tile_m(int shape) { return shape == 4 ? 16 : (shape == 2 || shape == 3) ? 32 : 64; }
int gemm_tile_n(int shape) {
  return shape == 0 ? 64 : shape == 2 ? 32 : shape == 5 ? 8 : shape == 6 ? 4 : shape == 7 ? 128 : 16;
}

template <int BM, int BN>
static cudaError_t gemm_tile(const GemmTask* d_tasks, const GemmPair* d_pairs, const GemmTile* d_tiles, int ntiles,
                             int pina, int pin, int pout, int pacc, void* ws, cudaStream_t s, int emul) {
  if (emul == 1 && pina == P32 && pin == P32 && pacc == P64 && pout == P64)
    k_gemm_df<BM, BN><<<ntiles, NT, 0, s>>>(d_tasks, d_pairs, d_tiles, (cd*)ws);
  else if (emul == 2 && pina == P64 && pin == P64 && pacc == P64 && pout == P64)
    k_gemm_dd<BM, BN><<<ntiles, NT, 0, s>>>(d_tasks, d_pairs, d_tiles, (cd*)ws);
  else if (pina == P64 && pin == P64 && pacc == P64 && pout == P64)
    k_gemm<cd, cd, double, cd, BM, BN><<<ntiles, NT, 0, s>>>(d_tasks, d_pairs, d_tiles, (cd*)ws);
  else if (pina == P32 && pin == P32 && pacc == P32 && pout == P32)
    k_gemm<cf, cf, float, cf, BM, BN><<<ntiles, NT, 0, s>>>(d_tasks, d_pairs, d_tiles, (cf*)ws);
  else if (pina == P32 && pin == P32 && pacc == P64 && pout == P64)
    k_gemm<cf, cf, double, cd, BM, BN><<<ntiles, NT, 0, s>>>(d_tasks, d_pairs, d_tiles, (cd*)ws);
  else if (pina == P64 && pin == P64 && pacc == P64 && pout == P32)
    k_gemm<cd, cd, double, cf, BM, BN><<<ntiles, NT, 0, s>>>(d_tasks, d_pairs, d_tiles, (cd*)ws);
  else if (pina == P64 && pin == P32 && pacc == P64 && pout == P64)
    k_gemm<cd, cf, double, cd, BM, BN><<<ntiles, NT, 0, s>>>(d_tasks, d_pairs, d_tiles, (cd*)ws);
  else if (pina == P64 && pin == P32 && pacc == P32 && pout == P32)
    k_gemm<cd, cf, float, cf, BM, BN><<<ntiles, NT, 0, s>>>(d_tasks, d_pairs, d_tiles, (cf*)ws);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

#ifndef UMMA_BKC
#define UMMA_BKC 8
#endif
#ifndef UMMA_S
#define UMMA_S 2
#endif

template <int BKC, int S, int BN>
static cudaError_t gemm_umma(const GemmTask* d_tasks, const GemmPair* d_pairs, const GemmTile* d_tiles, int ntiles,
                             cf* ws, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(k_gemm_umma<BKC, S, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               umma::Cfg<BKC, S, BN>::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_gemm_umma<BKC, S, BN><<<ntiles, NT, umma::Cfg<BKC, S, BN>::SMEM, s>>>(d_tasks, d_pairs, d_tiles, ws);
  return cudaGetLastError();
}

unsigned int gemm_umma_timeouts() {
  unsigned int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_umma_timeouts, sizeof(v)) != cudaSuccess) return ~0u;
  return v;
}

cudaError_t gemm(const GemmTask* d_tasks, const GemmPair* d_pairs, const GemmTile* d_tiles, int ntiles, int pin,
                 int pout, int pacc, void* ws, cudaStream_t s, int shape, int pina, int tensor, int emul) {
  if (ntiles <= 0) return cudaSuccess;
  if (pina < 0) pina = pin;
  if (shape == 7) {  // 64 x 128: tcgen05 tiles of complex64 products only
    if (tensor != 2 || pina != P32 || pin != P32 || pacc != P32 || pout != P32) return cudaErrorInvalidValue;
    return gemm_umma<UMMA_BKC, UMMA_S, 128>(d_tasks, d_pairs, d_tiles, ntiles, (cf*)ws, s);
  }
  if (tensor && shape == 0 && pina == P32 && pin == P32 && pacc == P32 && pout == P32) {
    if (tensor == 2) return gemm_umma<UMMA_BKC, UMMA_S, 64>(d_tasks, d_pairs, d_tiles, ntiles, (cf*)ws, s);
    k_gemm_tc<<<ntiles, NT, 0, s>>>(d_tasks, d_pairs, d_tiles, (cf*)ws);
    return cudaGetLastError();
  }
  switch (shape) {
    case 0: return gemm_tile<64, 64>(d_tasks, d_pairs, d_tiles, ntiles, pina, pin, pout, pacc, ws, s, emul);
    case 1: return gemm_tile<64, 16>(d_tasks, d_pairs, d_tiles, ntiles, pina, pin, pout, pacc, ws, s, emul);
    case 2: return gemm_tile<32, 32>(d_tasks, d_pairs, d_tiles, ntiles, pina, pin, pout, pacc, ws, s, emul);
    case 3: return gemm_tile<32, 16>(d_tasks, d_pairs, d_tiles, ntiles, pina, pin, pout, pacc, ws, s, emul);
    case 4: return gemm_tile<16, 16>(d_tasks, d_pairs, d_tiles, ntiles, pina, pin, pout, pacc, ws, s, emul);
    case 5: return emul ? cudaErrorInvalidValue : gemm_tile<64, 8>(d_tasks, d_pairs, d_tiles, ntiles, pina, pin, pout, pacc, ws, s, 0);
    case 6: return emul ? cudaErrorInvalidValue : gemm_tile<64, 4>(d_tasks, d_pairs, d_tiles, ntiles, pina, pin, pout, pacc, ws, s, 0);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t gemm_mirror(const GemmTask* d_tasks, int ntasks, int maxmn, int pout, int bm, cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  int gx = (maxmn + 255) / 256;
  if (gx > 64) gx = 64;
  if (gx < 1) gx = 1;
  for (int t0 = 0; t0 < ntasks; t0 += 65535) {
    const dim3 grid(gx, ntasks - t0 < 65535 ? ntasks - t0 : 65535);
    if (pout == P64) k_gemm_mirror<cd><<<grid, 256, 0, s>>>(d_tasks + t0, bm);
    else k_gemm_mirror<cf><<<grid, 256, 0, s>>>(d_tasks + t0, bm);
  }
  return cudaGetLastError();
}

cudaError_t gemm_reduce(const GemmTask* d_tasks, int ntasks, int maxmn, int pout, int pacc, const void* ws,
                        cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  int gx = (maxmn + 255) / 256;
  if (gx > 64) gx = 64;
  if (gx < 1) gx = 1;
  for (int t0 = 0; t0 < ntasks; t0 += 65535) {
    const dim3 grid(gx, ntasks - t0 < 65535 ? ntasks - t0 : 65535);
    if (pacc == P64 && pout == P64) k_gemm_reduce<double, cd><<<grid, 256, 0, s>>>(d_tasks + t0, (const cd*)ws);
    else if (pacc == P64 && pout == P32) k_gemm_reduce<double, cf><<<grid, 256, 0, s>>>(d_tasks + t0, (const cd*)ws);
    else if (pacc == P32 && pout == P32) k_gemm_reduce<float, cf><<<grid, 256, 0, s>>>(d_tasks + t0, (const cf*)ws);
    else return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace h2k
