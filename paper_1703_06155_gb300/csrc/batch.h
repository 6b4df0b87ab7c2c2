// Host-side builders for the batched task lists and their launch helpers.
#pragma once
#include <algorithm>

#include "h2_host.h"

namespace h2 {

inline size_t esz(int prec) { return prec == h2k::P64 ? sizeof(h2k::cd) : sizeof(h2k::cf); }

// C = alpha * sum op(A) op(B) + beta * C, tiled 64 x 64
struct GemmBatch {
  std::vector<h2k::GemmTask> t;
  std::vector<h2k::GemmPair> p;
  std::vector<h2k::GemmTile> tl;
  double flops = 0;
  void task(void* C, int ldc, int M, int N, double alpha, double beta) {
    t.push_back(h2k::GemmTask{C, ldc, M, N, (int)p.size(), 0, alpha, beta, 1, 0, 0, 0});
  }
  void pair(const void* A, int lda, int opA, const void* B, int ldb, int opB, int K) {
    if (K <= 0) return;
    p.push_back(h2k::GemmPair{A, B, lda, ldb, K, opA, opB});
    t.back().np++;
    flops += 8.0 * t.back().M * (double)t.back().N * K;
  }
  // mark the open task's C as Hermitian (square, sum of X X^H products)
  void hermitian() { t.back().herm = 1; }
  void close() {
    h2k::GemmTask& g = t.back();
    if (g.M <= 0 || g.N <= 0 || (g.np == 0 && g.beta == 1.0)) {
      p.resize(g.p0);
      t.pop_back();
    }
  }
  // Tile list; tasks whose K is long compared with the number of output tiles
  // are split along K (deterministic two-pass sum) so that a launch keeps the
  // SMs busy.  Returns the split-K workspace size in accumulator elements.
  double alg_flops = 0;  // 8 M N K per pair; Hermitian outputs: upper triangle only
  int shape = 0;         // output tile shape (h2k::gemm_tile_m / gemm_tile_n)
  int pina = -1;         // precision of the A operands if it differs from B's
  // fp64: FP64-accumulating launch (the FP64 pipe bounds it, so padding is
  // what costs); FP32 launches keep 64-wide tiles unless padding dominates
  // narrow_ok: the 64 x 8 / 64 x 4 shapes may be used; wide_ok: the 64 x 128
  // shape (tcgen05 tiles of complex64 products only) may be used
  int64_t plan(int target_ctas = 8 * 152, bool fp64 = true, int policy = 0, bool narrow_ok = true,
               bool wide_ok = false) {
    tl.clear();
    alg_flops = 0;
    std::vector<int64_t> kt(t.size(), 0);
    for (size_t ti = 0; ti < t.size(); ++ti)
      for (int q = t[ti].p0; q < t[ti].p0 + t[ti].np; ++q) kt[ti] += p[q].K;
    for (size_t ti = 0; ti < t.size(); ++ti) {
      const auto& g = t[ti];
      for (int q = g.p0; q < g.p0 + g.np; ++q)
        alg_flops += g.herm ? 4.0 * g.M * (double)(g.M + 1) * p[q].K : 8.0 * g.M * (double)g.N * p[q].K;
    }
    // tile shape: least padded work, small tiles charged for their lower
    // arithmetic intensity; Hermitian outputs need square tiles
    bool anyherm = false;
    for (auto& g : t) anyherm |= g.herm != 0;
    static const double pen64[8] = {1.0, 1.08, 1.15, 1.3, 1.3, 1.2, 1.3, 1.0},
                        pen32[8] = {1.0, 1.6, 2.2, 3.5, 5.0, 2.5, 3.0, 0.8};
    const double* penalty = fp64 ? pen64 : pen32;
    double best = -1;
    bool narrow = !anyherm;
    for (auto& g : t) narrow = narrow && g.N <= 16;
    for (int sh = 0; sh < 8; ++sh) {
      if (anyherm && (sh == 1 || sh == 3 || sh >= 5)) continue;
      if ((sh == 5 || sh == 6) && !narrow_ok) continue;
      if (sh == 7 && !wide_ok) continue;
      if (policy == 1 && sh != (narrow ? 1 : 0)) continue;
      const int bm = h2k::gemm_tile_m(sh), bn = h2k::gemm_tile_n(sh);
      double w = 0;
      for (size_t ti = 0; ti < t.size(); ++ti) {
        const auto& g = t[ti];
        const double a = (g.M + bm - 1) / bm, b = (g.N + bn - 1) / bn;
        w += (g.herm ? a * (a + 1) / 2 : a * b) * bm * (double)bn * (double)kt[ti];
      }
      w *= penalty[sh];
      if (best < 0 || w < best) {
        best = w;
        shape = sh;
      }
    }
    const int bm = h2k::gemm_tile_m(shape), bn = h2k::gemm_tile_n(shape);
    auto ntile = [&](const h2k::GemmTask& g) {
      const int64_t a = (g.M + bm - 1) / bm, b = (g.N + bn - 1) / bn;
      return g.herm ? a * (a + 1) / 2 : a * b;
    };
    int64_t tiles0 = 0;
    for (auto& g : t) tiles0 += ntile(g);
    int64_t ws = 0;
    for (size_t ti = 0; ti < t.size(); ++ti) {
      h2k::GemmTask& g = t[ti];
      const int64_t K = kt[ti];
      int nk = 1;
      if (tiles0 < target_ctas && K >= 128) {
        nk = (int)std::min<int64_t>((target_ctas + tiles0 - 1) / tiles0, K / 64);
        nk = std::max(1, std::min(nk, 64));
      }
      g.nk = nk;
      g.ksz = nk > 1 ? (int)(((K + nk - 1) / nk + 7) / 8 * 8) : 0;
      if (nk > 1) {
        nk = (int)((K + g.ksz - 1) / g.ksz);
        g.nk = nk;
        g.ws_off = ws;
        ws += (int64_t)nk * g.M * g.N;
      }
      for (int kc = 0; kc < g.nk; ++kc)
        for (int tn = 0; tn * bn < g.N; ++tn)
          for (int tm = 0; tm * bm < g.M; ++tm)
            if (!g.herm || tm <= tn) tl.push_back(h2k::GemmTile{(int)ti, tm, tn, kc});
    }
    return ws;
  }
  bool empty() const { return t.empty(); }
  void clear() { t.clear(); p.clear(); tl.clear(); flops = 0; }
};

// in-place X <- op(A) X (left) or X <- X op(A) (right)
struct ApplyBatch {
  std::vector<h2k::ApplyTask> t;
  int maxp = 0;
  double flops = 0;
  void add(const void* A, int lda, int op, void* X, int ldx, int p, int w, int lo) {
    if (p <= 0 || w <= 0 || lo >= p) return;
    t.push_back(h2k::ApplyTask{A, X, lda, ldx, p, w, lo, op});
    maxp = std::max(maxp, p);
    flops += 8.0 * (double)(p - lo) * p * w;
  }
  bool empty() const { return t.empty(); }
  void clear() { t.clear(); maxp = 0; flops = 0; }
};

struct CopyBatch {
  std::vector<h2k::CopyTask> t;
  // dst[0:rows,0:cols] (=|+=) src[0:srows,0:scols] zero-padded
  void add(const void* src, int sprec, int lds, int srows, int scols, void* dst, int dprec, int ldd, int rows,
           int cols, int mode = 0, double alpha = 1.0) {
    if (rows <= 0 || cols <= 0) return;
    t.push_back(h2k::CopyTask{src, dst, lds, ldd, rows, cols, srows, scols, sprec, dprec, mode, 0, alpha});
  }
  bool empty() const { return t.empty(); }
  void clear() { t.clear(); }
};

void run_gemm(Ctx& c, GemmBatch& b, int pin, int pout, int pacc, const char* what);
void run_apply(Ctx& c, ApplyBatch& b, bool left, int prec, const char* what);
// the same application by the batched GEMM: op(A) X (left) or X op(A)
// (right) into a workspace, the output split over many CTAs, then copied back
void run_apply_gemm(Ctx& c, ApplyBatch& b, bool left, int prec, const char* what);
inline void run_apply_narrow(Ctx& c, ApplyBatch& b, int prec, const char* what) {
  run_apply_gemm(c, b, true, prec, what);
}
void run_copy(Ctx& c, CopyBatch& b, const char* what);

// host-side bounds checks of the task lists (checks.cpp, H2_CHECKS)
void check_gemm(const GemmBatch& b, int pina, int pin, int pout, const char* what);
void check_copy(const CopyBatch& b, const char* what);
void check_apply(const ApplyBatch& b, bool left, int prec, const char* what);
void check_lu(const std::vector<h2k::LuTask>& lu, int prec);

}  // namespace h2
