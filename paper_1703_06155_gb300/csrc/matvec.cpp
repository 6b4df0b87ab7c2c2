// FP64 H^2 matrix-vector product and the explicit inverse of eq. (35).
//
// y = Z x with Z_ts = V_t S_ts V_s^T (eq. 2) and nested bases (eq. 3):
//   upward    xh_t = V_t^T x_t (leaves), xh_t = T_t^T [xh_t1; xh_t2]
//   coupling  yh_t = sum_s S_ts xh_s over the admissible pairs of each level
//   downward  [yh_t1; yh_t2] += T_t yh_t, y_t = V_t yh_t at the leaves
//   near      y_t += sum_s Z_ts x_s over the dense leaf blocks
// y = Z^H x uses the conjugate-transposed blocks: V^H / T^H upward, S_ts^H
// into yh_s, conj(T) / conj(V) downward, Z_ts^H into y_s.
// Every stage is one batched GEMM launch over all clusters of a level.
#include <algorithm>

#include "batch.h"

namespace h2 {
using namespace h2k;

// The product for a group of instances: each stage (and each level-from-leaf
// index of the upward / downward passes) is one launch over all instances.
// xs[q], ys[q]: instance q's vectors in tree order (FP64, N x nrhs).
void matvec_tree_group(const std::vector<Ctx*>& cs, const std::vector<const cd*>& xs, const std::vector<cd*>& ys,
                       int nrhs, bool adj) {
  Ctx& lc = *cs[0];
  const size_t nq = cs.size();
  struct Lay {
    std::vector<std::vector<size_t>> koff;
    std::vector<size_t> K, base;
    cd* buf;
    size_t tot;
  };
  std::vector<Lay> ly(nq);
  int depth = 0;
  for (size_t q = 0; q < nq; ++q) {
    Ctx& c = *cs[q];
    const H2Host& H = c.H;
    const int L = H.L, l0 = H.l0;
    depth = std::max(depth, L - l0);
    Lay& y = ly[q];
    y.koff.assign(L + 1, {});
    y.K.assign(L + 1, 0);
    y.base.assign(L + 1, 0);
    y.tot = 0;
    for (int l = l0; l <= L; ++l) {
      y.koff[l].assign(size_t(1) << l, 0);
      for (int t = 0; t < (1 << l); ++t) {
        y.koff[l][t] = y.K[l];
        y.K[l] += H.rank[l][t];
      }
      y.base[l] = y.tot;
      y.tot += y.K[l] * nrhs;
    }
    y.buf = (cd*)dev_ensure(c, c.scratch2, (2 * y.tot + 1) * sizeof(cd));
  }
  auto xh = [&](size_t q, int l, int t) { return ly[q].buf + ly[q].base[l] + ly[q].koff[l][t]; };
  auto yh = [&](size_t q, int l, int t) { return ly[q].buf + ly[q].tot + ly[q].base[l] + ly[q].koff[l][t]; };
  const int opUp = adj ? OP_H : OP_T, opDown = adj ? OP_C : OP_N;
  // upward pass: leaves, then level L - d for d = 1, 2, ...
  {
    GemmBatch g;
    for (size_t q = 0; q < nq; ++q) {
      Ctx& c = *cs[q];
      const H2Host& H = c.H;
      const int L = H.L;
      for (int t = 0; t < (1 << L); ++t) {
        const int kt = H.rank[L][t], nt = (int)H.tree.size[L][t];
        if (kt == 0) continue;
        g.task(xh(q, L, t), (int)ly[q].K[L], kt, nrhs, 1.0, 0.0);
        g.pair((const cd*)c.dV.p + c.V_off[t], nt, opUp, xs[q] + H.tree.start[L][t], (int)H.tree.N, OP_N, nt);
        g.close();
      }
    }
    run_gemm(lc, g, P64, P64, P64, "matvec up leaf");
  }
  for (int d = 1; d <= depth; ++d) {
    GemmBatch g;
    for (size_t q = 0; q < nq; ++q) {
      Ctx& c = *cs[q];
      const H2Host& H = c.H;
      const int l = H.L - d;
      if (l < H.l0) continue;
      for (int t = 0; t < (1 << l); ++t) {
        const int kt = H.rank[l][t];
        const int k1 = H.rank[l + 1][2 * t], k2 = H.rank[l + 1][2 * t + 1];
        if (kt == 0) continue;
        g.task(xh(q, l, t), (int)ly[q].K[l], kt, nrhs, 1.0, 0.0);
        g.pair((const cd*)c.dT.p + c.T_off[l][t], k1 + k2, opUp, xh(q, l + 1, 2 * t), (int)ly[q].K[l + 1], OP_N,
               k1 + k2);
        g.close();
      }
    }
    run_gemm(lc, g, P64, P64, P64, "matvec up");
  }
  // couplings of every level
  {
    GemmBatch g;
    for (size_t q = 0; q < nq; ++q) {
      Ctx& c = *cs[q];
      const H2Host& H = c.H;
      const cd* Sd = (const cd*)c.dS.p;
      for (int l = H.l0; l <= H.L; ++l) {
        std::vector<std::vector<int>> by(size_t(1) << l);
        for (size_t u = 0; u < H.part.adm[l].size(); ++u) {
          const auto [t, s2] = H.part.adm[l][u];
          by[adj ? s2 : t].push_back((int)u);
        }
        for (int v = 0; v < (1 << l); ++v) {
          const int kv = H.rank[l][v];
          if (kv == 0) continue;
          g.task(yh(q, l, v), (int)ly[q].K[l], kv, nrhs, 1.0, 0.0);
          for (int u : by[v]) {
            const auto [t, s2] = H.part.adm[l][u];
            if (!adj)
              g.pair(Sd + c.S_off[l][u], H.rank[l][t], OP_N, xh(q, l, s2), (int)ly[q].K[l], OP_N, H.rank[l][s2]);
            else
              g.pair(Sd + c.S_off[l][u], H.rank[l][t], OP_H, xh(q, l, t), (int)ly[q].K[l], OP_N, H.rank[l][t]);
          }
          g.close();
        }
      }
    }
    run_gemm(lc, g, P64, P64, P64, "matvec couple");
  }
  // downward pass: level L - d for d = depth .. 1
  for (int d = depth; d >= 1; --d) {
    GemmBatch g;
    for (size_t q = 0; q < nq; ++q) {
      Ctx& c = *cs[q];
      const H2Host& H = c.H;
      const int l = H.L - d;
      if (l < H.l0) continue;
      for (int t = 0; t < (1 << l); ++t) {
        const int kt = H.rank[l][t];
        const int k1 = H.rank[l + 1][2 * t], k2 = H.rank[l + 1][2 * t + 1];
        if (kt == 0 || k1 + k2 == 0) continue;
        g.task(yh(q, l + 1, 2 * t), (int)ly[q].K[l + 1], k1 + k2, nrhs, 1.0, 1.0);
        g.pair((const cd*)c.dT.p + c.T_off[l][t], k1 + k2, opDown, yh(q, l, t), (int)ly[q].K[l], OP_N, kt);
        g.close();
      }
    }
    run_gemm(lc, g, P64, P64, P64, "matvec down");
  }
  // leaves: basis part and dense near field
  {
    GemmBatch g;
    for (size_t q = 0; q < nq; ++q) {
      Ctx& c = *cs[q];
      const H2Host& H = c.H;
      const int L = H.L;
      const int64_t N = H.tree.N;
      const cd* Vd = (const cd*)c.dV.p;
      const cd* Dd = (const cd*)c.dD.p;
      std::vector<std::vector<int>> by(size_t(1) << L);
      for (size_t u = 0; u < H.part.inad[L].size(); ++u) {
        const auto [t, s2] = H.part.inad[L][u];
        by[adj ? s2 : t].push_back((int)u);
      }
      for (int v = 0; v < (1 << L); ++v) {
        const int nv = (int)H.tree.size[L][v], kv = H.rank[L][v];
        g.task(ys[q] + H.tree.start[L][v], (int)N, nv, nrhs, 1.0, 0.0);
        if (kv > 0) g.pair(Vd + c.V_off[v], nv, opDown, yh(q, L, v), (int)ly[q].K[L], OP_N, kv);
        for (int u : by[v]) {
          const auto [t, s2] = H.part.inad[L][u];
          const int nt = (int)H.tree.size[L][t], ns = (int)H.tree.size[L][s2];
          if (!adj) g.pair(Dd + c.D_off[u], nt, OP_N, xs[q] + H.tree.start[L][s2], (int)N, OP_N, ns);
          else g.pair(Dd + c.D_off[u], nt, OP_H, xs[q] + H.tree.start[L][t], (int)N, OP_N, nt);
        }
        g.close();
      }
    }
    run_gemm(lc, g, P64, P64, P64, "matvec leaf");
  }
}

void matvec_tree(Ctx& c, const cd* x, cd* y, int nrhs, bool adj) { matvec_tree_group({&c}, {x}, {y}, nrhs, adj); }

// Explicit factor-form inverse (eq. 35): the diagonal inverses L^{-1}P and
// U^{-1} and the inverse of the final block exist after the factorization;
// add -U^{-1} U_ik for every U panel (-F^{-1} Z_i'k for block LDL^T factors),
// so the backward sweep is matrix-vector products only.

void invert(Ctx& c) {
  if (!c.factored) fail(H2_ESTATE, "invert before factorize");
  c.epoch++;
  const int prec = c.prec;
  const size_t es = esz(prec);
  for (LevelF& F : c.lev) {
    F.Ub_off.assign(F.nbr_first.back(), 0);
    size_t tot = 0;
    for (int i = 0; i < F.nc; ++i)
      for (size_t q = 0; q < F.nbrs[i].size(); ++q) {
        const int k = F.nbrs[i][q];
        const int clo = (k == i) ? F.m[i] : (F.batch_of[k] < F.batch_of[i] ? F.m[k] : 0);
        F.Ub_off[F.nbr_first[i] + q] = tot;
        tot += (size_t)F.m[i] * (F.n[k] - clo);
      }
    char* Ub = (char*)dev_ensure(c, F.Ub_buf, (tot + 1) * es);
    GemmBatch g;
    ApplyBatch ua;
    for (int i = 0; i < F.nc; ++i) {
      const int mi = F.m[i], ni = F.n[i];
      if (mi <= 0) continue;
      // LU: -U^{-1} (L^{-1}P Z_i'k), the U panel holding L^{-1}P Z_i'k;
      // block LDL^T: -F^{-1} Z_i'k = -U^{-1} (L^{-1}P Z_i'k) from the raw block
      const char* Linv = (char*)F.inv_buf.p + F.inv_off[i] * es;
      const char* Uinv = Linv + (size_t)ni * ni * es;
      for (size_t q = 0; q < F.nbrs[i].size(); ++q) {
        const int k = F.nbrs[i][q];
        const int clo = (k == i) ? F.m[i] : (F.batch_of[k] < F.batch_of[i] ? F.m[k] : 0);
        const char* blk = (char*)F.near_buf.p + F.near_off.at(F.near_id.at(pkey(i, k))) * es;
        char* Ubq = Ub + F.Ub_off[F.nbr_first[i] + q] * es;
        g.task(Ubq, mi, mi, F.n[k] - clo, -1.0, 0.0);
        if (!F.sym)
          g.pair(Uinv, mi, OP_N, blk + (size_t)clo * ni * es, ni, OP_N, mi);
        else if (i > k)  // Z_i'k = rows clo.. of the stored (k, i), transposed
          g.pair(Linv, mi, OP_N, blk + (size_t)clo * es, F.n[k], OP_T, mi);
        else
          g.pair(Linv, mi, OP_N, blk + (size_t)clo * ni * es, ni, OP_N, mi);
        g.close();
        if (F.sym) ua.add(Uinv, mi, OP_N, Ubq, mi, mi, F.n[k] - clo, 0);
      }
    }
    run_gemm(c, g, prec, prec, prec, "inverse panels");
    run_apply(c, ua, true, prec, "inverse panels U^-1");
  }
  ck(cudaStreamSynchronize(c.stream), "invert sync");
  c.inverted = true;
}

}  // namespace h2
