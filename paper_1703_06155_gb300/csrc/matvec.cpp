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

void matvec_tree(Ctx& c, const cd* x, cd* y, int nrhs, bool adj) {
  const H2Host& H = c.H;
  const int L = H.L, l0 = H.l0;
  const int64_t N = H.tree.N;
  std::vector<std::vector<size_t>> koff(L + 1);
  std::vector<size_t> K(L + 1, 0), base(L + 1, 0);
  size_t tot = 0;
  for (int l = l0; l <= L; ++l) {
    koff[l].assign(size_t(1) << l, 0);
    for (int t = 0; t < (1 << l); ++t) {
      koff[l][t] = K[l];
      K[l] += H.rank[l][t];
    }
    base[l] = tot;
    tot += K[l] * nrhs;
  }
  cd* buf = (cd*)dev_ensure(c, c.scratch2, (2 * tot + 1) * sizeof(cd));
  auto xh = [&](int l, int t) { return buf + base[l] + koff[l][t]; };
  auto yh = [&](int l, int t) { return buf + tot + base[l] + koff[l][t]; };
  const cd* Vd = (const cd*)c.dV.p;
  const cd* Td = (const cd*)c.dT.p;
  const cd* Sd = (const cd*)c.dS.p;
  const cd* Dd = (const cd*)c.dD.p;
  const int opUp = adj ? OP_H : OP_T, opDown = adj ? OP_C : OP_N;
  // upward pass
  {
    GemmBatch g;
    for (int t = 0; t < (1 << L); ++t) {
      const int kt = H.rank[L][t], nt = (int)H.tree.size[L][t];
      if (kt == 0) continue;
      g.task(xh(L, t), (int)K[L], kt, nrhs, 1.0, 0.0);
      g.pair(Vd + c.V_off[t], nt, opUp, x + H.tree.start[L][t], (int)N, OP_N, nt);
      g.close();
    }
    run_gemm(c, g, P64, P64, P64, "matvec up leaf");
  }
  for (int l = L - 1; l >= l0; --l) {
    GemmBatch g;
    for (int t = 0; t < (1 << l); ++t) {
      const int kt = H.rank[l][t];
      const int k1 = H.rank[l + 1][2 * t], k2 = H.rank[l + 1][2 * t + 1];
      if (kt == 0) continue;
      g.task(xh(l, t), (int)K[l], kt, nrhs, 1.0, 0.0);
      g.pair(Td + c.T_off[l][t], k1 + k2, opUp, xh(l + 1, 2 * t), (int)K[l + 1], OP_N, k1 + k2);
      g.close();
    }
    run_gemm(c, g, P64, P64, P64, "matvec up");
  }
  // couplings
  {
    GemmBatch g;
    for (int l = l0; l <= L; ++l) {
      std::vector<std::vector<int>> by(size_t(1) << l);
      for (size_t q = 0; q < H.part.adm[l].size(); ++q) {
        const auto [t, s] = H.part.adm[l][q];
        by[adj ? s : t].push_back((int)q);
      }
      for (int u = 0; u < (1 << l); ++u) {
        const int ku = H.rank[l][u];
        if (ku == 0) continue;
        g.task(yh(l, u), (int)K[l], ku, nrhs, 1.0, 0.0);
        for (int q : by[u]) {
          const auto [t, s] = H.part.adm[l][q];
          if (!adj) g.pair(Sd + c.S_off[l][q], H.rank[l][t], OP_N, xh(l, s), (int)K[l], OP_N, H.rank[l][s]);
          else g.pair(Sd + c.S_off[l][q], H.rank[l][t], OP_H, xh(l, t), (int)K[l], OP_N, H.rank[l][t]);
        }
        g.close();
      }
    }
    run_gemm(c, g, P64, P64, P64, "matvec couple");
  }
  // downward pass
  for (int l = l0; l < L; ++l) {
    GemmBatch g;
    for (int t = 0; t < (1 << l); ++t) {
      const int kt = H.rank[l][t];
      const int k1 = H.rank[l + 1][2 * t], k2 = H.rank[l + 1][2 * t + 1];
      if (kt == 0 || k1 + k2 == 0) continue;
      g.task(yh(l + 1, 2 * t), (int)K[l + 1], k1 + k2, nrhs, 1.0, 1.0);
      g.pair(Td + c.T_off[l][t], k1 + k2, opDown, yh(l, t), (int)K[l], OP_N, kt);
      g.close();
    }
    run_gemm(c, g, P64, P64, P64, "matvec down");
  }
  // leaves: basis part and dense near field
  {
    std::vector<std::vector<int>> by(size_t(1) << L);
    for (size_t q = 0; q < H.part.inad[L].size(); ++q) {
      const auto [t, s] = H.part.inad[L][q];
      by[adj ? s : t].push_back((int)q);
    }
    GemmBatch g;
    for (int u = 0; u < (1 << L); ++u) {
      const int nu = (int)H.tree.size[L][u], ku = H.rank[L][u];
      g.task(y + H.tree.start[L][u], (int)N, nu, nrhs, 1.0, 0.0);
      if (ku > 0) g.pair(Vd + c.V_off[u], nu, opDown, yh(L, u), (int)K[L], OP_N, ku);
      for (int q : by[u]) {
        const auto [t, s] = H.part.inad[L][q];
        const int nt = (int)H.tree.size[L][t], ns = (int)H.tree.size[L][s];
        if (!adj) g.pair(Dd + c.D_off[q], nt, OP_N, x + H.tree.start[L][s], (int)N, OP_N, ns);
        else g.pair(Dd + c.D_off[q], nt, OP_H, x + H.tree.start[L][t], (int)N, OP_N, nt);
      }
      g.close();
    }
    run_gemm(c, g, P64, P64, P64, "matvec leaf");
  }
}

// Explicit factor-form inverse (eq. 35): the diagonal inverses L^{-1}P and
// U^{-1} exist already; add -U^{-1} U_ik for every U panel and the inverse of
// the final block, so the backward sweep is matrix-vector products only.
void root_solve_public(Ctx& c, char* x, int ld, int nrhs, bool adjoint);

void invert(Ctx& c) {
  if (!c.factored) fail(H2_ESTATE, "invert before factorize");
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
    for (int i = 0; i < F.nc; ++i) {
      const int mi = F.m[i], ni = F.n[i];
      if (mi <= 0) continue;
      const char* Uinv = (char*)F.inv_buf.p + (F.inv_off[i] + (size_t)ni * ni) * es;
      for (size_t q = 0; q < F.nbrs[i].size(); ++q) {
        const int k = F.nbrs[i][q];
        const int clo = (k == i) ? F.m[i] : (F.batch_of[k] < F.batch_of[i] ? F.m[k] : 0);
        g.task(Ub + F.Ub_off[F.nbr_first[i] + q] * es, mi, mi, F.n[k] - clo, -1.0, 0.0);
        g.pair(Uinv, mi, OP_N,
               (char*)F.near_buf.p + (F.near_off.at(F.near_id.at(pkey(i, k))) + (size_t)clo * ni) * es, ni, OP_N, mi);
        g.close();
      }
    }
    run_gemm(c, g, prec, prec, prec, "inverse panels");
  }
  RootF& R = c.root;
  if (R.n > 0) {
    char* Ri = (char*)dev_ensure(c, R.Rinv, (size_t)R.n * R.n * es);
    ck(cudaMemsetAsync(Ri, 0, (size_t)R.n * R.n * es, c.stream), "Rinv memset");
    ck(set_diag(Ri, R.n, R.n, prec, 1.0, c.stream), "Rinv identity");
    root_solve_public(c, Ri, R.n, R.n, false);
  }
  ck(cudaStreamSynchronize(c.stream), "invert sync");
  c.inverted = true;
}

}  // namespace h2
