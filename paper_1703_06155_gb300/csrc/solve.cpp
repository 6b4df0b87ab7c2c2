// Forward substitution (Algorithm 5, eqs. 36-39), the final block, backward
// substitution (Algorithm 6, eqs. 40-42), the adjoint traversal of the same
// factors, the explicit inverse of eq. (35), and the FP64 H^2 matvec.
//
// Per level the right-hand sides live in a level vector whose cluster c
// occupies rows voff[c] .. voff[c]+n_c (column-major, nrhs columns).  The
// eliminated part (rows 0..m_c) of every level vector is kept after the
// forward sweep; the backward sweep fills the kept part (rows m_c..n_c) from
// the parent level and then solves for the eliminated part.
#include <algorithm>
#include <chrono>
#include <map>

#include "batch.h"

namespace h2 {
using namespace h2k;

namespace {

struct Vec {
  char* p;
  int64_t ld;
};

// "j was eliminated before i" decides whether block (i, j) of the factors
// has n_j or only the kept k~_j columns of j (and likewise for rows).
inline int lo_at(const LevelF& F, int j, int i) {
  if (j == i) return F.m[i];
  return F.batch_of[j] < F.batch_of[i] ? F.m[j] : 0;
}

char* NBp(Ctx& c, const LevelF& F, int j, int k) {
  return (char*)F.near_buf.p + F.near_off.at(F.near_id.at(pkey(j, k))) * esz(c.prec);
}

void merge_vec(Ctx& c, const LevelF& F, const LevelF& Pn, Vec v, Vec vp, int nrhs, bool up) {
  const int prec = c.prec;
  const size_t es = esz(prec);
  CopyBatch cb;
  for (int p = 0; p < Pn.nc; ++p)
    for (int a = 2 * p; a <= 2 * p + 1; ++a) {
      const int o = (a & 1) ? F.kt[a - 1] : 0;
      char* child = v.p + (size_t)(F.voff[a] + F.m[a]) * es;
      char* par = vp.p + (size_t)(Pn.voff[p] + o) * es;
      if (up) cb.add(child, prec, (int)v.ld, F.kt[a], nrhs, par, prec, (int)vp.ld, F.kt[a], nrhs);
      else cb.add(par, prec, (int)vp.ld, F.kt[a], nrhs, child, prec, (int)v.ld, F.kt[a], nrhs);
    }
  run_copy(c, cb, up ? "vec merge" : "vec scatter");
}

void root_vec(Ctx& c, const LevelF& F, Vec v, Vec vr, int nrhs, bool up) {
  const int prec = c.prec;
  const size_t es = esz(prec);
  CopyBatch cb;
  int off = 0;
  for (int a = 0; a < F.nc; ++a) {
    char* lv = v.p + (size_t)(F.voff[a] + F.m[a]) * es;
    char* rv = vr.p + (size_t)off * es;
    if (up) cb.add(lv, prec, (int)v.ld, F.kt[a], nrhs, rv, prec, (int)vr.ld, F.kt[a], nrhs);
    else cb.add(rv, prec, (int)vr.ld, F.kt[a], nrhs, lv, prec, (int)v.ld, F.kt[a], nrhs);
    off += F.kt[a];
  }
  run_copy(c, cb, up ? "root gather" : "root scatter");
}

// x <- R^{-1} x (or R^{-H} x) with the blocked LU of the final block
void root_solve(Ctx& c, char* x, int ld, int nrhs, bool adjoint) {
  RootF& R = c.root;
  const int n = R.n, nb = R.nb, prec = c.prec;
  if (n == 0) return;
  const size_t es = esz(prec);
  char* Rm = (char*)R.R.p;
  char* Li = (char*)R.Linv.p;
  char* Ui = (char*)R.Uinv.p;
  const int npan = (n + nb - 1) / nb;
  auto panel = [&](int pi, int& k0, int& kb) { k0 = pi * nb; kb = std::min(nb, n - k0); };
  if (!adjoint) {
    ck(swap_rows(x, ld, (const int*)R.piv.p, 0, n, 0, nrhs, prec, 0, c.stream), "root swaps");
    c.launches++;
    for (int pi = 0; pi < npan; ++pi) {
      int k0, kb;
      panel(pi, k0, kb);
      ApplyBatch ab;
      ab.add(Li + (size_t)pi * nb * nb * es, kb, OP_N, x + (size_t)k0 * es, ld, kb, nrhs, 0);
      run_apply(c, ab, true, prec, "root fwd");
      const int rest = n - k0 - kb;
      if (rest > 0) {
        GemmBatch g;
        g.task(x + (size_t)(k0 + kb) * es, ld, rest, nrhs, -1.0, 1.0);
        g.pair(Rm + ((size_t)(k0 + kb) + (size_t)k0 * n) * es, n, OP_N, x + (size_t)k0 * es, ld, OP_N, kb);
        g.close();
        run_gemm(c, g, prec, prec, prec, "root fwd update");
      }
    }
    for (int pi = npan - 1; pi >= 0; --pi) {
      int k0, kb;
      panel(pi, k0, kb);
      const int rest = n - k0 - kb;
      if (rest > 0) {
        GemmBatch g;
        g.task(x + (size_t)k0 * es, ld, kb, nrhs, -1.0, 1.0);
        g.pair(Rm + ((size_t)k0 + (size_t)(k0 + kb) * n) * es, n, OP_N, x + (size_t)(k0 + kb) * es, ld, OP_N, rest);
        g.close();
        run_gemm(c, g, prec, prec, prec, "root bwd update");
      }
      ApplyBatch ab;
      ab.add(Ui + (size_t)pi * nb * nb * es, kb, OP_N, x + (size_t)k0 * es, ld, kb, nrhs, 0);
      run_apply(c, ab, true, prec, "root bwd");
    }
  } else {
    // R = P^T L U  ->  R^{-H} = P^T L^{-H} U^{-H}
    for (int pi = 0; pi < npan; ++pi) {
      int k0, kb;
      panel(pi, k0, kb);
      ApplyBatch ab;
      ab.add(Ui + (size_t)pi * nb * nb * es, kb, OP_H, x + (size_t)k0 * es, ld, kb, nrhs, 0);
      run_apply(c, ab, true, prec, "root adj U");
      const int rest = n - k0 - kb;
      if (rest > 0) {
        GemmBatch g;
        g.task(x + (size_t)(k0 + kb) * es, ld, rest, nrhs, -1.0, 1.0);
        g.pair(Rm + ((size_t)k0 + (size_t)(k0 + kb) * n) * es, n, OP_H, x + (size_t)k0 * es, ld, OP_N, kb);
        g.close();
        run_gemm(c, g, prec, prec, prec, "root adj U update");
      }
    }
    for (int pi = npan - 1; pi >= 0; --pi) {
      int k0, kb;
      panel(pi, k0, kb);
      const int rest = n - k0 - kb;
      if (rest > 0) {
        GemmBatch g;
        g.task(x + (size_t)k0 * es, ld, kb, nrhs, -1.0, 1.0);
        g.pair(Rm + ((size_t)(k0 + kb) + (size_t)k0 * n) * es, n, OP_H, x + (size_t)(k0 + kb) * es, ld, OP_N, rest);
        g.close();
        run_gemm(c, g, prec, prec, prec, "root adj L update");
      }
      ApplyBatch ab;
      ab.add(Li + (size_t)pi * nb * nb * es, kb, OP_H, x + (size_t)k0 * es, ld, kb, nrhs, 0);
      run_apply(c, ab, true, prec, "root adj L");
    }
    ck(swap_rows(x, ld, (const int*)R.piv.p, 0, n, 0, nrhs, prec, 1, c.stream), "root swaps");
    c.launches++;
  }
}

}  // namespace

void root_solve_public(Ctx& c, char* x, int ld, int nrhs, bool adjoint) { root_solve(c, x, ld, nrhs, adjoint); }

void solve_tree(Ctx& c, void* xv, int nrhs, bool adjoint, bool use_inverse) {
  if (!c.factored) fail(H2_ESTATE, "solve before factorize");
  const int prec = c.prec;
  const size_t es = esz(prec);
  const int nlev = (int)c.lev.size();
  // level vectors: level 0 is x itself (tree order, ld N)
  std::vector<Vec> vec(nlev);
  size_t tot = 0;
  std::vector<size_t> off(nlev, 0);
  for (int li = 1; li < nlev; ++li) {
    off[li] = tot;
    tot += (size_t)c.lev[li].vlen * nrhs;
  }
  const size_t roff = tot;
  tot += (size_t)c.root.n * nrhs;
  char* buf = (char*)dev_ensure(c, c.vecbuf, (tot + 1) * es);
  vec[0] = Vec{(char*)xv, c.H.tree.N};
  for (int li = 1; li < nlev; ++li) vec[li] = Vec{buf + off[li] * es, c.lev[li].vlen};
  Vec vr{buf + roff * es, c.root.n};

  auto Q = [&](const LevelF& F, int i) { return (char*)F.Q_buf.p + F.Q_off[i] * es; };
  auto Linv = [&](const LevelF& F, int i) { return (char*)F.inv_buf.p + F.inv_off[i] * es; };
  auto Uinv = [&](const LevelF& F, int i) {
    return (char*)F.inv_buf.p + (F.inv_off[i] + (size_t)F.n[i] * F.n[i]) * es;
  };
  auto seg = [&](const Vec& v, const LevelF& F, int i, int r0) { return v.p + (size_t)(F.voff[i] + r0) * es; };

  if (!adjoint) {
    // ---------------- forward: L y = b (Algorithm 5) ----------------
    for (int li = 0; li < nlev; ++li) {
      LevelF& F = c.lev[li];
      Vec v = vec[li];
      for (const auto& bt : F.batches) {
        ApplyBatch a1, a2;
        for (int i : bt) {
          a1.add(Q(F, i), F.n[i], OP_H, seg(v, F, i, 0), (int)v.ld, F.n[i], nrhs, 0);
          if (F.m[i] > 0) a2.add(Linv(F, i), F.m[i], OP_N, seg(v, F, i, 0), (int)v.ld, F.m[i], nrhs, 0);
        }
        run_apply_narrow(c, a1, prec, "fwd Q^H");
        run_apply_narrow(c, a2, prec, "fwd L^-1");
        std::map<int, std::vector<int>> tg;
        for (int i : bt)
          if (F.m[i] > 0)
            for (int j : F.nbrs[i]) tg[j].push_back(i);
        GemmBatch g;
        for (auto& [j, cl] : tg) {
          const int rlo = lo_at(F, j, cl[0]);
          g.task(seg(v, F, j, rlo), (int)v.ld, F.n[j] - rlo, nrhs, -1.0, 1.0);
          for (int i : cl) g.pair(NBp(c, F, j, i) + (size_t)rlo * es, F.n[j], OP_N, seg(v, F, i, 0), (int)v.ld, OP_N, F.m[i]);
          g.close();
        }
        run_gemm(c, g, prec, prec, prec, "fwd update");
      }
      if (li + 1 < nlev) merge_vec(c, F, c.lev[li + 1], v, vec[li + 1], nrhs, true);
    }
    root_vec(c, c.lev[nlev - 1], vec[nlev - 1], vr, nrhs, true);
    if (use_inverse && c.root.n > 0) {
      char* tmp = (char*)dev_ensure(c, c.vecbuf2, (size_t)c.root.n * nrhs * es);
      GemmBatch g;
      g.task(tmp, c.root.n, c.root.n, nrhs, 1.0, 0.0);
      g.pair(c.root.Rinv.p, c.root.n, OP_N, vr.p, (int)vr.ld, OP_N, c.root.n);
      g.close();
      run_gemm(c, g, prec, prec, prec, "root inverse apply");
      CopyBatch cb;
      cb.add(tmp, prec, c.root.n, c.root.n, nrhs, vr.p, prec, (int)vr.ld, c.root.n, nrhs);
      run_copy(c, cb, "root inverse copy");
    } else {
      root_solve(c, vr.p, (int)vr.ld, nrhs, false);
    }
    root_vec(c, c.lev[nlev - 1], vec[nlev - 1], vr, nrhs, false);
    // ---------------- backward: U x = y (Algorithm 6) ----------------
    for (int li = nlev - 1; li >= 0; --li) {
      LevelF& F = c.lev[li];
      Vec v = vec[li];
      for (int b = (int)F.batches.size() - 1; b >= 0; --b) {
        const auto& bt = F.batches[b];
        GemmBatch g;
        ApplyBatch a1, a2;
        for (int i : bt) {
          const int mi = F.m[i];
          if (mi <= 0) continue;
          if (!use_inverse) {
            g.task(seg(v, F, i, 0), (int)v.ld, mi, nrhs, -1.0, 1.0);
            for (int k : F.nbrs[i]) {
              const int clo = lo_at(F, k, i);
              g.pair(NBp(c, F, i, k) + (size_t)clo * F.n[i] * es, F.n[i], OP_N, seg(v, F, k, clo), (int)v.ld, OP_N,
                     F.n[k] - clo);
            }
            g.close();
          } else {
            // eq. (35): x_i' = U^{-1} x_i' + sum_k (-U^{-1} U_ik) x_k
            g.task(seg(v, F, i, 0), (int)v.ld, mi, nrhs, 1.0, 1.0);
            for (size_t q = 0; q < F.nbrs[i].size(); ++q) {
              const int k = F.nbrs[i][q];
              const int clo = lo_at(F, k, i);
              g.pair((char*)F.Ub_buf.p + F.Ub_off[F.nbr_first[i] + q] * es, mi, OP_N, seg(v, F, k, clo), (int)v.ld,
                     OP_N, F.n[k] - clo);
            }
            g.close();
          }
          a1.add(Uinv(F, i), mi, OP_N, seg(v, F, i, 0), (int)v.ld, mi, nrhs, 0);
        }
        if (!use_inverse) {
          run_gemm(c, g, prec, prec, prec, "bwd update");
          run_apply_narrow(c, a1, prec, "bwd U^-1");
        } else {
          run_apply_narrow(c, a1, prec, "inv U^-1");
          run_gemm(c, g, prec, prec, prec, "inv update");
        }
        for (int i : bt) a2.add(Q(F, i), F.n[i], OP_C, seg(v, F, i, 0), (int)v.ld, F.n[i], nrhs, 0);
        run_apply_narrow(c, a2, prec, "bwd conj Q");
      }
      if (li > 0) merge_vec(c, c.lev[li - 1], F, vec[li - 1], v, nrhs, false);
    }
  } else {
    // ------------- adjoint: Z^{-H} = (U^{-1}-part)^H then (L^{-1}-part)^H -------------
    for (int li = 0; li < nlev; ++li) {
      LevelF& F = c.lev[li];
      Vec v = vec[li];
      for (const auto& bt : F.batches) {
        ApplyBatch a1, a2;
        for (int i : bt) {
          a1.add(Q(F, i), F.n[i], OP_T, seg(v, F, i, 0), (int)v.ld, F.n[i], nrhs, 0);
          if (F.m[i] > 0) a2.add(Uinv(F, i), F.m[i], OP_H, seg(v, F, i, 0), (int)v.ld, F.m[i], nrhs, 0);
        }
        run_apply_narrow(c, a1, prec, "adj Q^T");
        run_apply_narrow(c, a2, prec, "adj U^-H");
        std::map<int, std::vector<int>> tg;
        for (int i : bt)
          if (F.m[i] > 0)
            for (int k : F.nbrs[i]) tg[k].push_back(i);
        GemmBatch g;
        for (auto& [k, cl] : tg) {
          const int clo = lo_at(F, k, cl[0]);
          g.task(seg(v, F, k, clo), (int)v.ld, F.n[k] - clo, nrhs, -1.0, 1.0);
          for (int i : cl)
            g.pair(NBp(c, F, i, k) + (size_t)clo * F.n[i] * es, F.n[i], OP_H, seg(v, F, i, 0), (int)v.ld, OP_N, F.m[i]);
          g.close();
        }
        run_gemm(c, g, prec, prec, prec, "adj U^H update");
      }
      if (li + 1 < nlev) merge_vec(c, F, c.lev[li + 1], v, vec[li + 1], nrhs, true);
    }
    root_vec(c, c.lev[nlev - 1], vec[nlev - 1], vr, nrhs, true);
    root_solve(c, vr.p, (int)vr.ld, nrhs, true);
    root_vec(c, c.lev[nlev - 1], vec[nlev - 1], vr, nrhs, false);
    for (int li = nlev - 1; li >= 0; --li) {
      LevelF& F = c.lev[li];
      Vec v = vec[li];
      for (int b = (int)F.batches.size() - 1; b >= 0; --b) {
        const auto& bt = F.batches[b];
        GemmBatch g;
        ApplyBatch a1, a2;
        for (int i : bt) {
          const int mi = F.m[i];
          if (mi > 0) {
            g.task(seg(v, F, i, 0), (int)v.ld, mi, nrhs, -1.0, 1.0);
            for (int j : F.nbrs[i]) {
              const int rlo = lo_at(F, j, i);
              g.pair(NBp(c, F, j, i) + (size_t)rlo * es, F.n[j], OP_H, seg(v, F, j, rlo), (int)v.ld, OP_N, F.n[j] - rlo);
            }
            g.close();
            a1.add(Linv(F, i), mi, OP_H, seg(v, F, i, 0), (int)v.ld, mi, nrhs, 0);
          }
          a2.add(Q(F, i), F.n[i], OP_N, seg(v, F, i, 0), (int)v.ld, F.n[i], nrhs, 0);
        }
        run_gemm(c, g, prec, prec, prec, "adj L^H update");
        run_apply_narrow(c, a1, prec, "adj L^-H");
        run_apply_narrow(c, a2, prec, "adj Q");
      }
      if (li > 0) merge_vec(c, c.lev[li - 1], F, vec[li - 1], v, nrhs, false);
    }
  }
}

}  // namespace h2
