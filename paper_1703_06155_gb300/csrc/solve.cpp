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

// x_c <- R_c^{-1} x_c (or R_c^{-H} x_c) with the blocked LU of the final block
// of every instance c; panel step pi of all instances shares the launches.
void root_solve_group(Ctx& lc, const std::vector<Ctx*>& cs, const std::vector<char*>& xs,
                      const std::vector<int>& lds, int nrhs, bool adjoint) {
  const int prec = lc.prec;
  const size_t es = esz(prec);
  int npan_max = 0;
  for (Ctx* c : cs)
    if (c->root.n > 0) npan_max = std::max(npan_max, (c->root.n + c->root.nb - 1) / c->root.nb);
  if (npan_max == 0) return;
  auto swaps = [&](int reverse) {
    std::vector<SwapTask> sw;
    for (size_t q = 0; q < cs.size(); ++q)
      if (cs[q]->root.n > 0)
        sw.push_back(SwapTask{xs[q], (const int*)cs[q]->root.piv.p, lds[q], 0, cs[q]->root.n, 0, nrhs, reverse});
    const int i0 = lc.st.add(sw);
    lc.st.upload(lc);
    ck(swap_rows_batch(lc.st.ptr<SwapTask>(i0), (int)sw.size(), prec, lc.stream), "root swaps");
    lc.launches++;
  };
  // step(pi, kind) adds instance q's work of panel pi to the batches
  auto panel = [&](size_t q, int pi, int& k0, int& kb) {
    const RootF& R = cs[q]->root;
    k0 = pi * R.nb;
    kb = std::min(R.nb, R.n - k0);
    return k0 < R.n;
  };
  auto rm = [&](size_t q) { return (char*)cs[q]->root.R.p; };
  auto li = [&](size_t q, int pi) { return (char*)cs[q]->root.Linv.p + (size_t)pi * cs[q]->root.nb * cs[q]->root.nb * es; };
  auto ui = [&](size_t q, int pi) { return (char*)cs[q]->root.Uinv.p + (size_t)pi * cs[q]->root.nb * cs[q]->root.nb * es; };
  if (!adjoint) {
    swaps(0);
    for (int pi = 0; pi < npan_max; ++pi) {
      ApplyBatch ab;
      GemmBatch g;
      for (size_t q = 0; q < cs.size(); ++q) {
        int k0, kb;
        if (!panel(q, pi, k0, kb)) continue;
        const int n = cs[q]->root.n, ld = lds[q];
        char* x = xs[q];
        ab.add(li(q, pi), kb, OP_N, x + (size_t)k0 * es, ld, kb, nrhs, 0);
        const int rest = n - k0 - kb;
        if (rest > 0) {
          g.task(x + (size_t)(k0 + kb) * es, ld, rest, nrhs, -1.0, 1.0);
          g.pair(rm(q) + ((size_t)(k0 + kb) + (size_t)k0 * n) * es, n, OP_N, x + (size_t)k0 * es, ld, OP_N, kb);
          g.close();
        }
      }
      run_apply(lc, ab, true, prec, "root fwd");
      run_gemm(lc, g, prec, prec, prec, "root fwd update");
    }
    for (int pi = npan_max - 1; pi >= 0; --pi) {
      ApplyBatch ab;
      GemmBatch g;
      for (size_t q = 0; q < cs.size(); ++q) {
        int k0, kb;
        if (!panel(q, pi, k0, kb)) continue;
        const int n = cs[q]->root.n, ld = lds[q];
        char* x = xs[q];
        const int rest = n - k0 - kb;
        if (rest > 0) {
          g.task(x + (size_t)k0 * es, ld, kb, nrhs, -1.0, 1.0);
          g.pair(rm(q) + ((size_t)k0 + (size_t)(k0 + kb) * n) * es, n, OP_N, x + (size_t)(k0 + kb) * es, ld, OP_N,
                 rest);
          g.close();
        }
        ab.add(ui(q, pi), kb, OP_N, x + (size_t)k0 * es, ld, kb, nrhs, 0);
      }
      run_gemm(lc, g, prec, prec, prec, "root bwd update");
      run_apply(lc, ab, true, prec, "root bwd");
    }
  } else {
    // R = P^T L U  ->  R^{-H} = P^T L^{-H} U^{-H}
    for (int pi = 0; pi < npan_max; ++pi) {
      ApplyBatch ab;
      GemmBatch g;
      for (size_t q = 0; q < cs.size(); ++q) {
        int k0, kb;
        if (!panel(q, pi, k0, kb)) continue;
        const int n = cs[q]->root.n, ld = lds[q];
        char* x = xs[q];
        ab.add(ui(q, pi), kb, OP_H, x + (size_t)k0 * es, ld, kb, nrhs, 0);
        const int rest = n - k0 - kb;
        if (rest > 0) {
          g.task(x + (size_t)(k0 + kb) * es, ld, rest, nrhs, -1.0, 1.0);
          g.pair(rm(q) + ((size_t)k0 + (size_t)(k0 + kb) * n) * es, n, OP_H, x + (size_t)k0 * es, ld, OP_N, kb);
          g.close();
        }
      }
      run_apply(lc, ab, true, prec, "root adj U");
      run_gemm(lc, g, prec, prec, prec, "root adj U update");
    }
    for (int pi = npan_max - 1; pi >= 0; --pi) {
      ApplyBatch ab;
      GemmBatch g;
      for (size_t q = 0; q < cs.size(); ++q) {
        int k0, kb;
        if (!panel(q, pi, k0, kb)) continue;
        const int n = cs[q]->root.n, ld = lds[q];
        char* x = xs[q];
        const int rest = n - k0 - kb;
        if (rest > 0) {
          g.task(x + (size_t)k0 * es, ld, kb, nrhs, -1.0, 1.0);
          g.pair(rm(q) + ((size_t)(k0 + kb) + (size_t)k0 * n) * es, n, OP_H, x + (size_t)(k0 + kb) * es, ld, OP_N,
                 rest);
          g.close();
        }
        ab.add(li(q, pi), kb, OP_H, x + (size_t)k0 * es, ld, kb, nrhs, 0);
      }
      run_gemm(lc, g, prec, prec, prec, "root adj L update");
      run_apply(lc, ab, true, prec, "root adj L");
    }
    swaps(1);
  }
}

}  // namespace

void root_solve_grouped(Ctx& lc, const std::vector<Ctx*>& cs, const std::vector<char*>& xs,
                        const std::vector<int>& lds, int nrhs, bool adjoint) {
  root_solve_group(lc, cs, xs, lds, nrhs, adjoint);
}

// One instance's level vectors for a solve
struct SolveVecs {
  std::vector<Vec> vec;  // vec[0] = x itself (tree order, ld N)
  Vec vr;                // final-block vector
  Vec vt;                // block LDL^T: F^{-1} y of the batch's clusters
};

// Forward (Algorithm 5) / backward (Algorithm 6) substitution, or the adjoint
// traversal, for a group of instances: level-from-leaf index d and colour b
// of every instance share the launches.  xs[q]: instance q's vector in tree
// order (bulk precision, N x nrhs).
static void solve_tree_sweeps(const std::vector<Ctx*>& cs, const std::vector<void*>& xs, int nrhs, bool adjoint,
                              bool use_inverse) {
  Ctx& lc = *cs[0];
  const int prec = lc.prec;
  const size_t es = esz(prec);
  const size_t nq = cs.size();
  std::vector<SolveVecs> sv(nq);
  int depth = 0;
  for (size_t q = 0; q < nq; ++q) {
    Ctx& c = *cs[q];
    if (!c.factored) fail(H2_ESTATE, "solve before factorize");
    if (c.prec != prec) fail(H2_EINVAL, "instances factorized in different precisions");
    const int nlev = (int)c.lev.size();
    depth = std::max(depth, nlev);
    std::vector<size_t> off(nlev, 0);
    size_t tot = 0;
    for (int li = 1; li < nlev; ++li) {
      off[li] = tot;
      tot += (size_t)c.lev[li].vlen * nrhs;
    }
    const size_t roff = tot;
    tot += (size_t)c.root.n * nrhs;
    // block LDL^T: F^{-1} y_i' of a batch, laid out like a level vector
    int64_t tld = 0;
    if (c.fac_ldlt)
      for (const LevelF& F : c.lev) tld = std::max(tld, F.vlen);
    const size_t toff = tot;
    tot += (size_t)tld * nrhs;
    char* buf = (char*)dev_ensure(c, c.vecbuf, (tot + 1) * es);
    sv[q].vec.resize(nlev);
    sv[q].vec[0] = Vec{(char*)xs[q], c.H.tree.N};
    for (int li = 1; li < nlev; ++li) sv[q].vec[li] = Vec{buf + off[li] * es, c.lev[li].vlen};
    sv[q].vr = Vec{buf + roff * es, c.root.n};
    sv[q].vt = Vec{buf + toff * es, tld};
    if (adjoint && c.fac_ldlt) fail(H2_EINTERNAL, "block LDL^T factors: adjoint sweeps are not used");
  }
  auto has = [&](size_t q, int d) { return d < (int)cs[q]->lev.size(); };
  auto top = [&](size_t q) { return (int)cs[q]->lev.size() - 1; };
  auto Q = [&](const LevelF& F, int i) { return (char*)F.Q_buf.p + F.Q_off[i] * es; };
  auto Linv = [&](const LevelF& F, int i) { return (char*)F.inv_buf.p + F.inv_off[i] * es; };
  auto Uinv = [&](const LevelF& F, int i) {
    return (char*)F.inv_buf.p + (F.inv_off[i] + (size_t)F.n[i] * F.n[i]) * es;
  };
  auto seg = [&](const Vec& v, const LevelF& F, int i, int r0) { return v.p + (size_t)(F.voff[i] + r0) * es; };
  auto nbat = [&](int d) {
    size_t nb = 0;
    for (size_t q = 0; q < nq; ++q)
      if (has(q, d)) nb = std::max(nb, cs[q]->lev[d].batches.size());
    return (int)nb;
  };
  // children -> parent (up) or parent -> children (down) between level d and d+1
  auto merge = [&](int d, bool up) {
    CopyBatch cb;
    for (size_t q = 0; q < nq; ++q) {
      if (!has(q, d + 1)) continue;
      const LevelF& F = cs[q]->lev[d];
      const LevelF& Pn = cs[q]->lev[d + 1];
      const Vec v = sv[q].vec[d], vp = sv[q].vec[d + 1];
      for (int p = 0; p < Pn.nc; ++p)
        for (int a = 2 * p; a <= 2 * p + 1; ++a) {
          const int o = (a & 1) ? F.kt[a - 1] : 0;
          char* child = v.p + (size_t)(F.voff[a] + F.m[a]) * es;
          char* par = vp.p + (size_t)(Pn.voff[p] + o) * es;
          if (up) cb.add(child, prec, (int)v.ld, F.kt[a], nrhs, par, prec, (int)vp.ld, F.kt[a], nrhs);
          else cb.add(par, prec, (int)vp.ld, F.kt[a], nrhs, child, prec, (int)v.ld, F.kt[a], nrhs);
        }
    }
    run_copy(lc, cb, up ? "vec merge" : "vec scatter");
  };
  // kept parts of the top level <-> final-block vector
  auto rootvec = [&](bool up) {
    CopyBatch cb;
    for (size_t q = 0; q < nq; ++q) {
      const LevelF& F = cs[q]->lev.back();
      const Vec v = sv[q].vec[top(q)], vr = sv[q].vr;
      int off = 0;
      for (int a = 0; a < F.nc; ++a) {
        char* lv = v.p + (size_t)(F.voff[a] + F.m[a]) * es;
        char* rv = vr.p + (size_t)off * es;
        if (up) cb.add(lv, prec, (int)v.ld, F.kt[a], nrhs, rv, prec, (int)vr.ld, F.kt[a], nrhs);
        else cb.add(rv, prec, (int)vr.ld, F.kt[a], nrhs, lv, prec, (int)v.ld, F.kt[a], nrhs);
        off += F.kt[a];
      }
    }
    run_copy(lc, cb, up ? "root gather" : "root scatter");
  };
  // final block: x_r <- R^{-1} x_r (R^{-H} for the adjoint) with the explicit
  // inverse formed at factorization time: one GEMM for all instances
  auto root = [&](bool adj) {
    GemmBatch g;
    CopyBatch cb;
    for (size_t q = 0; q < nq; ++q) {
      Ctx& c = *cs[q];
      const int n = c.root.n;
      if (n == 0) continue;
      char* tmp = (char*)dev_ensure(c, c.vecbuf2, (size_t)n * nrhs * es);
      g.task(tmp, n, n, nrhs, 1.0, 0.0);
      g.pair(c.root.Rinv.p, n, adj ? OP_H : OP_N, sv[q].vr.p, (int)sv[q].vr.ld, OP_N, n);
      g.close();
      cb.add(tmp, prec, n, n, nrhs, sv[q].vr.p, prec, (int)sv[q].vr.ld, n, nrhs);
    }
    run_gemm(lc, g, prec, prec, prec, adj ? "root inverse^H apply" : "root inverse apply");
    run_copy(lc, cb, "root inverse copy");
  };

  if (!adjoint) {
    // ---------------- forward: L y = b (Algorithm 5) ----------------
    for (int d = 0; d < depth; ++d) {
      for (int b = 0; b < nbat(d); ++b) {
        ApplyBatch a1, a2, at;
        GemmBatch g, gt;
        for (size_t q = 0; q < nq; ++q) {
          if (!has(q, d) || b >= (int)cs[q]->lev[d].batches.size()) continue;
          Ctx& c = *cs[q];
          const LevelF& F = c.lev[d];
          const Vec v = sv[q].vec[d], vt = sv[q].vt;
          const auto& bt = F.batches[b];
          for (int i : bt) {
            a1.add(Q(F, i), F.n[i], OP_H, seg(v, F, i, 0), (int)v.ld, F.n[i], nrhs, 0);
            if (F.m[i] <= 0) continue;
            if (!F.sym) {
              a2.add(Linv(F, i), F.m[i], OP_N, seg(v, F, i, 0), (int)v.ld, F.m[i], nrhs, 0);
            } else {
              // block LDL^T: t_i = F^{-1} y_i' = U^{-1} (L^{-1}P y_i'); y_i' stays
              gt.task(seg(vt, F, i, 0), (int)vt.ld, F.m[i], nrhs, 1.0, 0.0);
              gt.pair(Linv(F, i), F.m[i], OP_N, seg(v, F, i, 0), (int)v.ld, OP_N, F.m[i]);
              gt.close();
              at.add(Uinv(F, i), F.m[i], OP_N, seg(vt, F, i, 0), (int)vt.ld, F.m[i], nrhs, 0);
            }
          }
          std::map<int, std::vector<int>> tg;
          for (int i : bt)
            if (F.m[i] > 0)
              for (int j : F.nbrs[i]) tg[j].push_back(i);
          for (auto& [j, cl] : tg) {
            const int rlo = lo_at(F, j, cl[0]);
            g.task(seg(v, F, j, rlo), (int)v.ld, F.n[j] - rlo, nrhs, -1.0, 1.0);
            for (int i : cl) {
              if (!F.sym)
                g.pair(NBp(c, F, j, i) + (size_t)rlo * es, F.n[j], OP_N, seg(v, F, i, 0), (int)v.ld, OP_N, F.m[i]);
              else if (j > i)  // Z_ji' = the stored (i, j) transposed
                g.pair(NBp(c, F, j, i) + (size_t)rlo * F.n[i] * es, F.n[i], OP_T, seg(vt, F, i, 0), (int)vt.ld,
                       OP_N, F.m[i]);
              else
                g.pair(NBp(c, F, j, i) + (size_t)rlo * es, F.n[j], OP_N, seg(vt, F, i, 0), (int)vt.ld, OP_N,
                       F.m[i]);
            }
            g.close();
          }
        }
        run_apply_narrow(lc, a1, prec, "fwd Q^H");
        run_apply_narrow(lc, a2, prec, "fwd L^-1");
        run_gemm(lc, gt, prec, prec, prec, "fwd L^-1 y");
        run_apply_narrow(lc, at, prec, "fwd U^-1 y");
        run_gemm(lc, g, prec, prec, prec, "fwd update");
      }
      merge(d, true);
    }
    rootvec(true);
    root(false);
    rootvec(false);
    // ---------------- backward: U x = y (Algorithm 6) ----------------
    for (int d = depth - 1; d >= 0; --d) {
      for (int b = nbat(d) - 1; b >= 0; --b) {
        GemmBatch g;
        ApplyBatch a0, a1, a2;
        for (size_t q = 0; q < nq; ++q) {
          if (!has(q, d) || b >= (int)cs[q]->lev[d].batches.size()) continue;
          Ctx& c = *cs[q];
          const LevelF& F = c.lev[d];
          const Vec v = sv[q].vec[d];
          const auto& bt = F.batches[b];
          for (int i : bt) {
            const int mi = F.m[i];
            if (mi <= 0) continue;
            if (!use_inverse) {
              // LU: y_i' -= (L^{-1}P Z_i'k) x_k; block LDL^T: y_i' -= Z_i'k x_k
              g.task(seg(v, F, i, 0), (int)v.ld, mi, nrhs, -1.0, 1.0);
              for (int k : F.nbrs[i]) {
                const int clo = lo_at(F, k, i);
                if (F.sym && i > k)  // the stored (k, i) transposed
                  g.pair(NBp(c, F, i, k) + (size_t)clo * es, F.n[k], OP_T, seg(v, F, k, clo), (int)v.ld, OP_N,
                         F.n[k] - clo);
                else
                  g.pair(NBp(c, F, i, k) + (size_t)clo * F.n[i] * es, F.n[i], OP_N, seg(v, F, k, clo), (int)v.ld,
                         OP_N, F.n[k] - clo);
              }
              g.close();
            } else {
              // eq. (35): x_i' = U^{-1} x_i' + sum_k (-U^{-1} U_ik) x_k
              g.task(seg(v, F, i, 0), (int)v.ld, mi, nrhs, 1.0, 1.0);
              for (size_t u = 0; u < F.nbrs[i].size(); ++u) {
                const int k = F.nbrs[i][u];
                const int clo = lo_at(F, k, i);
                g.pair((char*)F.Ub_buf.p + F.Ub_off[F.nbr_first[i] + u] * es, mi, OP_N, seg(v, F, k, clo),
                       (int)v.ld, OP_N, F.n[k] - clo);
              }
              g.close();
            }
            // x_i' = U^{-1} (...) (LU) or F^{-1} (...) = U^{-1} L^{-1}P (...) (block LDL^T)
            if (F.sym) a0.add(Linv(F, i), mi, OP_N, seg(v, F, i, 0), (int)v.ld, mi, nrhs, 0);
            a1.add(Uinv(F, i), mi, OP_N, seg(v, F, i, 0), (int)v.ld, mi, nrhs, 0);
          }
          for (int i : bt) a2.add(Q(F, i), F.n[i], OP_C, seg(v, F, i, 0), (int)v.ld, F.n[i], nrhs, 0);
        }
        if (!use_inverse) {
          run_gemm(lc, g, prec, prec, prec, "bwd update");
          run_apply_narrow(lc, a0, prec, "bwd L^-1");
          run_apply_narrow(lc, a1, prec, "bwd U^-1");
        } else {
          run_apply_narrow(lc, a0, prec, "inv L^-1");
          run_apply_narrow(lc, a1, prec, "inv U^-1");
          run_gemm(lc, g, prec, prec, prec, "inv update");
        }
        run_apply_narrow(lc, a2, prec, "bwd conj Q");
      }
      if (d > 0) merge(d - 1, false);
    }
  } else {
    // ------------- adjoint: Z^{-H} = (U^{-1}-part)^H then (L^{-1}-part)^H -------------
    for (int d = 0; d < depth; ++d) {
      for (int b = 0; b < nbat(d); ++b) {
        ApplyBatch a1, a2;
        GemmBatch g;
        for (size_t q = 0; q < nq; ++q) {
          if (!has(q, d) || b >= (int)cs[q]->lev[d].batches.size()) continue;
          Ctx& c = *cs[q];
          const LevelF& F = c.lev[d];
          const Vec v = sv[q].vec[d];
          const auto& bt = F.batches[b];
          for (int i : bt) {
            a1.add(Q(F, i), F.n[i], OP_T, seg(v, F, i, 0), (int)v.ld, F.n[i], nrhs, 0);
            if (F.m[i] > 0) a2.add(Uinv(F, i), F.m[i], OP_H, seg(v, F, i, 0), (int)v.ld, F.m[i], nrhs, 0);
          }
          std::map<int, std::vector<int>> tg;
          for (int i : bt)
            if (F.m[i] > 0)
              for (int k : F.nbrs[i]) tg[k].push_back(i);
          for (auto& [k, cl] : tg) {
            const int clo = lo_at(F, k, cl[0]);
            g.task(seg(v, F, k, clo), (int)v.ld, F.n[k] - clo, nrhs, -1.0, 1.0);
            for (int i : cl)
              g.pair(NBp(c, F, i, k) + (size_t)clo * F.n[i] * es, F.n[i], OP_H, seg(v, F, i, 0), (int)v.ld, OP_N,
                     F.m[i]);
            g.close();
          }
        }
        run_apply_narrow(lc, a1, prec, "adj Q^T");
        run_apply_narrow(lc, a2, prec, "adj U^-H");
        run_gemm(lc, g, prec, prec, prec, "adj U^H update");
      }
      merge(d, true);
    }
    rootvec(true);
    root(true);
    rootvec(false);
    for (int d = depth - 1; d >= 0; --d) {
      for (int b = nbat(d) - 1; b >= 0; --b) {
        GemmBatch g;
        ApplyBatch a1, a2;
        for (size_t q = 0; q < nq; ++q) {
          if (!has(q, d) || b >= (int)cs[q]->lev[d].batches.size()) continue;
          Ctx& c = *cs[q];
          const LevelF& F = c.lev[d];
          const Vec v = sv[q].vec[d];
          const auto& bt = F.batches[b];
          for (int i : bt) {
            const int mi = F.m[i];
            if (mi > 0) {
              g.task(seg(v, F, i, 0), (int)v.ld, mi, nrhs, -1.0, 1.0);
              for (int j : F.nbrs[i]) {
                const int rlo = lo_at(F, j, i);
                g.pair(NBp(c, F, j, i) + (size_t)rlo * es, F.n[j], OP_H, seg(v, F, j, rlo), (int)v.ld, OP_N,
                       F.n[j] - rlo);
              }
              g.close();
              a1.add(Linv(F, i), mi, OP_H, seg(v, F, i, 0), (int)v.ld, mi, nrhs, 0);
            }
            a2.add(Q(F, i), F.n[i], OP_N, seg(v, F, i, 0), (int)v.ld, F.n[i], nrhs, 0);
          }
        }
        run_gemm(lc, g, prec, prec, prec, "adj L^H update");
        run_apply_narrow(lc, a1, prec, "adj L^-H");
        run_apply_narrow(lc, a2, prec, "adj Q");
      }
      if (d > 0) merge(d - 1, false);
    }
  }
}

// With h2_opts.solve_graph the sweeps of a given (instances, vectors, nrhs,
// direction) are run normally once with the graph's own staging buffers,
// captured into a CUDA graph on the second call and replayed afterwards; any
// device (re)allocation or refactorization of an instance retires the graph.
void solve_tree_group(const std::vector<Ctx*>& cs, const std::vector<void*>& xs, int nrhs, bool adjoint,
                      bool use_inverse) {
  Ctx& lc = *cs[0];
  if (!lc.opts.solve_graph) {
    solve_tree_sweeps(cs, xs, nrhs, adjoint, use_inverse);
    return;
  }
  SolveGraph* g = nullptr;
  for (auto& u : lc.graphs)
    if (u->cs == cs && u->xs == xs && u->nrhs == nrhs && u->adjoint == adjoint && u->inverse == use_inverse) {
      g = u.get();
      break;
    }
  auto state = [&](std::vector<uint64_t>& gens, std::vector<uint64_t>& epochs) {
    gens.clear();
    epochs.clear();
    for (Ctx* c : cs) {
      gens.push_back(c->gen);
      epochs.push_back(c->epoch);
    }
  };
  std::vector<uint64_t> gens, epochs;
  state(gens, epochs);
  if (g && g->exec && g->gens == gens && g->epochs == epochs) {
    ProfScope ps(lc, "solve graph", 0.0);
    ck(cudaGraphLaunch(g->exec, lc.stream), "graph launch");
    lc.launches += g->nlaunch;
    return;
  }
  if (!g || g->gens != gens || g->epochs != epochs) {
    // first call (or stale): run normally with the graph's staging buffers
    if (!g) {
      if (lc.graphs.size() >= 8) lc.graphs.erase(lc.graphs.begin());
      lc.graphs.push_back(std::make_unique<SolveGraph>());
      g = lc.graphs.back().get();
      g->cs = cs;
      g->xs = xs;
      g->nrhs = nrhs;
      g->adjoint = adjoint;
      g->inverse = use_inverse;
    }
    if (g->exec) {
      cudaGraphExecDestroy(g->exec);
      g->exec = nullptr;
    }
    lc.st.swap(g->st);
    try {
      lc.st.begin();
      solve_tree_sweeps(cs, xs, nrhs, adjoint, use_inverse);
    } catch (...) {
      lc.st.swap(g->st);
      throw;
    }
    lc.st.swap(g->st);
    state(g->gens, g->epochs);
    return;
  }
  // second call with unchanged buffers: capture, instantiate, launch
  lc.st.swap(g->st);
  lc.st.begin();
  const int64_t l0 = lc.launches;
  for (Ctx* c : cs) c->capturing = true;
  cudaGraph_t graph = nullptr;
  bool ok = cudaStreamBeginCapture(lc.stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    try {
      solve_tree_sweeps(cs, xs, nrhs, adjoint, use_inverse);
    } catch (...) {
      ok = false;
    }
    ok = (cudaStreamEndCapture(lc.stream, &graph) == cudaSuccess) && ok;
  }
  for (Ctx* c : cs) c->capturing = false;
  lc.st.swap(g->st);
  if (ok && graph) ok = cudaGraphInstantiate(&g->exec, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  if (!ok) {
    // capture refused something: run the sweeps normally this time
    cudaGetLastError();
    if (g->exec) cudaGraphExecDestroy(g->exec);
    g->exec = nullptr;
    g->epochs.clear();
    lc.launches = l0;
    solve_tree_sweeps(cs, xs, nrhs, adjoint, use_inverse);
    return;
  }
  g->nlaunch = lc.launches - l0;
  ck(cudaGraphLaunch(g->exec, lc.stream), "graph launch");
}

void solve_tree(Ctx& c, void* xv, int nrhs, bool adjoint, bool use_inverse) {
  solve_tree_group({&c}, {xv}, nrhs, adjoint, use_inverse);
}

}  // namespace h2
