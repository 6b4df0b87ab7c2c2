// C ABI of libh2 (include/h2.h).  Every entry point converts internal errors
// into an h2_status and a per-context message; nothing throws across the ABI.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <functional>
#include <numeric>
#include <set>
#include <sstream>

#include "batch.h"

using namespace h2;
using namespace h2k;

struct h2_ctx {
  Ctx c;
  DevBuf tA, tB, tC, tR, hb, hx, invscale;
  DevBuf bpts, bsq, bflat, bG;  // construction scratch
};

namespace h2 {
Ctx* ctx_core(h2_ctx* x) { return &x->c; }
const double* ctx_invscale(h2_ctx* x) { return (const double*)x->invscale.p; }
}  // namespace h2

namespace {

thread_local std::string g_err;

h2_status guard(h2_ctx* ctx, const std::function<void()>& f) {
  try {
    if (ctx) ctx->c.err.clear();
    f();
    return H2_OK;
  } catch (const Err& e) {
    if (ctx) ctx->c.err = e.msg;
    g_err = e.msg;
    return e.st;
  } catch (const std::exception& e) {
    if (ctx) ctx->c.err = std::string("internal: ") + e.what();
    g_err = e.what();
    return H2_EINTERNAL;
  }
}

void finish_setup(h2_ctx* x, void* stream) {
  Ctx& c = x->c;
  c.stream = (cudaStream_t)stream;
  upload_h2(c);
  std::vector<double> inv(c.H.dscale.size());
  for (size_t i = 0; i < inv.size(); ++i) inv[i] = 1.0 / c.H.dscale[i];
  dev_ensure(c, x->invscale, inv.size() * sizeof(double));
  ck(cudaMemcpy(x->invscale.p, inv.data(), inv.size() * sizeof(double), cudaMemcpyHostToDevice), "upload");
}

// out (global) = A^{-1} in (global), A = S^{-1} Z S, S = diag(dscale)
void apply_Ainv(h2_ctx* x, const cd* in, cd* out, int nrhs, bool adj, bool inv) {
  Ctx& c = x->c;
  const int64_t N = c.H.tree.N;
  void* t = dev_ensure(c, x->tA, (size_t)N * nrhs * esz(c.prec));
  const double* sc = (const double*)c.dscale.p;
  const double* isc = (const double*)x->invscale.p;
  // Z (S x) = S b ; adjoint: Z^H (S^{-1} x) = S^{-1} b.  Block LDL^T factors
  // of the symmetric Z solve the adjoint as Z^{-H} r = conj(Z^{-1} conj(r)).
  const int cj = adj && c.fac_ldlt ? 1 : 0;
  ck(permute_scale(in, t, (const int64_t*)c.dperm.p, adj ? isc : sc, N, nrhs, P64, c.prec, 0, cj, c.stream),
     "permute in");
  solve_tree(c, t, nrhs, adj && !cj, inv);
  ck(permute_scale(t, out, (const int64_t*)c.dperm.p, adj ? sc : isc, N, nrhs, c.prec, P64, 1, cj, c.stream),
     "permute out");
}

void apply_A(h2_ctx* x, const cd* in, cd* out, int nrhs, bool adj) {
  Ctx& c = x->c;
  const int64_t N = c.H.tree.N;
  cd* t1 = (cd*)dev_ensure(c, x->tB, (size_t)N * nrhs * sizeof(cd));
  cd* t2 = (cd*)dev_ensure(c, x->tC, (size_t)N * nrhs * sizeof(cd));
  const double* sc = (const double*)c.dscale.p;
  const double* isc = (const double*)x->invscale.p;
  ck(permute_scale(in, t1, (const int64_t*)c.dperm.p, adj ? isc : sc, N, nrhs, P64, P64, 0, 0, c.stream), "perm");
  matvec_tree(c, t1, t2, nrhs, adj);
  ck(permute_scale(t2, out, (const int64_t*)c.dperm.p, adj ? sc : isc, N, nrhs, P64, P64, 1, 0, c.stream), "perm");
}

std::vector<double> col_norms(h2_ctx* x, const cd* v, int nrhs) {
  Ctx& c = x->c;
  double* d = (double*)dev_ensure(c, c.normbuf, (size_t)nrhs * sizeof(double) + 64);
  ck(col_norms2(v, c.H.tree.N, nrhs, d, c.stream), "norms");
  std::vector<double> h(nrhs);
  ck(cudaMemcpyAsync(h.data(), d, nrhs * sizeof(double), cudaMemcpyDeviceToHost, c.stream), "norms D2H");
  ck(cudaStreamSynchronize(c.stream), "norms sync");
  for (auto& v2 : h) v2 = std::sqrt(v2);
  return h;
}

// ---- groups of independent instances (h2_*_batch) ----------------------

std::vector<Ctx*> cores(const std::vector<h2_ctx*>& xs) {
  std::vector<Ctx*> cs;
  for (h2_ctx* x : xs) cs.push_back(&x->c);
  return cs;
}

// outs[q] = A_q^{-1} ins[q] for every instance, one launch per stage
void apply_Ainv_group(const std::vector<h2_ctx*>& xs, const std::vector<const cd*>& ins,
                      const std::vector<cd*>& outs, int nrhs, bool adj, bool inv) {
  Ctx& lc = xs[0]->c;
  std::vector<void*> ts;
  // block LDL^T factors: Z^{-H} r = conj(Z^{-1} conj(r)) (as apply_Ainv)
  for (h2_ctx* x : xs)
    if (x->c.fac_ldlt != lc.fac_ldlt) fail(H2_EINVAL, "instances factorized in different forms (ldlt)");
  const int cj = adj && lc.fac_ldlt ? 1 : 0;
  for (size_t q = 0; q < xs.size(); ++q) {
    Ctx& c = xs[q]->c;
    const int64_t N = c.H.tree.N;
    void* t = dev_ensure(c, xs[q]->tA, (size_t)N * nrhs * esz(c.prec));
    ck(permute_scale(ins[q], t, (const int64_t*)c.dperm.p,
                     adj ? (const double*)xs[q]->invscale.p : (const double*)c.dscale.p, N, nrhs, P64, c.prec, 0, cj,
                     lc.stream),
       "permute in");
    ts.push_back(t);
  }
  solve_tree_group(cores(xs), ts, nrhs, adj && !cj, inv);
  for (size_t q = 0; q < xs.size(); ++q) {
    Ctx& c = xs[q]->c;
    ck(permute_scale(ts[q], outs[q], (const int64_t*)c.dperm.p,
                     adj ? (const double*)c.dscale.p : (const double*)xs[q]->invscale.p, c.H.tree.N, nrhs, c.prec,
                     P64, 1, cj, lc.stream),
       "permute out");
  }
}

// outs[q] = A_q ins[q] (FP64 H^2 matvec) for every instance
void apply_A_group(const std::vector<h2_ctx*>& xs, const std::vector<const cd*>& ins, const std::vector<cd*>& outs,
                   int nrhs, bool adj) {
  Ctx& lc = xs[0]->c;
  std::vector<const cd*> t1s;
  std::vector<cd*> t2s;
  for (size_t q = 0; q < xs.size(); ++q) {
    Ctx& c = xs[q]->c;
    const int64_t N = c.H.tree.N;
    cd* t1 = (cd*)dev_ensure(c, xs[q]->tB, (size_t)N * nrhs * sizeof(cd));
    cd* t2 = (cd*)dev_ensure(c, xs[q]->tC, (size_t)N * nrhs * sizeof(cd));
    ck(permute_scale(ins[q], t1, (const int64_t*)c.dperm.p,
                     adj ? (const double*)xs[q]->invscale.p : (const double*)c.dscale.p, N, nrhs, P64, P64, 0, 0,
                     lc.stream),
       "perm");
    t1s.push_back(t1);
    t2s.push_back(t2);
  }
  matvec_tree_group(cores(xs), t1s, t2s, nrhs, adj);
  for (size_t q = 0; q < xs.size(); ++q) {
    Ctx& c = xs[q]->c;
    ck(permute_scale(t2s[q], outs[q], (const int64_t*)c.dperm.p,
                     adj ? (const double*)c.dscale.p : (const double*)xs[q]->invscale.p, c.H.tree.N, nrhs, P64, P64, 1,
                     0, lc.stream),
       "perm");
  }
}

// per-instance max over columns of ||v|| (one synchronize for the group)
std::vector<std::vector<double>> col_norms_group(const std::vector<h2_ctx*>& xs, const std::vector<const cd*>& vs,
                                                 int nrhs) {
  Ctx& lc = xs[0]->c;
  std::vector<std::vector<double>> h(xs.size(), std::vector<double>(nrhs));
  for (size_t q = 0; q < xs.size(); ++q) {
    Ctx& c = xs[q]->c;
    double* d = (double*)dev_ensure(c, c.normbuf, (size_t)nrhs * sizeof(double) + 64);
    ck(col_norms2(vs[q], c.H.tree.N, nrhs, d, lc.stream), "norms");
    ck(cudaMemcpyAsync(h[q].data(), d, nrhs * sizeof(double), cudaMemcpyDeviceToHost, lc.stream), "norms D2H");
  }
  ck(cudaStreamSynchronize(lc.stream), "norms sync");
  for (auto& v : h)
    for (auto& v2 : v) v2 = std::sqrt(v2);
  return h;
}

// Far-field sample Grams of one level on the GPU (kgram.cu).
void gpu_gram(h2_ctx* x, double k, double w, const std::vector<std::vector<int64_t>>& rows,
              const std::vector<std::vector<int64_t>>& ranges, std::vector<std::vector<cplx>>& G) {
  Ctx& c = x->c;
  const int nc = (int)rows.size();
  std::vector<int64_t> flat;
  std::vector<size_t> roff(nc), goff(nc);
  size_t gtot = 0;
  for (int t = 0; t < nc; ++t) {
    roff[t] = flat.size();
    flat.insert(flat.end(), rows[t].begin(), rows[t].end());
    flat.insert(flat.end(), ranges[t].begin(), ranges[t].end());
    goff[t] = gtot;
    gtot += rows[t].size() * rows[t].size();
  }
  G.assign(nc, {});
  if (gtot == 0) return;
  int64_t* dflat = (int64_t*)dev_ensure(c, x->bflat, flat.size() * sizeof(int64_t));
  ck(cudaMemcpy(dflat, flat.data(), flat.size() * sizeof(int64_t), cudaMemcpyHostToDevice), "gram rows");
  cd* dG = (cd*)dev_ensure(c, x->bG, gtot * sizeof(cd));
  std::vector<KGramTask> tasks;
  std::vector<KGramTile> tiles;
  std::vector<int> owner;
  for (int t = 0; t < nc; ++t) {
    const int nr = (int)rows[t].size();
    if (nr == 0) continue;
    tasks.push_back(KGramTask{dflat + roff[t], dflat + roff[t] + nr, dG + goff[t], nr, (int)ranges[t].size() / 2});
    owner.push_back(t);
    const int nt = (nr + 63) / 64;
    for (int tn = 0; tn < nt; ++tn)
      for (int tm = 0; tm <= tn; ++tm) tiles.push_back(KGramTile{(int)tasks.size() - 1, tm, tn});
  }
  ck(cudaStreamSynchronize(c.stream), "sync");
  c.st.begin();
  const int i0 = c.st.add(tasks), i1 = c.st.add(tiles);
  c.st.upload(c);
  ck(kernel_gram(c.st.ptr<KGramTask>(i0), c.st.ptr<KGramTile>(i1), (int)tiles.size(), (const double*)x->bpts.p,
                 (const double*)x->bsq.p, k, w, c.stream),
     "kernel gram");
  std::vector<cplx> hG(gtot);
  ck(cudaMemcpyAsync(hG.data(), dG, gtot * sizeof(cd), cudaMemcpyDeviceToHost, c.stream), "gram D2H");
  ck(cudaStreamSynchronize(c.stream), "gram sync");
  for (int t : owner) {
    const int nr = (int)rows[t].size();
    std::vector<cplx> g(hG.begin() + goff[t], hG.begin() + goff[t] + (size_t)nr * nr);
    for (int j = 0; j < nr; ++j)
      for (int i = j + 1; i < nr; ++i)
        if (i / 64 > j / 64) g[(size_t)i + (size_t)j * nr] = std::conj(g[(size_t)j + (size_t)i * nr]);
    G[t] = std::move(g);
  }
}

}  // namespace

extern "C" {

void h2_default_opts(h2_opts* o) {
  if (!o) return;
  o->leafsize = 64;
  o->eta = 1.0;
  o->sign = 1.0;
  o->ordering = H2_ORDER_COLORED;
  o->proxy_min = 0;
  o->proxy_radius = 3.0;
  o->arena_cap_bytes = 0;
  o->host_only = 0;
  o->profile = 0;
  o->apply_path = 0;
  o->solve_graph = 0;
  o->split_target = 0;
  o->cluster_max = 0;
  o->tile_policy = 0;
  o->tensor_cores = 2;
  o->gram_emulation = 1;
  o->eig_solver = 2;
  o->stop_level = 0;
  o->proxy_margin = 0.3;
  o->matvec_emulation = 1;
  o->ldlt = 2;
}

h2_status h2_set_opts(h2_ctx* ctx, const h2_opts* o) {
  if (!ctx || !o || o->apply_path < 0 || o->apply_path > 2 || o->split_target < 0 || o->cluster_max < 0 ||
      o->cluster_max > 16 || o->tile_policy < 0 || o->tile_policy > 1 || o->profile < 0 || o->profile > 2 ||
      o->tensor_cores < 0 || o->tensor_cores > 2 || o->gram_emulation < 0 || o->gram_emulation > 1 ||
      o->eig_solver < 0 || o->eig_solver > 2 || o->stop_level < 0 || o->matvec_emulation < 0 ||
      o->matvec_emulation > 2 || o->ldlt < 0 || o->ldlt > 2)
    return H2_EINVAL;
  h2_opts& c = ctx->c.opts;
  c.apply_path = o->apply_path;
  c.solve_graph = o->solve_graph;
  c.split_target = o->split_target;
  c.cluster_max = o->cluster_max;
  c.tile_policy = o->tile_policy;
  c.tensor_cores = o->tensor_cores;
  c.gram_emulation = o->gram_emulation;
  c.eig_solver = o->eig_solver;
  c.stop_level = o->stop_level;
  c.matvec_emulation = o->matvec_emulation;
  c.ldlt = o->ldlt;
  c.profile = o->profile;
  ctx->c.graphs.clear();
  return H2_OK;
}

const char* h2_status_string(int s) {
  switch (s) {
    case H2_OK: return "ok";
    case H2_EINVAL: return "invalid argument";
    case H2_ENOMEM: return "out of memory";
    case H2_ESINGULAR: return "singular pivot";
    case H2_ENOCONV: return "refinement did not converge";
    case H2_ETIMEOUT: return "device wait timed out";
    case H2_ECUDA: return "CUDA error";
    case H2_EINTERNAL: return "internal error";
    case H2_ESTATE: return "call out of order";
  }
  return "unknown status";
}

const char* h2_last_error(const h2_ctx* ctx) { return ctx ? ctx->c.err.c_str() : g_err.c_str(); }

h2_status h2_build(const double* pts, int64_t N, double k, double h, const double* chi, int64_t chi_len, double eps,
                   const h2_opts* opts, void* stream, h2_ctx** out) {
  if (!out) return H2_EINVAL;
  *out = nullptr;
  if (!pts || N <= 0 || !chi || !(chi_len == 1 || chi_len == N) || !(eps > 0) || !(k >= 0) || !(h > 0)) {
    g_err = "h2_build: bad argument";
    return H2_EINVAL;
  }
  h2_ctx* x = new h2_ctx();
  h2_default_opts(&x->c.opts);
  if (opts) x->c.opts = *opts;
  if (x->c.opts.leafsize < 1 || !(x->c.opts.eta > 0) || x->c.opts.tensor_cores < 0 || x->c.opts.tensor_cores > 2 ||
      x->c.opts.gram_emulation < 0 || x->c.opts.gram_emulation > 1 || x->c.opts.eig_solver < 0 ||
      x->c.opts.eig_solver > 2 || x->c.opts.stop_level < 0 || x->c.opts.matvec_emulation < 0 ||
      x->c.opts.matvec_emulation > 2 || x->c.opts.ldlt < 0 || x->c.opts.ldlt > 2) {
    delete x;
    g_err = "h2_build: bad options";
    return H2_EINVAL;
  }
  const h2_status st = guard(x, [&]() {
    const auto t0 = std::chrono::steady_clock::now();
    Ctx& c = x->c;
    c.stream = (cudaStream_t)stream;
    const double w = k * k * h * h * h / (4.0 * M_PI);
    std::vector<double> pts_tree, sq_tree;
    auto tree_arrays = [&]() {
      if (!pts_tree.empty()) return;
      const int64_t n = c.H.tree.N;
      pts_tree.resize(3 * n);
      sq_tree.resize(n);
      for (int64_t p = 0; p < n; ++p) {
        const int64_t g = c.H.tree.perm[p];
        for (int d = 0; d < 3; ++d) pts_tree[3 * p + d] = pts[3 * g + d];
        sq_tree[p] = c.H.dscale[g];
      }
      // proxy sample points (positions N, N + 1, ...) of the proxy construction
      pts_tree.insert(pts_tree.end(), c.H.proxy_pts.begin(), c.H.proxy_pts.end());
      sq_tree.insert(sq_tree.end(), c.H.proxy_w.begin(), c.H.proxy_w.end());
    };
    GramFn gram = [&](int, const std::vector<std::vector<int64_t>>& rows,
                      const std::vector<std::vector<int64_t>>& ranges, std::vector<std::vector<cplx>>& G) {
      tree_arrays();
      if (c.opts.host_only) {
        host_gram(pts_tree.data(), sq_tree.data(), k, w, rows, ranges, G);
        return;
      }
      if (!x->bpts.p) {
        dev_ensure(c, x->bpts, pts_tree.size() * sizeof(double));
        dev_ensure(c, x->bsq, sq_tree.size() * sizeof(double));
        ck(cudaMemcpy(x->bpts.p, pts_tree.data(), pts_tree.size() * sizeof(double), cudaMemcpyHostToDevice), "pts");
        ck(cudaMemcpy(x->bsq.p, sq_tree.data(), sq_tree.size() * sizeof(double), cudaMemcpyHostToDevice), "sq");
      }
      gpu_gram(x, k, w, rows, ranges, G);
    };
    const std::string e = build_h2(pts, N, k, h, chi, chi_len, eps, x->c.opts, x->c.H, gram);
    if (!e.empty()) fail(H2_EINVAL, e);
    x->c.H.symmetric = true;  // Z = I + s D^{1/2} K D^{1/2}
    if (!x->c.opts.host_only) finish_setup(x, stream);
    x->bpts.release();
    x->bsq.release();
    x->bflat.release();
    x->bG.release();
    x->c.stats.t_build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  });
  if (st != H2_OK) {
    g_err = x->c.err;
    delete x;
    return st;
  }
  *out = x;
  return H2_OK;
}

h2_status h2_load(int64_t N, int L, int l0, const int64_t* perm, const int64_t* leaf_size, const int64_t* rank,
                  const double* V, const double* T, const int64_t* n_adm, const int64_t* adm, const double* S,
                  int64_t n_near, const int64_t* near, const double* D, const double* dscale, const h2_opts* opts,
                  void* stream, h2_ctx** out) {
  if (!out) return H2_EINVAL;
  *out = nullptr;
  if (N <= 0 || L < 0 || l0 < 0 || l0 > L || L > 30 || !perm || !leaf_size || !rank || !n_adm || !near || !D) {
    g_err = "h2_load: bad argument";
    return H2_EINVAL;
  }
  h2_ctx* x = new h2_ctx();
  h2_default_opts(&x->c.opts);
  if (opts) x->c.opts = *opts;
  const h2_status st = guard(x, [&]() {
    H2Host& H = x->c.H;
    Tree& tr = H.tree;
    tr.N = N;
    tr.L = L;
    tr.perm.assign(perm, perm + N);
    {
      std::vector<char> seen(N, 0);
      for (int64_t p = 0; p < N; ++p) {
        if (perm[p] < 0 || perm[p] >= N || seen[perm[p]]) fail(H2_EINVAL, "perm is not a permutation");
        seen[perm[p]] = 1;
      }
    }
    tr.start.assign(L + 1, {});
    tr.size.assign(L + 1, {});
    int64_t s = 0;
    for (int c = 0; c < (1 << L); ++c) {
      if (leaf_size[c] < 0) fail(H2_EINVAL, "negative leaf size");
      tr.start[L].push_back(s);
      tr.size[L].push_back(leaf_size[c]);
      s += leaf_size[c];
    }
    if (s != N) fail(H2_EINVAL, "leaf sizes do not sum to N");
    for (int l = L - 1; l >= 0; --l)
      for (int c = 0; c < (1 << l); ++c) {
        tr.start[l].push_back(tr.start[l + 1][2 * c]);
        tr.size[l].push_back(tr.size[l + 1][2 * c] + tr.size[l + 1][2 * c + 1]);
      }
    H.L = L;
    H.l0 = l0;
    H.part.l0 = l0;
    H.part.adm.assign(L + 1, {});
    H.part.inad.assign(L + 1, {});
    H.rank.assign(L + 1, {});
    const int64_t* rk = rank;
    for (int l = l0; l <= L; ++l) {
      H.rank[l].assign(rk, rk + (1 << l));
      for (int v : H.rank[l])
        if (v < 0) fail(H2_EINVAL, "negative rank");
      rk += (1 << l);
    }
    // leaf bases
    H.V.assign(size_t(1) << L, {});
    const double* vp = V;
    for (int c = 0; c < (1 << L); ++c) {
      const size_t cnt = (size_t)tr.size[L][c] * H.rank[L][c];
      if (cnt && !V) fail(H2_EINVAL, "V missing");
      H.V[c].resize(cnt);
      for (size_t q = 0; q < cnt; ++q) H.V[c][q] = cplx(vp[2 * q], vp[2 * q + 1]);
      vp += 2 * cnt;
    }
    H.T.assign(L + 1, {});
    const double* tp = T;
    for (int l = l0; l < L; ++l) {
      H.T[l].assign(size_t(1) << l, {});
      for (int c = 0; c < (1 << l); ++c) {
        const size_t cnt = (size_t)(H.rank[l + 1][2 * c] + H.rank[l + 1][2 * c + 1]) * H.rank[l][c];
        if (cnt && !T) fail(H2_EINVAL, "T missing");
        H.T[l][c].resize(cnt);
        for (size_t q = 0; q < cnt; ++q) H.T[l][c][q] = cplx(tp[2 * q], tp[2 * q + 1]);
        tp += 2 * cnt;
      }
    }
    H.S.assign(L + 1, {});
    const int64_t* ap = adm;
    const double* sp = S;
    for (int l = l0; l <= L; ++l) {
      const int64_t na = n_adm[l - l0];
      for (int64_t q = 0; q < na; ++q) {
        const int t = (int)ap[2 * q], u = (int)ap[2 * q + 1];
        if (t < 0 || u < 0 || t >= (1 << l) || u >= (1 << l)) fail(H2_EINVAL, "admissible pair out of range");
        H.part.adm[l].push_back({t, u});
        const size_t cnt = (size_t)H.rank[l][t] * H.rank[l][u];
        std::vector<cplx> m(cnt);
        for (size_t e = 0; e < cnt; ++e) m[e] = cplx(sp[2 * e], sp[2 * e + 1]);
        sp += 2 * cnt;
        H.S[l].push_back(std::move(m));
      }
      ap += 2 * na;
    }
    const double* dp = D;
    for (int64_t q = 0; q < n_near; ++q) {
      const int t = (int)near[2 * q], u = (int)near[2 * q + 1];
      if (t < 0 || u < 0 || t >= (1 << L) || u >= (1 << L)) fail(H2_EINVAL, "near pair out of range");
      H.part.inad[L].push_back({t, u});
      const size_t cnt = (size_t)tr.size[L][t] * tr.size[L][u];
      std::vector<cplx> m(cnt);
      for (size_t e = 0; e < cnt; ++e) m[e] = cplx(dp[2 * e], dp[2 * e + 1]);
      dp += 2 * cnt;
      H.D.push_back(std::move(m));
    }
    for (int l = l0; l <= L; ++l) {
      // sort the admissible pairs and keep their couplings aligned
      std::vector<size_t> idx(H.part.adm[l].size());
      std::iota(idx.begin(), idx.end(), 0);
      std::sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return H.part.adm[l][a] < H.part.adm[l][b]; });
      std::vector<Pair> ap2;
      std::vector<std::vector<cplx>> S2;
      for (size_t q : idx) {
        ap2.push_back(H.part.adm[l][q]);
        S2.push_back(std::move(H.S[l][q]));
      }
      H.part.adm[l] = ap2;
      H.S[l] = std::move(S2);
    }
    {
      std::vector<size_t> idx(H.part.inad[L].size());
      std::iota(idx.begin(), idx.end(), 0);
      std::sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return H.part.inad[L][a] < H.part.inad[L][b]; });
      std::vector<Pair> np2;
      std::vector<std::vector<cplx>> D2;
      for (size_t q : idx) {
        np2.push_back(H.part.inad[L][q]);
        D2.push_back(std::move(H.D[q]));
      }
      H.part.inad[L] = np2;
      H.D = std::move(D2);
    }
    // inadmissible pairs above the leaves: parents of visited pairs
    for (int l = L - 1; l >= 0; --l) {
      std::set<Pair> ps;
      for (auto [a, b] : H.part.inad[l + 1]) ps.insert({a / 2, b / 2});
      if (l + 1 >= l0)
        for (auto [a, b] : H.part.adm[l + 1]) ps.insert({a / 2, b / 2});
      H.part.inad[l].assign(ps.begin(), ps.end());
    }
    // blocks must cover each entry exactly once (checked by block areas and
    // by the near / admissible lists being disjoint per level)
    {
      double area = 0;
      for (int l = 0; l <= L; ++l) {
        std::set<Pair> a(H.part.adm[l].begin(), H.part.adm[l].end());
        if (a.size() != H.part.adm[l].size()) fail(H2_EINVAL, "duplicate admissible pair");
        for (auto [t, u] : H.part.adm[l]) area += (double)tr.size[l][t] * tr.size[l][u];
      }
      std::set<Pair> nr(H.part.inad[L].begin(), H.part.inad[L].end());
      if (nr.size() != H.part.inad[L].size()) fail(H2_EINVAL, "duplicate near pair");
      for (auto [t, u] : H.part.inad[L]) area += (double)tr.size[L][t] * tr.size[L][u];
      if (area != (double)N * (double)N) fail(H2_EINVAL, "blocks do not partition the matrix");
      for (int l = 0; l <= L; ++l)
        for (auto pr : H.part.adm[l])
          if (std::binary_search(H.part.inad[l].begin(), H.part.inad[l].end(), pr))
            fail(H2_EINVAL, "pair both admissible and inadmissible");
      for (int l = 0; l < l0; ++l)
        if (!H.part.adm[l].empty()) fail(H2_EINVAL, "admissible pair above l0");
    }
    // symmetric iff every admissible and near block equals the transpose of
    // its mirror block
    {
      bool sym = true;
      for (int l = l0; l <= L && sym; ++l)
        for (size_t q = 0; q < H.part.adm[l].size() && sym; ++q) {
          const auto [t, u] = H.part.adm[l][q];
          const auto it = std::lower_bound(H.part.adm[l].begin(), H.part.adm[l].end(), Pair{u, t});
          if (it == H.part.adm[l].end() || *it != Pair{u, t}) { sym = false; break; }
          const auto& A = H.S[l][q];
          const auto& B = H.S[l][it - H.part.adm[l].begin()];
          const int kt = H.rank[l][t], ku = H.rank[l][u];
          double nrm = 0, dif = 0;
          for (int i = 0; i < kt; ++i)
            for (int j = 0; j < ku; ++j) {
              nrm += std::norm(A[(size_t)i + (size_t)j * kt]);
              dif += std::norm(A[(size_t)i + (size_t)j * kt] - B[(size_t)j + (size_t)i * ku]);
            }
          if (dif > 1e-24 * nrm) sym = false;
        }
      for (size_t q = 0; q < H.part.inad[L].size() && sym; ++q) {
        const auto [t, u] = H.part.inad[L][q];
        const auto it = std::lower_bound(H.part.inad[L].begin(), H.part.inad[L].end(), Pair{u, t});
        if (it == H.part.inad[L].end() || *it != Pair{u, t}) { sym = false; break; }
        const auto& A = H.D[q];
        const auto& B = H.D[it - H.part.inad[L].begin()];
        const int nt = (int)tr.size[L][t], nu = (int)tr.size[L][u];
        double nrm = 0, dif = 0;
        for (int i = 0; i < nt; ++i)
          for (int j = 0; j < nu; ++j) {
            nrm += std::norm(A[(size_t)i + (size_t)j * nt]);
            dif += std::norm(A[(size_t)i + (size_t)j * nt] - B[(size_t)j + (size_t)i * nu]);
          }
        if (dif > 1e-24 * nrm) sym = false;
      }
      H.symmetric = sym;
    }
    H.dscale.assign(N, 1.0);
    if (dscale)
      for (int64_t i = 0; i < N; ++i) {
        if (!(dscale[i] > 0)) fail(H2_EINVAL, "dscale must be > 0");
        H.dscale[i] = dscale[i];
      }
    finish_setup(x, stream);
  });
  if (st != H2_OK) {
    g_err = x->c.err;
    delete x;
    return st;
  }
  *out = x;
  return H2_OK;
}

h2_status h2_export_sizes(const h2_ctx* ctx, int64_t* N, int* L, int* l0, int64_t* nV, int64_t* nT, int64_t* nS,
                          int64_t* n_adm_total, int64_t* n_near, int64_t* nD) {
  if (!ctx) return H2_EINVAL;
  const H2Host& H = ctx->c.H;
  int64_t v = 0, t = 0, s = 0, na = 0, d = 0;
  for (const auto& a : H.V) v += (int64_t)a.size();
  for (int l = H.l0; l < H.L; ++l)
    for (const auto& a : H.T[l]) t += (int64_t)a.size();
  for (int l = H.l0; l <= H.L; ++l) {
    na += (int64_t)H.part.adm[l].size();
    for (const auto& a : H.S[l]) s += (int64_t)a.size();
  }
  for (const auto& a : H.D) d += (int64_t)a.size();
  if (N) *N = H.tree.N;
  if (L) *L = H.L;
  if (l0) *l0 = H.l0;
  if (nV) *nV = v;
  if (nT) *nT = t;
  if (nS) *nS = s;
  if (n_adm_total) *n_adm_total = na;
  if (n_near) *n_near = (int64_t)H.part.inad[H.L].size();
  if (nD) *nD = d;
  return H2_OK;
}

h2_status h2_export(const h2_ctx* ctx, int64_t* perm, int64_t* leaf_size, int64_t* rank, double* V, double* T,
                    int64_t* n_adm, int64_t* adm, double* S, int64_t* near, double* D, double* dscale) {
  if (!ctx) return H2_EINVAL;
  const H2Host& H = ctx->c.H;
  auto put = [](double*& p, const std::vector<cplx>& a) {
    for (const cplx& z : a) {
      *p++ = z.real();
      *p++ = z.imag();
    }
  };
  if (perm) std::copy(H.tree.perm.begin(), H.tree.perm.end(), perm);
  if (leaf_size) std::copy(H.tree.size[H.L].begin(), H.tree.size[H.L].end(), leaf_size);
  if (rank)
    for (int l = H.l0; l <= H.L; ++l)
      for (int v : H.rank[l]) *rank++ = v;
  if (V)
    for (const auto& a : H.V) put(V, a);
  if (T)
    for (int l = H.l0; l < H.L; ++l)
      for (const auto& a : H.T[l]) put(T, a);
  for (int l = H.l0; l <= H.L; ++l) {
    if (n_adm) n_adm[l - H.l0] = (int64_t)H.part.adm[l].size();
    if (adm)
      for (auto [a, b] : H.part.adm[l]) {
        *adm++ = a;
        *adm++ = b;
      }
    if (S)
      for (const auto& a : H.S[l]) put(S, a);
  }
  if (near)
    for (auto [a, b] : H.part.inad[H.L]) {
      *near++ = a;
      *near++ = b;
    }
  if (D)
    for (const auto& a : H.D) put(D, a);
  if (dscale) std::copy(H.dscale.begin(), H.dscale.end(), dscale);
  return H2_OK;
}

static bool host_only(h2_ctx* ctx) {
  if (ctx->c.opts.host_only) {
    ctx->c.err = "context was built with host_only";
    return true;
  }
  return false;
}

h2_status h2_factorize(h2_ctx* ctx, double eps_fill, int prec) {
  if (!ctx) return H2_EINVAL;
  if (host_only(ctx)) return H2_ESTATE;
  if (!(eps_fill >= 0) || (prec != H2_FP64 && prec != H2_MIXED)) {
    ctx->c.err = "h2_factorize: bad argument";
    return H2_EINVAL;
  }
  return guard(ctx, [&]() {
    try {
      factorize(ctx->c, eps_fill, prec == H2_FP64 ? P64 : P32);
    } catch (...) {
      drop_factors(ctx->c);
      throw;
    }
  });
}

h2_status h2_invert(h2_ctx* ctx) {
  if (!ctx) return H2_EINVAL;
  if (host_only(ctx)) return H2_ESTATE;
  return guard(ctx, [&]() { invert(ctx->c); });
}

h2_status h2_solve(h2_ctx* ctx, const void* b, void* xo, int nrhs, unsigned flags, double tol, int max_iter, int* iters,
                   double* resid, void* stream) {
  if (!ctx) return H2_EINVAL;
  if (host_only(ctx)) return H2_ESTATE;
  if (!b || !xo || nrhs <= 0 || (flags & ~15u)) {
    ctx->c.err = "h2_solve: bad argument";
    return H2_EINVAL;
  }
  if (iters) *iters = 0;
  if (resid) *resid = -1;
  h2_status conv = H2_OK;
  const h2_status st = guard(ctx, [&]() {
    Ctx& c = ctx->c;
    if (!c.factored) fail(H2_ESTATE, "h2_solve before h2_factorize");
    if ((flags & H2_USE_INVERSE) && !c.inverted) fail(H2_ESTATE, "H2_USE_INVERSE before h2_invert");
    if ((flags & H2_USE_INVERSE) && (flags & H2_ADJOINT)) fail(H2_EINVAL, "H2_USE_INVERSE with H2_ADJOINT");
    c.stream = (cudaStream_t)stream;
    const auto t0 = std::chrono::steady_clock::now();
    const int64_t l0 = c.launches;
    ck(cudaStreamSynchronize(c.stream), "sync");
    c.st.begin();
    const int64_t N = c.H.tree.N;
    const size_t bytes = (size_t)N * nrhs * sizeof(cd);
    const cd* db = (const cd*)b;
    cd* dx = (cd*)xo;
    if (flags & H2_HOST) {
      db = (const cd*)dev_ensure(c, ctx->hb, bytes);
      dx = (cd*)dev_ensure(c, ctx->hx, bytes);
      ck(cudaMemcpyAsync((void*)db, b, bytes, cudaMemcpyHostToDevice, c.stream), "b H2D");
    }
    const bool adj = flags & H2_ADJOINT, inv = flags & H2_USE_INVERSE;
    if (!(flags & H2_REFINE)) {
      apply_Ainv(ctx, db, dx, nrhs, adj, inv);
    } else {
      cd* r = (cd*)dev_ensure(c, ctx->tR, bytes);
      cd* dxx = dx;
      if (dx == db) {  // x aliases b: keep a copy of b for the residual
        cd* bc = (cd*)dev_ensure(c, ctx->hb, bytes);
        ck(cudaMemcpyAsync(bc, db, bytes, cudaMemcpyDeviceToDevice, c.stream), "copy b");
        db = bc;
      }
      apply_Ainv(ctx, db, dxx, nrhs, adj, inv);
      const std::vector<double> nb = col_norms(ctx, db, nrhs);
      int it = 0;
      double rel = 0;
      const bool emul = c.opts.matvec_emulation >= 1 && tol >= 1e-11;
      for (;;) {
        {
          // the residual's products in double-float (h2_opts.matvec_emulation)
          MvEmul me(c, emul);
          apply_A(ctx, dxx, r, nrhs, adj);
        }
        ck(axpby(db, r, r, (int64_t)N * nrhs, 1.0, -1.0, c.stream), "residual");
        const std::vector<double> nr = col_norms(ctx, r, nrhs);
        rel = 0;
        for (int q = 0; q < nrhs; ++q) rel = std::max(rel, nb[q] > 0 ? nr[q] / nb[q] : nr[q]);
        if (rel <= tol || it >= max_iter) break;
        // correction: x += A^{-1} r  (r is overwritten by the correction)
        apply_Ainv(ctx, r, r, nrhs, adj, inv);
        ck(axpby(dxx, r, dxx, (int64_t)N * nrhs, 1.0, 1.0, c.stream), "update");
        ++it;
      }
      if (iters) *iters = it;
      if (resid) *resid = rel;
      c.stats.refine_iters = it;
      c.stats.refine_resid = rel;
      if (rel > tol) conv = H2_ENOCONV;
    }
    if (flags & H2_HOST) ck(cudaMemcpyAsync(xo, dx, bytes, cudaMemcpyDeviceToHost, c.stream), "x D2H");
    ck(cudaStreamSynchronize(c.stream), "solve sync");
    prof_resolve(c);
    c.stats.launches_solve = c.launches - l0;
    c.stats.t_solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  });
  if (st == H2_OK && conv != H2_OK) {
    ctx->c.err = "refinement stopped above the tolerance";
    return conv;
  }
  return st;
}

// Validates a group argument: count > 0, distinct GPU contexts.
static bool group_ok(h2_ctx* const* ctxs, int count, std::vector<h2_ctx*>& xs) {
  if (!ctxs || count <= 0) return false;
  std::set<h2_ctx*> seen;
  for (int q = 0; q < count; ++q) {
    if (!ctxs[q] || ctxs[q]->c.opts.host_only || !seen.insert(ctxs[q]).second) return false;
    xs.push_back(ctxs[q]);
  }
  return true;
}

h2_status h2_factorize_batch(h2_ctx* const* ctxs, int count, double eps_fill, int prec) {
  std::vector<h2_ctx*> xs;
  if (!group_ok(ctxs, count, xs)) return H2_EINVAL;
  if (!(eps_fill >= 0) || (prec != H2_FP64 && prec != H2_MIXED)) {
    xs[0]->c.err = "h2_factorize_batch: bad argument";
    return H2_EINVAL;
  }
  std::vector<cudaStream_t> own;
  for (h2_ctx* x : xs) own.push_back(x->c.stream);
  const h2_status st = guard(xs[0], [&]() {
    try {
      factorize_group(cores(xs), eps_fill, prec == H2_FP64 ? P64 : P32);
    } catch (...) {
      for (h2_ctx* x : xs) drop_factors(x->c);
      throw;
    }
  });
  for (size_t q = 0; q < xs.size(); ++q) {
    xs[q]->c.stream = own[q];
    if (st != H2_OK && q > 0) xs[q]->c.err = "h2_factorize_batch failed: " + xs[0]->c.err;
  }
  return st;
}

h2_status h2_solve_batch(h2_ctx* const* ctxs, int count, const void* const* b, void* const* xo, int nrhs,
                         unsigned flags, double tol, int max_iter, int* iters, double* resid, void* stream) {
  std::vector<h2_ctx*> xs;
  if (!group_ok(ctxs, count, xs) || !b || !xo || nrhs <= 0 || (flags & ~7u)) return H2_EINVAL;
  for (int q = 0; q < count; ++q)
    if (!b[q] || !xo[q]) return H2_EINVAL;
  if (iters) *iters = 0;
  if (resid) *resid = -1;
  h2_status conv = H2_OK;
  const h2_status st = guard(xs[0], [&]() {
    const bool adj = flags & H2_ADJOINT, inv = flags & H2_USE_INVERSE;
    if (inv && adj) fail(H2_EINVAL, "H2_USE_INVERSE with H2_ADJOINT");
    for (h2_ctx* x : xs) {
      if (!x->c.factored) fail(H2_ESTATE, "h2_solve_batch before factorization");
      if (inv && !x->c.inverted) fail(H2_ESTATE, "H2_USE_INVERSE before h2_invert");
      x->c.stream = (cudaStream_t)stream;
    }
    Ctx& lc = xs[0]->c;
    const auto t0 = std::chrono::steady_clock::now();
    const int64_t l0 = lc.launches;
    ck(cudaStreamSynchronize(lc.stream), "sync");
    for (h2_ctx* x : xs) x->c.st.begin();
    std::vector<const cd*> db;
    std::vector<cd*> dx;
    for (int q = 0; q < count; ++q) {
      db.push_back((const cd*)b[q]);
      dx.push_back((cd*)xo[q]);
    }
    if (!(flags & H2_REFINE)) {
      apply_Ainv_group(xs, db, dx, nrhs, adj, inv);
    } else {
      std::vector<cd*> r;
      for (int q = 0; q < count; ++q) {
        Ctx& c = xs[q]->c;
        const size_t bytes = (size_t)c.H.tree.N * nrhs * sizeof(cd);
        r.push_back((cd*)dev_ensure(c, xs[q]->tR, bytes));
        if (dx[q] == db[q]) {  // x aliases b: keep a copy of b for the residual
          cd* bc = (cd*)dev_ensure(c, xs[q]->hb, bytes);
          ck(cudaMemcpyAsync(bc, db[q], bytes, cudaMemcpyDeviceToDevice, lc.stream), "copy b");
          db[q] = bc;
        }
      }
      apply_Ainv_group(xs, db, dx, nrhs, adj, inv);
      const auto nb = col_norms_group(xs, db, nrhs);
      int it = 0;
      double rel = 0;
      std::vector<const cd*> cx(dx.begin(), dx.end()), cr(r.begin(), r.end());
      const bool emul = lc.opts.matvec_emulation >= 1 && tol >= 1e-11;
      for (;;) {
        {
          MvEmul me(lc, emul);
          apply_A_group(xs, cx, r, nrhs, adj);
        }
        for (int q = 0; q < count; ++q)
          ck(axpby(db[q], r[q], r[q], xs[q]->c.H.tree.N * (int64_t)nrhs, 1.0, -1.0, lc.stream), "residual");
        const auto nr = col_norms_group(xs, cr, nrhs);
        rel = 0;
        for (int q = 0; q < count; ++q)
          for (int k = 0; k < nrhs; ++k) rel = std::max(rel, nb[q][k] > 0 ? nr[q][k] / nb[q][k] : nr[q][k]);
        if (rel <= tol || it >= max_iter) break;
        apply_Ainv_group(xs, cr, r, nrhs, adj, inv);
        for (int q = 0; q < count; ++q)
          ck(axpby(dx[q], r[q], dx[q], xs[q]->c.H.tree.N * (int64_t)nrhs, 1.0, 1.0, lc.stream), "update");
        ++it;
      }
      if (iters) *iters = it;
      if (resid) *resid = rel;
      if (rel > tol) conv = H2_ENOCONV;
    }
    ck(cudaStreamSynchronize(lc.stream), "solve sync");
    prof_resolve(lc);
    lc.stats.launches_solve = lc.launches - l0;
    lc.stats.t_solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  });
  if (st == H2_OK && conv != H2_OK) {
    xs[0]->c.err = "refinement stopped above the tolerance";
    return conv;
  }
  return st;
}

h2_status h2_matvec(h2_ctx* ctx, const void* xi, void* y, int nrhs, unsigned flags, void* stream) {
  if (!ctx) return H2_EINVAL;
  if (host_only(ctx)) return H2_ESTATE;
  if (!xi || !y || nrhs <= 0 || xi == y || (flags & ~(H2_ADJOINT | H2_HOST))) {
    ctx->c.err = "h2_matvec: bad argument";
    return H2_EINVAL;
  }
  return guard(ctx, [&]() {
    Ctx& c = ctx->c;
    c.stream = (cudaStream_t)stream;
    ck(cudaStreamSynchronize(c.stream), "sync");
    c.st.begin();
    const size_t bytes = (size_t)c.H.tree.N * nrhs * sizeof(cd);
    const cd* dx = (const cd*)xi;
    cd* dy = (cd*)y;
    if (flags & H2_HOST) {
      dx = (const cd*)dev_ensure(c, ctx->hb, bytes);
      dy = (cd*)dev_ensure(c, ctx->hx, bytes);
      ck(cudaMemcpyAsync((void*)dx, xi, bytes, cudaMemcpyHostToDevice, c.stream), "x H2D");
    }
    MvEmul me(c, c.opts.matvec_emulation == 2);
    apply_A(ctx, dx, dy, nrhs, flags & H2_ADJOINT);
    if (flags & H2_HOST) ck(cudaMemcpyAsync(y, dy, bytes, cudaMemcpyDeviceToHost, c.stream), "y D2H");
    ck(cudaStreamSynchronize(c.stream), "matvec sync");
    prof_resolve(c);
  });
}

h2_status h2_grad_chi(h2_ctx* ctx, const void* x, const void* mu, const void* g, int nrhs, double alpha,
                      double* grad, unsigned flags, void* stream) {
  if (!ctx) return H2_EINVAL;
  if (host_only(ctx)) return H2_ESTATE;
  if (!x || !mu || !grad || nrhs <= 0 || (flags & ~H2_GRAD_ACCUMULATE)) {
    ctx->c.err = "h2_grad_chi: bad argument (device x, mu, grad; nrhs > 0; flags 0 or H2_GRAD_ACCUMULATE)";
    return H2_EINVAL;
  }
  return guard(ctx, [&]() {
    Ctx& c = ctx->c;
    ck(grad_chi((const cd*)x, (const cd*)mu, (const cd*)g, (const double*)c.dscale.p, c.H.tree.N, nrhs, alpha, grad,
                (flags & H2_GRAD_ACCUMULATE) ? 1 : 0, (cudaStream_t)stream),
       "grad_chi");
    c.launches++;
  });
}

h2_status h2_set_chi(h2_ctx* ctx, const double* chi, int64_t chi_len) {
  if (!ctx) return H2_EINVAL;
  const int64_t N = ctx->c.H.tree.N;
  if (!chi || !(chi_len == 1 || chi_len == N)) {
    ctx->c.err = "h2_set_chi: bad argument (chi_len must be 1 or N)";
    return H2_EINVAL;
  }
  for (int64_t i = 0; i < chi_len; ++i)
    if (!(chi[i] > 0) || !std::isfinite(chi[i])) {
      ctx->c.err = "h2_set_chi: chi must be finite and > 0 for every cell";
      return H2_EINVAL;
    }
  return guard(ctx, [&]() {
    Ctx& c = ctx->c;
    H2Host& H = c.H;
    std::vector<double> sq(N), e(N);
    for (int64_t g = 0; g < N; ++g) sq[g] = std::sqrt(chi_len == 1 ? chi[0] : chi[g]);
    for (int64_t p = 0; p < N; ++p) {
      const int64_t g = H.tree.perm[p];
      e[p] = sq[g] / H.dscale[g];
    }
    // the factors and everything derived from the old matrix are void from here on
    c.factored = false;
    c.inverted = false;
    c.epoch++;
    c.graphs.clear();
    c.snorm2_cache.clear();
    c.cov_level = -1;
    rescale_h2(H, e);
    H.dscale = sq;
    if (!c.opts.host_only) finish_setup(ctx, c.stream);
  });
}

h2_status h2_level_ranks(const h2_ctx* ctx, int level, int* k0, int* kt, int64_t n) {
  if (!ctx) return H2_EINVAL;
  const Ctx& c = ctx->c;
  for (const LevelF& F : c.lev)
    if (F.l == level) {
      if (n < F.nc) return H2_EINVAL;
      for (int i = 0; i < F.nc; ++i) {
        if (k0) k0[i] = F.k0[i];
        if (kt) kt[i] = F.kt[i];
      }
      return c.factored ? H2_OK : H2_ESTATE;
    }
  return c.factored ? H2_EINVAL : H2_ESTATE;
}

h2_status h2_stats(const h2_ctx* ctx, char* json, size_t cap) {
  if (!ctx || !json || cap == 0) return H2_EINVAL;
  const Ctx& c = ctx->c;
  std::ostringstream o;
  o.precision(10);
  o << "{\"N\":" << c.H.tree.N << ",\"L\":" << c.H.L << ",\"l0\":" << c.H.l0 << ",\"factored\":" << (c.factored ? 1 : 0)
    << ",\"prec\":\"" << (c.prec == P64 ? "fp64" : "mixed") << "\",\"eps_fill\":" << c.eps_fill
    << ",\"stop_level\":" << c.stats.stop_level << ",\"t_build_ms\":" << c.stats.t_build_ms
    << ",\"t_build_phases_ms\":{\"gram\":" << c.H.t_gram_ms << ",\"id\":" << c.H.t_id_ms
    << ",\"couplings\":" << c.H.t_coupling_ms << ",\"near\":" << c.H.t_near_ms << "}"
    << ",\"t_factor_ms\":" << c.stats.t_factor_ms
    << ",\"t_solve_ms\":" << c.stats.t_solve_ms << ",\"t_factor_sync_ms\":" << c.stats.t_sync_ms
    << ",\"flops_factor\":" << c.stats.flops_factor
    << ",\"launches_factor\":" << c.stats.launches_factor << ",\"launches_solve\":" << c.stats.launches_solve
    << ",\"refine_iters\":" << c.stats.refine_iters << ",\"refine_resid\":" << c.stats.refine_resid
    << ",\"symmetric\":" << (c.H.symmetric ? 1 : 0) << ",\"ldlt\":" << (c.fac_ldlt ? 1 : 0) << ",\"dev_bytes\":" << c.dev_bytes << ",\"dev_peak\":" << c.dev_peak << ",\"root_n\":" << c.root.n
    << ",\"build_rank_max\":[";
  for (int l = c.H.l0; l <= c.H.L; ++l) {
    int mx = 0;
    for (int v : c.H.rank[l]) mx = std::max(mx, v);
    o << (l > c.H.l0 ? "," : "") << mx;
  }
  o << "],\"mem\":{";
  {
    // device bytes by kind: the H^2 matrix (FP64), the factors kept for the
    // solves, the per-level working arenas, and other scratch
    size_t h2 = 0, kept = 0, work = 0;
    for (const DevBuf* b : {&c.dV, &c.dT, &c.dS, &c.dD, &c.dperm, &c.dscale, &c.dVp, &c.dTp}) h2 += b->bytes;
    for (const LevelF& F : c.lev)
      for (const DevBuf* b : {&F.near_buf, &F.Q_buf, &F.inv_buf, &F.piv_buf, &F.Ub_buf}) kept += b->bytes;
    for (const DevBuf* b : {&c.root.R, &c.root.piv, &c.root.Linv, &c.root.Uinv, &c.root.Rinv}) kept += b->bytes;
    for (const DevBuf* b : {&c.fill_pp[0], &c.fill_pp[1], &c.B_pp[0], &c.B_pp[1], &c.Vp_pp[0], &c.Vp_pp[1]})
      work += b->bytes;
    size_t near_bytes = 0;
    for (const LevelF& F : c.lev) near_bytes += F.near_elems * esz(c.prec);
    o << "\"h2\":" << h2 << ",\"factors\":" << kept << ",\"level_work\":" << work
      << ",\"near_blocks\":" << near_bytes
      << ",\"other\":" << (c.dev_bytes > h2 + kept + work ? c.dev_bytes - h2 - kept - work : 0);
  }
  o << "},\"levels\":[";
  for (size_t li = 0; li < c.lev.size(); ++li) {
    const LevelF& F = c.lev[li];
    int nmax = 0, k0max = 0, ktmax = 0, pushed = 0, live = 0, csp = 0, csp_fill = 0;
    long msum = 0;
    {
      // C_sp (Sec. V, Table IV): most blocks in one block row of the level,
      // near + admissible, and with the pushed fill-in targets
      std::vector<int> rowc(F.nc, 0), rowf(F.nc, 0);
      for (int i = 0; i < F.nc; ++i) rowc[i] = (int)F.nbrs[i].size();
      for (auto pr : c.H.part.adm[F.l]) rowc[pr.first]++;
      for (size_t q = 0; q < F.fill_pairs.size(); ++q)
        if (F.fill_live[q] && !F.fill_is_adm[q]) rowf[F.fill_pairs[q].first]++;
      for (int i = 0; i < F.nc; ++i) {
        csp = std::max(csp, rowc[i]);
        csp_fill = std::max(csp_fill, rowc[i] + rowf[i]);
      }
    }
    for (int i = 0; i < F.nc; ++i) {
      nmax = std::max(nmax, F.n[i]);
      k0max = std::max(k0max, F.k0[i]);
      ktmax = std::max(ktmax, F.kt[i]);
      msum += F.m[i];
    }
    for (size_t q = 0; q < F.fill_pairs.size(); ++q) {
      live += F.fill_live[q];
      pushed += F.fill_live[q] && !F.fill_is_adm[q];
    }
    o << (li ? "," : "") << "{\"l\":" << F.l << ",\"clusters\":" << F.nc << ",\"n_max\":" << nmax
      << ",\"k0_max\":" << k0max << ",\"kt_max\":" << ktmax << ",\"eliminated\":" << msum
      << ",\"batches\":" << F.batches.size() << ",\"near\":" << F.near_pairs.size()
      << ",\"adm\":" << c.H.part.adm[F.l].size() << ",\"fill_live\":" << live << ",\"pushed_live\":" << pushed
      << ",\"ritz_max\":" << F.st_ritz_max << ",\"ritz_mean\":" << (F.st_ritz_n ? (double)F.st_ritz_sum / F.st_ritz_n : 0.0)
      << ",\"jacobi_sweeps_max\":" << F.st_sweeps_max << ",\"csp\":" << csp << ",\"csp_fill\":" << csp_fill << "}";
  }
  o << "],\"kernels\":{";
  {
    bool first = true;
    for (const auto& [tag, a] : c.prof) {
      o << (first ? "" : ",") << "\"" << tag << "\":{\"launches\":" << a.launches << ",\"ms\":" << a.ms
        << ",\"flops\":" << a.flops << ",\"bytes\":" << a.bytes;
      if (a.pipe) o << ",\"pipe\":\"" << a.pipe << "\"";
      o << "}";
      first = false;
    }
  }
  o << "},\"paths\":{";
  {
    bool first = true;
    for (const auto& [k, v] : c.paths) {
      o << (first ? "" : ",") << "\"" << k << "\":" << v;
      first = false;
    }
  }
  o << "}}";
  const std::string s = o.str();
  const size_t n = std::min(cap - 1, s.size());
  std::memcpy(json, s.data(), n);
  json[n] = 0;
  return s.size() < cap ? H2_OK : H2_EINVAL;
}

void h2_destroy(h2_ctx* ctx) { delete ctx; }

}  // extern "C"
